"""FP64 CPU oracle of the ptychography cycle (AP, DM, LLK, ML gradient; far and near field).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline legs of ``bench.py``, never by the product package.  It shares
no code with the CUDA path.  See ``oracle/ptycho.py`` for the operators, the
paper passages they follow and the readings taken where the paper is silent.
"""
from .ptycho import *  # noqa: F401,F403
from .ptycho import unit_count  # noqa: F401
