"""libptycho: the far-field ptychography projection cycle (AP, DM, Poisson LLK
and its gradient) as hand-written CUDA for NVIDIA GB300 (sm_103a), behind the
C ABI of ``include/ptycho.h``, with a thin PyTorch-facing binding.

The method is that of the PyNX paper (Favre-Nicolin et al., 2020): the
ptychography operators ObjProbe2Psi, FT/IFT, ApplyAmplitude, Psi2ObjProbe, AP,
DM, LLK and ML (Section 4 and the appendix operator table).
"""
import importlib

from ._lib import PtychoError, SUPPORTED_SIZES, load  # noqa: F401

_LAZY = ("Ptycho", "PtychoBatch", "PtychoLLK", "fft2", "counts_to_float", "encode_counts8", "counts8_to_float",
         "fma_tflops")


def __getattr__(name):
    # the torch-facing API is imported on first use
    if name in _LAZY:
        mod = importlib.import_module(__name__ + ".ptycho")
        return getattr(mod, name)
    raise AttributeError(name)
