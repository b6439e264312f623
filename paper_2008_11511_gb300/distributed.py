"""Data-parallel split of one ptychography problem over several GPUs.

Frames are independent within a cycle, so the positions can be sharded across
ranks; the only exchange per cycle is the sum of the Psi2ObjProbe numerators
and denominators (object: Ho x Wo x {Re N_O, Im N_O, D_O, 0}; probe:
K x N x N x {Re N_P, Im N_P, D_P, 0}) and of the log-likelihood.  Every rank
then normalises the same sums, so O and P stay identical on all ranks.

The paper's own multi-GPU mode (PtychoSplit, Section 4) instead runs the parts
asynchronously and stitches them at the end; this module provides the
synchronous form, whose result equals the single-GPU cycle.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def split_positions(positions, world: int, rank: int) -> np.ndarray:
    """Indices of the frames owned by ``rank``: positions sorted by (row, col) and
    cut into ``world`` contiguous, nearly equal spatial blocks."""
    pos = np.asarray(positions)
    order = np.lexsort((pos[:, 1], pos[:, 0]))
    return np.sort(np.array_split(order, world)[rank])


def allreduce_accumulators(acc_obj: torch.Tensor | None, acc_probe: torch.Tensor | None,
                           llk: torch.Tensor | None = None, group=None):
    """Sum the given packed accumulators (and the LLK) over all ranks in place."""
    for t in (acc_obj, acc_probe, llk):
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


def _overlap_update_split(pb, update_obj, update_probe, llk, group):
    """Probe stage on the summed probe accumulator, object gather of this rank's
    frames, all-reduce of the object accumulator, object stage."""
    from .ptycho import PTX_STAGE_OBJ_GATHER, PTX_STAGE_OBJ_NORMALISE, PTX_STAGE_PROBE
    acc_o, acc_p = pb.accumulators()
    allreduce_accumulators(None, acc_p if update_probe else None, llk, group=group)
    st = (PTX_STAGE_PROBE if update_probe else 0) | (PTX_STAGE_OBJ_GATHER if update_obj else 0)
    if st:
        pb.normalise(stages=st)
    if update_obj:
        allreduce_accumulators(acc_o, None, group=group)
        pb.normalise(stages=PTX_STAGE_OBJ_NORMALISE)


def dm_cycles_data_parallel(pb, ncycles: int, update_obj=True, update_probe=True, init_psi=False, group=None):
    """DM cycles of a Ptycho that holds this rank's frames only: the cycle's
    passes without the overlap update, then the update with one all-reduce of
    the probe sums and one of the object sums.  Returns the global per-cycle LLK."""
    out = torch.empty(max(ncycles, 1), dtype=torch.float64, device=pb.device)
    for c in range(ncycles):
        llk = pb.dm(1, update_obj=update_obj, update_probe=update_probe, init_psi=(init_psi and c == 0),
                    normalise=False, llk=out[c:c + 1])
        _overlap_update_split(pb, update_obj, update_probe, llk, group)
    return out[:ncycles]


def ap_cycles_data_parallel(pb, ncycles: int, update_obj=True, update_probe=True, group=None):
    """AP cycles with the same split as ``dm_cycles_data_parallel``."""
    out = torch.empty(max(ncycles, 1), dtype=torch.float64, device=pb.device)
    for c in range(ncycles):
        llk = pb.ap(1, update_obj=update_obj, update_probe=update_probe, normalise=False, llk=out[c:c + 1])
        _overlap_update_split(pb, update_obj, update_probe, llk, group)
    return out[:ncycles]
