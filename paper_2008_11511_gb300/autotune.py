"""Schedule autotuner: picks the schedule of a problem (or a batched handle) by
timing its own cycles: the batch lanes, the batch size, the column pass's tiling
(register-resident lines, or tiles brought in by tensor copies) and the frame
slots of the row-backward pass.

The candidates are run on the real data for a couple of cycles each, timed with
CUDA events on the launch stream; the object, probe and exit-wave state is
copied before and restored after, so tuning leaves the reconstruction where it
was.  Results are cached per (frame size, modes, frames, algorithm) so a second
handle with the same shape reuses them.
"""
from __future__ import annotations

import itertools

import torch

_CACHE: dict = {}


def _state_tensors(target):
    if hasattr(target, "items"):  # PtychoBatch
        ts = []
        for it in target.items:
            ts += [it["obj"], it["probe"], it["psi"]]
        return ts
    return [t for t in (target.obj, target.probe, target.psi) if t is not None]


def _key(target, algorithms):
    if hasattr(target, "items"):
        shape = tuple((tuple(it["probe"].shape), it["iobs"].shape[0]) for it in target.items)
    else:
        shape = ((tuple(target.probe.shape), target.J),)
    return shape, tuple(algorithms)


def _run(target, algorithms, n, init):
    if hasattr(target, "items"):
        return target.cycles(n, algorithms, init_psi=init)
    if algorithms[0] == "DM":
        return target.dm(n, init_psi=init)
    return target.ap(n)


PARAMS = ("lanes", "batch_frames", "tma", "bwd_slots")


def _apply(target, cand):
    for name, v in zip(PARAMS, cand):
        target.set_param(name, v)


def autotune(target, algorithms=("DM",), lanes=(1, 2, 3), batch_frames=(0, 32, 64), tma=(0,), bwd_slots=(0,),
             cycles: int = 2, use_cache: bool = True):
    """Time every (lanes, batch_frames, tma, bwd_slots) candidate and keep the
    fastest on ``target`` (a Ptycho or PtychoBatch).  ``tma`` = 1 feeds the
    256^2 column pass by tensor copies; ``bwd_slots`` = 0 sizes the row-backward
    pass by occupancy.  Returns (best, {candidate: ms per cycle})."""
    algorithms = list(algorithms)
    key = _key(target, algorithms) + (tuple(lanes), tuple(batch_frames), tuple(tma), tuple(bwd_slots))
    if use_cache and key in _CACHE:
        best = _CACHE[key]
        _apply(target, best)
        return best, {}
    saved = [t.clone() for t in _state_tensors(target)]
    stream = torch.cuda.current_stream(target.device)
    times = {}
    first = True
    for cand in itertools.product(lanes, batch_frames, tma, bwd_slots):
        _apply(target, cand)
        _run(target, algorithms, 1, first)  # warm-up (graph capture)
        first = False
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _run(target, algorithms, cycles, False)
        e1.record(stream)
        e1.synchronize()
        times[cand] = e0.elapsed_time(e1) / cycles
    for t, s in zip(_state_tensors(target), saved):
        t.copy_(s)
    best = min(times, key=times.get)
    _apply(target, best)
    _CACHE[key] = best
    return best, times
