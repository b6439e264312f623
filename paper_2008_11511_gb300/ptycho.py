"""PyTorch-facing API of libptycho.

PyTorch provides the device memory (object, probe, intensities, exit-wave
stack, scratch) and the stream; every step of the ptychography cycle runs in
libptycho's CUDA kernels.  Names follow the paper's operators (Section 4 and
the appendix operator table): AP, DM, LLK, ML, FT / IFT.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (PTX_DM_INIT_PSI, PTX_NO_GRAPH, PTX_NO_NORMALISE, PTX_STAGE_OBJ_GATHER, PTX_STAGE_OBJ_NORMALISE,
                   PTX_STAGE_PROBE, PTX_UPDATE_BACKGROUND, PTX_UPDATE_OBJ, PTX_UPDATE_PROBE, SUPPORTED_SIZES, Problem,
                   PtychoError)


def _stream_ptr(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _require_cuda(t: torch.Tensor, name: str, dtype):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Ptycho:
    """One far-field ptychography problem resident on the GPU (the paper's
    ``Ptycho`` object: data, object, probe modes and the exit-wave stack).

    obj:       complex64 (Ho, Wo) CUDA tensor, updated in place by the cycles
    probe:     complex64 (K, N, N) CUDA tensor, updated in place
    iobs:      float32 (J, N, N) CUDA tensor, FFT order (zero frequency at [0, 0])
    positions: int (J, 2) array of (row, col) top-left patch corners
    mask:      optional uint8/bool (N, N) array, nonzero = bad pixel
    psi:       complex64 (J, K, N, N) CUDA tensor, the exit-wave stack used by
               the AP and DM cycles; allocated when ``with_psi`` is set and none
               is given (LLK and gradient alone do not need it)
    nearfield: 0 for the far field; c = lambda z / pixel^2 > 0 for the near field
               (PropagateNearField; iobs and mask then in detector pixels)
    background: optional float32 (N, N) CUDA tensor, the incoherent background
               added to every frame's model intensity (updated in place by
               ``ap(..., update_background=True)``)
    """

    def __init__(self, obj: torch.Tensor, probe: torch.Tensor, iobs: torch.Tensor, positions, mask=None,
                 psi: torch.Tensor | None = None, with_psi: bool = True, nearfield: float = 0.0,
                 background: torch.Tensor | None = None):
        _require_cuda(obj, "obj", torch.complex64)
        _require_cuda(probe, "probe", torch.complex64)
        _require_cuda(iobs, "iobs", torch.float32)
        if probe.dim() != 3 or obj.dim() != 2 or iobs.dim() != 3:
            raise ValueError("shapes: obj (Ho, Wo), probe (K, N, N), iobs (J, N, N)")
        K, N, N2 = probe.shape
        J = iobs.shape[0]
        if N2 != N or tuple(iobs.shape[1:]) != (N, N):
            raise ValueError("probe and iobs frames must be N x N")
        self.device = obj.device
        pos = np.ascontiguousarray(np.asarray(positions, dtype=np.int32).reshape(J, 2))
        if psi is None and with_psi:
            psi = torch.empty((J, K, N, N), dtype=torch.complex64, device=self.device)
        if psi is not None:
            _require_cuda(psi, "psi", torch.complex64)
            if tuple(psi.shape) != (J, K, N, N):
                raise ValueError("psi must be (J, K, N, N)")
        m = None
        if mask is not None:
            m = np.ascontiguousarray(np.asarray(mask).astype(np.uint8).reshape(N, N))
        if background is not None:
            _require_cuda(background, "background", torch.float32)
            if tuple(background.shape) != (N, N):
                raise ValueError("background must be (N, N)")
        self.obj, self.probe, self.iobs, self.psi = obj, probe, iobs, psi
        self.N, self.K, self.J = N, K, J
        self.Ho, self.Wo = obj.shape
        self._prob = Problem(N=N, K=K, J=J, Ho=self.Ho, Wo=self.Wo, obj=obj.data_ptr(), probe=probe.data_ptr(),
                             positions=pos.ctypes.data, iobs=iobs.data_ptr(),
                             mask=(m.ctypes.data if m is not None else None),
                             psi=(psi.data_ptr() if psi is not None else None), nearfield=float(nearfield),
                             background=(background.data_ptr() if background is not None else None))
        self.nearfield = float(nearfield)
        self.background = background
        nbytes = ctypes.c_size_t(0)
        _lib.call("ptx_workspace_bytes", ctypes.byref(self._prob), 1, ctypes.byref(nbytes))
        with torch.cuda.device(self.device):
            self.scratch = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            _lib.call("ptx_create", ctypes.byref(h), ctypes.byref(self._prob), 1,
                      ctypes.c_void_p(self.scratch.data_ptr()), nbytes, _stream_ptr(self.device))
        self._h = h
        self._prob.positions = None
        self._prob.mask = None
        self.positions = pos
        self.mask = m

    # -- lifecycle -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            torch.cuda.current_stream(self.device).synchronize()
            _lib.load().ptx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _handle(self):
        if not self._h:
            raise RuntimeError("Ptycho handle is closed")
        return self._h

    # -- algorithms ------------------------------------------------------------
    @staticmethod
    def _flags(update_obj, update_probe, graph, normalise=True):
        f = 0
        if update_obj:
            f |= PTX_UPDATE_OBJ
        if update_probe:
            f |= PTX_UPDATE_PROBE
        if not graph:
            f |= PTX_NO_GRAPH
        if not normalise:
            f |= PTX_NO_NORMALISE
        return f

    def ap(self, ncycles: int, update_obj: bool = True, update_probe: bool = True, graph: bool = True,
           normalise: bool = True, llk: torch.Tensor | None = None, update_background: bool = False) -> torch.Tensor:
        """``ncycles`` alternating-projection cycles; returns the per-cycle LLK
        (float64 CUDA tensor of length ncycles).  ``update_background`` also
        optimises the incoherent background given at construction."""
        if self.psi is None:
            raise ValueError("AP needs the exit-wave stack: create Ptycho with with_psi=True")
        f = self._flags(update_obj, update_probe, graph, normalise)
        if update_background:
            if self.background is None:
                raise ValueError("update_background needs a background: create Ptycho with background=...")
            f |= PTX_UPDATE_BACKGROUND
        out = llk if llk is not None else torch.empty(max(ncycles, 1), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.call("ptx_ap_cycles", self._handle(), int(ncycles), f,
                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(self.device))
        return out[:ncycles]

    def dm(self, ncycles: int, update_obj: bool = True, update_probe: bool = True, init_psi: bool = False,
           graph: bool = True, normalise: bool = True, llk: torch.Tensor | None = None) -> torch.Tensor:
        """``ncycles`` difference-map cycles; ``init_psi`` sets Psi = P O first."""
        if self.psi is None:
            raise ValueError("DM needs the exit-wave stack: create Ptycho with with_psi=True")
        f = self._flags(update_obj, update_probe, graph, normalise)
        if init_psi:
            f |= PTX_DM_INIT_PSI
        out = llk if llk is not None else torch.empty(max(ncycles, 1), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.call("ptx_dm_cycles", self._handle(), int(ncycles), f, ctypes.c_void_p(out.data_ptr()),
                      _stream_ptr(self.device))
        return out[:ncycles]

    def position_shifts(self, filter_ratio: float = 0.1) -> torch.Tensor:
        """Per-frame least-squares position shifts (row, col) in pixels from the
        exit waves of the last AP cycle (float32 CUDA tensor (J, 2))."""
        out = torch.empty((self.J, 2), dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            _lib.call("ptx_position_shifts", self._handle(), 0, ctypes.c_float(filter_ratio),
                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(self.device))
        return out

    def set_positions(self, positions):
        """Replace the integer scan positions (J, 2) (rebuilds the object tiles)."""
        pos = np.ascontiguousarray(np.asarray(positions, dtype=np.int32).reshape(self.J, 2))
        with torch.cuda.device(self.device):
            _lib.call("ptx_set_positions", self._handle(), 0, ctypes.c_void_p(pos.ctypes.data),
                      _stream_ptr(self.device))
        self.positions = pos

    def refine_positions(self, filter_ratio: float = 0.1, step: float = 1.0, max_shift: float = 2.0):
        """One position-refinement step after an AP cycle: the per-frame shifts
        (scaled by ``step``, clipped to ``max_shift`` px) accumulate into
        sub-pixel positions, and frames whose rounded position changes move.
        Returns the sub-pixel positions (float64 (J, 2))."""
        if getattr(self, "_pos_f", None) is None:
            self._pos_f = np.ascontiguousarray(self.positions.astype(np.float64))
        d = np.ascontiguousarray(self.position_shifts(filter_ratio).cpu().numpy())
        new = np.ascontiguousarray(self.positions.astype(np.int32))
        moved = ctypes.c_int32()
        _lib.call("ptx_accumulate_shifts", int(self.J), ctypes.c_void_p(d.ctypes.data), float(step),
                  float(max_shift), int(self.Ho - self.N), int(self.Wo - self.N),
                  ctypes.c_void_p(self._pos_f.ctypes.data), ctypes.c_void_p(new.ctypes.data), ctypes.byref(moved))
        if moved.value > 0:
            self.set_positions(new)
        return self._pos_f.copy()

    def llk(self) -> torch.Tensor:
        """Exact Poisson LLK of the current object and probe (float64 CUDA scalar tensor)."""
        out = torch.empty(1, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.call("ptx_llk", self._handle(), ctypes.c_void_p(out.data_ptr()), _stream_ptr(self.device))
        return out[0]

    def ml_grad(self, grad_obj: bool = True, grad_probe: bool = True):
        """Poisson-LLK gradient: returns (llk, G_O or None, G_P or None) with
        G = dL/dRe z + i dL/dIm z (the PyTorch convention for real losses)."""
        go = torch.empty_like(self.obj) if grad_obj else None
        gp = torch.empty_like(self.probe) if grad_probe else None
        out = torch.empty(1, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.call("ptx_ml_grad", self._handle(), ctypes.c_void_p(go.data_ptr() if go is not None else None),
                      ctypes.c_void_p(gp.data_ptr() if gp is not None else None), ctypes.c_void_p(out.data_ptr()),
                      _stream_ptr(self.device))
        return out[0], go, gp

    def ml(self, ncycles: int, update_obj: bool = True, update_probe: bool = False, restart: bool = False,
           llk: torch.Tensor | None = None) -> torch.Tensor:
        """``ncycles`` maximum-likelihood conjugate-gradient steps (the ML operator;
        by default the object only, as the paper's ML defaults).  Returns the LLK
        before each step (float64 CUDA tensor).  ``restart`` forgets the previous
        direction."""
        f = self._flags(update_obj, update_probe, True)
        if restart:
            f |= _lib.PTX_ML_RESTART
        out = llk if llk is not None else torch.empty(max(ncycles, 1), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.call("ptx_ml_cycles", self._handle(), int(ncycles), f, ctypes.c_void_p(out.data_ptr()),
                      _stream_ptr(self.device))
        return out[:ncycles]

    def line_coeffs(self, d_obj: torch.Tensor | None, d_probe: torch.Tensor | None) -> torch.Tensor:
        """(L'(0), L''(0)) of the LLK along the direction (d_obj, d_probe)."""
        out = torch.empty(2, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.call("ptx_ml_line_coeffs", self._handle(),
                      ctypes.c_void_p(d_obj.data_ptr() if d_obj is not None else None),
                      ctypes.c_void_p(d_probe.data_ptr() if d_probe is not None else None),
                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(self.device))
        return out

    def normalise(self, update_obj: bool = True, update_probe: bool = True, stages: int | None = None):
        """Second half of Psi2ObjProbe after cycles run with ``normalise=False``:
        the probe from its accumulator, then the object gathered from Psi' with
        the new probe.  ``stages`` (PTX_STAGE_* bits) runs selected stages, for
        an all-reduce of ``accumulators()`` in between (data-parallel split)."""
        f = stages if stages is not None else self._flags(update_obj, update_probe, True)
        with torch.cuda.device(self.device):
            _lib.call("ptx_normalise", self._handle(), int(f), _stream_ptr(self.device))

    def accumulators(self):
        """Views of the object and probe accumulators: float32 (Ho, Wo, 4) and
        (K, N, N, 4) with {Re N, Im N, D, 0} per pixel."""
        po, so, pp, sp = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_void_p(), ctypes.c_size_t()
        _lib.call("ptx_accumulators", self._handle(), 0, ctypes.byref(po), ctypes.byref(so), ctypes.byref(pp),
                  ctypes.byref(sp))
        base = self.scratch.data_ptr()
        oo = po.value - base
        op = pp.value - base
        acc_o = self.scratch[oo:oo + so.value].view(torch.float32).view(self.Ho, self.Wo, 4)
        acc_p = self.scratch[op:op + sp.value].view(torch.float32).view(self.K, self.N, self.N, 4)
        return acc_o, acc_p

    def set_param(self, name: str, value: float):
        """A handle parameter, by the names and ranges of ptx_set_param: the
        inertia factors ``alpha_obj`` / ``alpha_probe``, the schedule
        (``lanes``, ``batch_frames``, ``bwd_slots``, ``tma``, ``tma_gather``,
        ``persistent``, ``pdl``), the number format of the DFT stages (``tc``,
        ``tc_rows``) and the self-test switches; PtychoError for an unknown name
        or a value out of range."""
        _lib.call("ptx_set_param", self._handle(), name.encode(), float(value))


class PtychoBatch:
    """Several independent ptychography problems (any frame sizes and scan
    lengths) in one handle: one CUDA graph per cycle over all of them, each
    problem with its own algorithm (AP or DM).

    problems: list of dicts with keys obj, probe, iobs, positions and optionally
    mask and psi (allocated when absent), as for :class:`Ptycho`."""

    def __init__(self, problems):
        if not problems:
            raise ValueError("no problems")
        self.items = []
        keep = []
        arr = (Problem * len(problems))()
        dev = None
        for i, d in enumerate(problems):
            obj, probe, iobs = d["obj"], d["probe"], d["iobs"]
            _require_cuda(obj, "obj", torch.complex64)
            _require_cuda(probe, "probe", torch.complex64)
            _require_cuda(iobs, "iobs", torch.float32)
            K, N, _ = probe.shape
            J = iobs.shape[0]
            dev = dev or obj.device
            psi = d.get("psi")
            if psi is None:
                psi = torch.empty((J, K, N, N), dtype=torch.complex64, device=dev)
            _require_cuda(psi, "psi", torch.complex64)
            pos = np.ascontiguousarray(np.asarray(d["positions"], dtype=np.int32).reshape(J, 2))
            m = d.get("mask")
            m = None if m is None else np.ascontiguousarray(np.asarray(m).astype(np.uint8).reshape(N, N))
            keep += [pos, m]
            arr[i] = Problem(N=N, K=K, J=J, Ho=obj.shape[0], Wo=obj.shape[1], obj=obj.data_ptr(),
                             probe=probe.data_ptr(), positions=pos.ctypes.data, iobs=iobs.data_ptr(),
                             mask=(m.ctypes.data if m is not None else None), psi=psi.data_ptr(),
                             nearfield=float(d.get("nearfield", 0.0)))
            self.items.append(dict(obj=obj, probe=probe, iobs=iobs, psi=psi, positions=pos, mask=m))
        self.device = dev
        self.nprob = len(problems)
        nbytes = ctypes.c_size_t(0)
        _lib.call("ptx_workspace_bytes", arr, self.nprob, ctypes.byref(nbytes))
        with torch.cuda.device(dev):
            self.scratch = torch.empty(int(nbytes.value), dtype=torch.uint8, device=dev)
            h = ctypes.c_void_p()
            _lib.call("ptx_create", ctypes.byref(h), arr, self.nprob, ctypes.c_void_p(self.scratch.data_ptr()), nbytes,
                      _stream_ptr(dev))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            torch.cuda.current_stream(self.device).synchronize()
            _lib.load().ptx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _handle(self):
        if not self._h:
            raise RuntimeError("PtychoBatch handle is closed")
        return self._h

    def cycles(self, ncycles: int, algorithms, update_obj: bool = True, update_probe: bool = True,
               init_psi: bool = False, graph: bool = True) -> torch.Tensor:
        """``ncycles`` cycles of every problem; ``algorithms`` lists "AP" / "DM" per
        problem.  Returns the LLK as a float64 CUDA tensor (ncycles, nprob)."""
        codes = np.array([_lib.PTX_ALGO_DM if str(a).upper() == "DM" else _lib.PTX_ALGO_AP for a in algorithms],
                         dtype=np.int32)
        if len(codes) != self.nprob:
            raise ValueError("one algorithm per problem")
        f = Ptycho._flags(update_obj, update_probe, graph)
        if init_psi:
            f |= PTX_DM_INIT_PSI
        out = torch.empty(max(ncycles, 1) * self.nprob, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.call("ptx_cycles", self._handle(), int(ncycles), f, ctypes.c_void_p(codes.ctypes.data),
                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(self.device))
        return out[:ncycles * self.nprob].view(ncycles, self.nprob)

    def set_param(self, name: str, value: float):
        _lib.call("ptx_set_param", self._handle(), name.encode(), float(value))


def fft2(x: torch.Tensor, direction: int = -1) -> torch.Tensor:
    """In-place orthonormal 2D FFT of complex64 frames (..., N, N) on the GPU
    (the FT operator; ``direction=+1`` is IFT).  Returns ``x``."""
    _require_cuda(x, "x", torch.complex64)
    N = x.shape[-1]
    if x.shape[-2] != N:
        raise ValueError("frames must be square")
    nframes = x.numel() // (N * N)
    with torch.cuda.device(x.device):
        _lib.call("ptx_fft2", ctypes.c_void_p(x.data_ptr()), int(nframes), int(N), int(direction),
                  _stream_ptr(x.device))
    return x


def fma_tflops(device=None, iters: int = 8192, blocks_per_sm: int = 8, repeats: int = 3) -> float:
    """Measured FP32 FMA throughput of the GPU in TFLOP/s (best of ``repeats``
    launches of ``ptx_fma_peak``, timed with CUDA events on the current stream):
    the ALU roof the FFT passes are compared against."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * blocks_per_sm
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    flops = ctypes.c_double()
    best = 0.0
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream(dev)
        for r in range(repeats + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _lib.call("ptx_fma_peak", int(blocks), int(iters), ctypes.c_void_p(sink.data_ptr()), ctypes.byref(flops),
                      _stream_ptr(dev))
            e1.record(stream)
            e1.synchronize()
            if r > 0:  # the first launch warms up
                best = max(best, flops.value / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def counts_to_float(dst: torch.Tensor, counts: torch.Tensor) -> torch.Tensor:
    """dst[...] = counts as float32, on the GPU (photon counts uploaded as
    16-bit integers and widened on the device, e.g. into a problem's ``iobs``).
    ``counts`` is a uint16 CUDA tensor with as many elements as ``dst``.
    Returns ``dst``."""
    _require_cuda(dst, "dst", torch.float32)
    _require_cuda(counts, "counts", torch.uint16)
    if counts.numel() != dst.numel():
        raise ValueError("counts and dst must have the same number of elements")
    with torch.cuda.device(dst.device):
        _lib.call("ptx_counts_to_float", ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(counts.data_ptr()),
                  ctypes.c_size_t(dst.numel()), _stream_ptr(dst.device))
    return dst


def encode_counts8(counts) -> tuple:
    """Host side of the one-byte count form (ptx_encode_counts8): ``counts``
    is a uint16 array (any shape); returns (uint8 array of the same shape with
    the counts clipped at 255, uint32 flat indices and uint16 values of the
    counts >= 255, in increasing index)."""
    import numpy as np
    c = np.ascontiguousarray(counts, dtype=np.uint16)
    n = c.size
    n_esc = ctypes.c_size_t(0)
    _lib.call("ptx_encode_counts8", ctypes.c_void_p(c.ctypes.data), ctypes.c_size_t(n), None, None, None,
              ctypes.c_size_t(0), ctypes.byref(n_esc))
    out8 = np.empty(c.shape, dtype=np.uint8)
    idx = np.empty(n_esc.value, dtype=np.uint32)
    val = np.empty(n_esc.value, dtype=np.uint16)
    _lib.call("ptx_encode_counts8", ctypes.c_void_p(c.ctypes.data), ctypes.c_size_t(n),
              ctypes.c_void_p(out8.ctypes.data), ctypes.c_void_p(idx.ctypes.data), ctypes.c_void_p(val.ctypes.data),
              ctypes.c_size_t(n_esc.value), ctypes.byref(n_esc))
    return out8, idx, val


def counts8_to_float(dst: torch.Tensor, counts8: torch.Tensor, esc_index: torch.Tensor,
                     esc_value: torch.Tensor) -> torch.Tensor:
    """dst[...] = the counts of the one-byte form, on the GPU: the uint8
    counts widened to float32, then the escapes (uint32 flat indices into dst,
    uint16 values) written over them.  CUDA tensors; returns ``dst``."""
    _require_cuda(dst, "dst", torch.float32)
    _require_cuda(counts8, "counts8", torch.uint8)
    if counts8.numel() != dst.numel():
        raise ValueError("counts8 and dst must have the same number of elements")
    if esc_index.numel() != esc_value.numel():
        raise ValueError("esc_index and esc_value must have the same length")
    n_esc = esc_index.numel()
    if n_esc:
        _require_cuda(esc_index, "esc_index", torch.uint32)
        _require_cuda(esc_value, "esc_value", torch.uint16)
    with torch.cuda.device(dst.device):
        _lib.call("ptx_counts8_to_float", ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(counts8.data_ptr()),
                  ctypes.c_size_t(dst.numel()), ctypes.c_void_p(esc_index.data_ptr() if n_esc else None),
                  ctypes.c_void_p(esc_value.data_ptr() if n_esc else None), ctypes.c_size_t(n_esc),
                  _stream_ptr(dst.device))
    return dst


class PtychoLLK(torch.autograd.Function):
    """L(O, P) = Poisson LLK as a differentiable function of the object and the
    probe.  ``forward`` copies (obj, probe) into the problem's buffers and calls
    ptx_llk; ``backward`` calls ptx_ml_grad, which recomputes the exit waves
    rather than storing them (the ML operator's gradient)."""

    @staticmethod
    def forward(ctx, obj: torch.Tensor, probe: torch.Tensor, problem: Ptycho):
        with torch.no_grad():
            problem.obj.copy_(obj)
            problem.probe.copy_(probe)
        ctx.problem = problem
        ctx.needs = (obj.requires_grad, probe.requires_grad)
        return problem.llk().clone()

    @staticmethod
    def backward(ctx, grad_out):
        pb = ctx.problem
        _, go, gp = pb.ml_grad(grad_obj=ctx.needs[0], grad_probe=ctx.needs[1])
        g = grad_out.to(torch.float32)
        return (go * g if go is not None else None, gp * g if gp is not None else None, None)


__all__ = ["Ptycho", "PtychoBatch", "PtychoLLK", "PtychoError", "fft2", "SUPPORTED_SIZES", "PTX_STAGE_PROBE",
           "PTX_STAGE_OBJ_GATHER", "PTX_STAGE_OBJ_NORMALISE"]
