"""Benchmark: difference-map cycle throughput on 256x256 frames (frames/s) and
its fraction of the HBM roof, on one GB300 per process.

Workload (one "step" = one full DM cycle over every frame): 4000 frames of
256 x 256 on a Fermat spiral over a 2048 x 2048 object, one probe mode, 1e6
photons per frame, a 2 % detector-gap mask; the synthetic stand-in for the
paper's far-field ptychography workloads (Table 1: 1000 x 256^2 frames).

Arms:
  default          libptycho CUDA path (CUDA graph replay of the cycle)
  --impl reference the FP64 CPU oracle (the only reference there is for this
                   method), timed on a bounded sample of the same workload

Output: one JSON line on rank 0.  Multi-GPU (torchrun): every rank runs an
independent replica of the workload (the DM cycle over one object has no
independent partition without a per-cycle all-reduce); value = frames of all
ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DM-cycle frames/s at 256² (plain FP32 vs chosen form, same GB300); % HBM roof"
UNIT = "frames/s"
WORKLOAD = "dm256"
FORMS = {0: "fp32 (plain)",
         1: "tf32 hi+lo tensor-core DFT stages in the column pass, fp32 elsewhere",
         2: "bf16 hi+mid+lo tensor-core DFT stages in the column pass, fp32 elsewhere",
         3: "bf16 hi+lo tensor-core DFT stages in the column pass (below fp32 accuracy), fp32 elsewhere"}
FORMS_ALL = {1: "tf32 hi+lo tensor-core DFT stages in every pass (column and rows)",
             2: "bf16 hi+mid+lo tensor-core DFT stages in every pass (column and rows)",
             3: "bf16 hi+lo tensor-core DFT stages in every pass (below fp32 accuracy)"}
PROFILES = os.path.join(ROOT, "profiles")


def workload_desc(s):
    return (f"DM cycle, {s.J} frames {s.N}x{s.N}, object {s.Ho}x{s.Wo}, K={s.K}, "
            f"{s.photons:.0e} photons/frame, {100 * s.mask.mean():.1f}% mask, spiral step {s.step_px:.1f} px")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0))}
    return {"hbm_gbs": 6800.0, "src": "fallback", "sm_max_mhz": 2070.0}


def alg_bytes_per_cycle(s, algo="DM"):
    """Bytes the cycle must move through HBM: Psi read (DM's 2 Phi - Psi), Psi'
    written, Psi' read again by the object update (which needs the updated probe,
    so it follows the probe update), I read, O and P read + write."""
    px = s.N * s.N
    b = s.J * px * 4 + s.Ho * s.Wo * 16 + s.K * px * 16 + s.J * s.K * px * 16
    if algo == "DM":
        b += s.J * s.K * px * 8
    return b


# per-kernel algorithmic HBM bytes per frame (DM) and nominal flops per frame
def kernel_models(s):
    import math
    px = s.N * s.N
    K = s.K
    fft1d = 5.0 * px * math.log2(s.N)  # one 1D pass over all rows (or columns) of a frame
    return {
        "row_fwd": {"bytes": K * px * 8, "flops": K * (fft1d + 10.0 * px)},
        "col": {"bytes": px * 4, "flops": K * (2 * fft1d + 12.0 * px) + 30.0 * px},
        "row_bwd": {"bytes": K * px * 8, "flops": K * (fft1d + 12.0 * px) + 4.0 * px},
        "obj_gather": {"bytes": K * px * 8, "flops": K * 11.0 * px},
    }


def _code_only(src: str) -> str:
    """C++ source without comments and blank lines (string and character
    literals kept), so that the hash follows the code, not its comments."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            i = src.find("\n", i)
            i = n if i < 0 else i
        elif src.startswith("/*", i):
            i = src.find("*/", i + 2)
            i = n if i < 0 else i + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).splitlines() if line.strip())


def source_hash():
    """Hash of the kernel sources' code (comments and blank lines ignored)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2008_11511_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".inc")):
            h.update(_code_only(open(os.path.join(d, f), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    p = os.path.join(PROFILES, "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(kernel)
    if not ent or ent.get("source_hash") != source_hash():
        return None
    return ent.get("dram_bytes_per_launch_full")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        med = statistics.median(sms) if sms else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sms)}


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample_rate(s, seconds=15.0, min_frames=32):
    """FP64 oracle DM-cycle throughput (frames/s) on a bounded sample of the
    workload's frames (same object, probe, mask and intensities)."""
    import oracle
    J = min_frames
    while True:
        idx = np.linspace(0, s.J - 1, J).astype(np.int64)
        data = oracle.Data.make(s.iobs[idx], s.positions[idx], s.mask)
        t0 = time.perf_counter()
        oracle.dm_cycle(s.obj0, s.probe0, None, data, init_psi=True)
        dt = time.perf_counter() - t0
        if dt >= seconds / 4 or J >= s.J:
            return J / dt, J, dt
        J = min(s.J, int(J * max(2.0, seconds / 4 / max(dt, 1e-3))))


def run_reference(args):
    """The oracle as the reference arm (rank 0 only)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from synthetic import make_config
    s = make_config(WORKLOAD)
    cores = len(os.sched_getaffinity(0))
    # size one step so that warmup + steps stay within a few minutes
    rate, J, dt = oracle_sample_rate(s, seconds=8.0)
    idx = np.linspace(0, s.J - 1, J).astype(np.int64)
    data = oracle.Data.make(s.iobs[idx], s.positions[idx], s.mask)
    obj, probe, psi = s.obj0, s.probe0, None
    for w in range(args.warmup):
        obj, probe, psi, _ = oracle.dm_cycle(obj, probe, psi, data, init_psi=(w == 0))
    t0 = time.perf_counter()
    for k in range(args.steps):
        obj, probe, psi, _ = oracle.dm_cycle(obj, probe, psi, data, init_psi=(psi is None))
    el = time.perf_counter() - t0
    value = J * args.steps / el
    sample = f"{J} of {s.J} frames per step (evenly spaced), full 2048^2 object, FP64 NumPy/SciPy"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "desc": workload_desc(s), "form": "fp64 oracle",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def exact_counts(x):
    """The intensities as uint16 photon counts when that is exact, else None."""
    if x.min() < 0 or x.max() > 65535 or not np.array_equal(x, np.rint(x)):
        return None
    return x.astype(np.uint16)


def e2e_form(args, s):
    """The upload form of the end-to-end leg: "u8" (one-byte counts plus an
    escape list), "u16" (uint16 counts) or "f32"; "auto" takes the smallest
    exact one (u8 while at most 10 % of the counts need an escape)."""
    if args.e2e_dtype == "f32":
        return "f32"
    counts = exact_counts(s.iobs)
    if counts is None:
        if args.e2e_dtype in ("u8", "u16"):
            raise SystemExit(f"--e2e-dtype {args.e2e_dtype}: the intensities are not exact uint16 counts")
        return "f32"
    if args.e2e_dtype == "u16":
        return "u16"
    if args.e2e_dtype == "u8" or (counts >= 255).mean() <= 0.10:
        return "u8"
    return "u16"


def run_e2e(args, s, pb, obj, probe, iobs, params, llk_buf, stream, dev, ws, form):
    """The end-to-end leg: per step the host -> device upload of the intensity
    stack from pinned memory, the DM cycle, the LLK read back; the upload of
    step k + 1 runs on copy streams while step k computes.

    The intensities go into the other of two device buffers, each with its own
    handle sharing the object, the probe and the exit waves.  The synthetic
    intensities are Poisson photon counts: form "u8" uploads them as one byte
    each plus the escape list of the counts >= 255 and decodes them into that
    float32 buffer with ``counts8_to_float`` on the copy stream; "u16" uploads
    uint16 counts and widens them with ``counts_to_float``; "f32" uploads the
    float32 frames.  The host-side encoding is done before the timed region.
    Returns (frames/s, bytes uploaded per step, description, runs)."""
    import torch
    from paper_2008_11511_gb300 import Ptycho, counts8_to_float, counts_to_float, encode_counts8
    host_llk = torch.empty(1, dtype=torch.float64).pin_memory()
    n_copy = max(1, args.copy_streams)
    bounds = [s.J * c // n_copy for c in range(n_copy + 1)]
    copy_streams = [torch.cuda.Stream(dev) for _ in range(n_copy)]
    copied = [[torch.cuda.Event() for _ in range(n_copy)] for _ in range(2)]
    used = [torch.cuda.Event(), torch.cuda.Event()]
    iobs2 = torch.empty_like(iobs)
    extra = Ptycho(obj, probe, iobs2, s.positions, s.mask, psi=pb.psi)
    for name, val in params:
        extra.set_param(name, val)
    iobs2.copy_(iobs)
    extra.dm(1, llk=llk_buf)  # graph capture outside the timed region
    bufs, handles = [iobs, iobs2], (pb, extra)
    px = s.N * s.N
    if form == "u8":
        c8, e_idx, e_val = encode_counts8(exact_counts(s.iobs))
        host = torch.from_numpy(c8).pin_memory()
        stage = [torch.empty(c8.shape, dtype=torch.uint8, device=dev) for _ in range(2)]
        # each copy stream's escapes, as indices relative to its first frame
        cuts = np.searchsorted(e_idx, [b * px for b in bounds])
        h_idx = [torch.from_numpy((e_idx[cuts[c]:cuts[c + 1]] - bounds[c] * px).astype(np.uint32)).pin_memory()
                 for c in range(n_copy)]
        h_val = [torch.from_numpy(np.ascontiguousarray(e_val[cuts[c]:cuts[c + 1]])).pin_memory()
                 for c in range(n_copy)]
        d_idx = [[torch.empty(h.numel(), dtype=torch.uint32, device=dev) for h in h_idx] for _ in range(2)]
        d_val = [[torch.empty(h.numel(), dtype=torch.uint16, device=dev) for h in h_val] for _ in range(2)]
        step_bytes = host.numel() + 6 * int(e_idx.size)
        desc = (f"one-byte photon counts with an escape list ({e_idx.size / s.iobs.size:.1%} of the counts >= 255: "
                "uint32 index + uint16 value) from pinned host memory, decoded to float32 on the device on the copy "
                "stream, into two device buffers")
    elif form == "u16":
        host = torch.from_numpy(exact_counts(s.iobs)).pin_memory()
        stage = [torch.empty(host.shape, dtype=torch.uint16, device=dev) for _ in range(2)]
        step_bytes = host.numel() * 2
        desc = ("uint16 photon counts (exact) from pinned host memory, widened to float32 on the device on the copy "
                "stream, into two device buffers")
    else:
        host = torch.from_numpy(s.iobs).pin_memory()
        stage = None
        step_bytes = host.numel() * 4
        desc = "float32 frames from pinned host memory into two device buffers"
    desc += f", on {n_copy} copy stream(s) one step ahead"

    def upload(nb, wait_used):
        for c, cs in enumerate(copy_streams):
            lo, hi = bounds[c], bounds[c + 1]
            with torch.cuda.stream(cs):
                if wait_used:
                    cs.wait_event(used[nb])
                if form == "u8":
                    stage[nb][lo:hi].copy_(host[lo:hi], non_blocking=True)
                    d_idx[nb][c].copy_(h_idx[c], non_blocking=True)
                    d_val[nb][c].copy_(h_val[c], non_blocking=True)
                    counts8_to_float(bufs[nb][lo:hi], stage[nb][lo:hi], d_idx[nb][c], d_val[nb][c])
                elif form == "u16":
                    stage[nb][lo:hi].copy_(host[lo:hi], non_blocking=True)
                    counts_to_float(bufs[nb][lo:hi], stage[nb][lo:hi])
                else:
                    bufs[nb][lo:hi].copy_(host[lo:hi], non_blocking=True)
                copied[nb][c].record(cs)

    # the host-to-device path is shared with the rest of the machine: the leg
    # is timed `repeats` times and the median kept (each run listed)
    e_steps = max(1, min(args.steps, 50))  # the first upload is not overlapped: it counts once per run
    runs = []
    for _ in range(max(1, args.e2e_repeats)):
        barrier(ws)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        upload(0, False)
        for k in range(e_steps):
            b = k % 2
            if k + 1 < e_steps:
                upload(1 - b, k >= 1)
            for ev in copied[b]:
                stream.wait_event(ev)
            l = handles[b].dm(1, llk=llk_buf)
            used[b].record(stream)
            host_llk.copy_(l[:1], non_blocking=True)
        stream.synchronize()
        for cs in copy_streams:
            cs.synchronize()
        el = time.perf_counter() - t0
        barrier(ws)
        el = max_over_ranks(el, ws)
        runs.append(s.J * e_steps * ws / el)
    torch.cuda.synchronize(dev)
    extra.close()  # both buffers hold the same values (the one host array, uploaded every step)
    desc += f"; median of {len(runs)} timed runs of {e_steps} steps"
    return statistics.median(runs), step_bytes, desc, runs


def _events_ms(fn, n, stream):
    """Median over n calls of fn() timed with CUDA events on `stream` (ms per call)."""
    import torch
    out = []
    for _ in range(n):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def run_extra_ml(dev, fma_peak, ws):
    """The ML workload (1000 frames of 256^2, object 1536^2): the Poisson-LLK
    gradient and one conjugate-gradient step, against the FP32 ALU roof (the
    gradient moves 0.3 GB but transforms every frame twice)."""
    import torch
    from paper_2008_11511_gb300 import Ptycho
    from synthetic import make_config
    s = make_config("ml256")
    obj = torch.tensor(s.obj0, device=dev)
    probe = torch.tensor(s.probe0, device=dev)
    iobs = torch.tensor(s.iobs, device=dev)
    pb = Ptycho(obj, probe, iobs, s.positions, s.mask, with_psi=False)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        pb.ml_grad()
        pb.ml(1)
    torch.cuda.synchronize(dev)
    ms_g = _events_ms(lambda: pb.ml_grad(), 10, stream)
    ms_cg = _events_ms(lambda: pb.ml(1), 10, stream)
    pb.close()
    m = kernel_models(s)
    # the gradient: forward transform and back-propagation of every frame
    flops = s.J * (m["row_fwd"]["flops"] + m["col"]["flops"] + m["row_bwd"]["flops"])
    tf = flops / (ms_g * 1e-3) / 1e12
    return {"workload": f"ML gradient and CG step, {s.J} frames {s.N}x{s.N}, object {s.Ho}x{s.Wo}, "
                        f"{s.photons:.0e} photons/frame",
            "ms_per_gradient": ms_g, "gradient_frames_per_s": s.J * ws / (ms_g * 1e-3),
            "ms_per_cg_step": ms_cg, "cg_frames_per_s": s.J * ws / (ms_cg * 1e-3),
            "roofline": {"kernel": "gradient (three passes)", "bound": "alu", "achieved": tf, "peak": fma_peak,
                         "unit": "TFLOP/s", "frac": tf / fma_peak, "flops_per_gradient": flops,
                         "peak_src": "measured FP32 FMA probe"}}


def run_extra_modes(dev, pk, ws, J=1500, H=2800):
    """Three incoherent probe modes of 512^2 (the multi-mode workload, on its
    first 1500 positions and a 2800^2 object that covers them): DM cycles
    against the HBM roof on the scope table's bytes."""
    import torch
    from paper_2008_11511_gb300 import Ptycho
    from synthetic import make_config
    s = make_config("modes512", J=J, Ho=H, Wo=H)
    obj = torch.tensor(s.obj0, device=dev)
    probe = torch.tensor(s.probe0, device=dev)
    iobs = torch.tensor(s.iobs, device=dev)
    pb = Ptycho(obj, probe, iobs, s.positions, s.mask, with_psi=True)
    stream = torch.cuda.current_stream(dev)
    llk = torch.empty(8, dtype=torch.float64, device=dev)
    pb.dm(2, init_psi=True, llk=llk)
    pb.dm(2, llk=llk)
    torch.cuda.synchronize(dev)
    ms = _events_ms(lambda: pb.dm(3, llk=llk), 3, stream) / 3
    # the same cycle with the column pass's DFT stages on the tensor cores
    forms = []
    for tc, rows in ((1, 0), (2, 0), (3, 0), (1, 1), (2, 1), (3, 1)):
        pb.set_param("tc", tc)
        pb.set_param("tc_rows", rows)
        pb.dm(1, llk=llk)
        torch.cuda.synchronize(dev)
        ms_f = _events_ms(lambda: pb.dm(3, llk=llk), 2, stream) / 3
        forms.append({"form": FORMS_ALL[tc] if rows else FORMS[tc], "ms_per_cycle": ms_f,
                      "frames_per_s": s.J * ws / (ms_f * 1e-3)})
    pb.set_param("tc", 0)
    pb.set_param("tc_rows", 0)
    pb.close()
    px = s.N * s.N
    b = s.J * s.K * px * 16 + s.J * px * 4 + s.Ho * s.Wo * 16 + s.K * px * 16
    gbs = b / (ms * 1e-3) / 1e9
    return {"workload": f"DM cycle, {s.J} frames {s.N}x{s.N}, K={s.K} modes, object {s.Ho}x{s.Wo}, "
                        f"{s.photons:.0e} photons/frame (first {J} positions of the 10000-position scan)",
            "ms_per_cycle": ms, "frames_per_s": s.J * ws / (ms * 1e-3),
            "frame_modes_per_s": s.J * s.K * ws / (ms * 1e-3), "other_form": forms,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / pk["hbm_gbs"], "alg_bytes_per_cycle": b, "peak_src": pk["src"]}}


def run_extra_batched(dev, ws, j_scale=0.25):
    """The batched workload (16 independent scans, frame sizes 128^2 to 512^2,
    AP and DM alternately), each scan's positions scaled by j_scale to bound the
    set-up time: cycles of all problems through one handle (one CUDA graph per
    cycle, schedule from the autotuner) against the same problems as 16
    separate handles run one after the other on the stream."""
    import torch
    from paper_2008_11511_gb300 import Ptycho, PtychoBatch
    from paper_2008_11511_gb300.autotune import autotune
    from synthetic import make_scan
    from synthetic.scans import batched_problem_specs
    specs = batched_problem_specs(j_scale=j_scale)
    scans = [make_scan(**d) for d in specs]
    algos = [d["algorithm"] for d in specs]
    items = [dict(obj=torch.tensor(s.obj0, device=dev), probe=torch.tensor(s.probe0, device=dev),
                  iobs=torch.tensor(s.iobs, device=dev), positions=s.positions, mask=s.mask) for s in scans]
    frames = sum(s.J for s in scans)
    stream = torch.cuda.current_stream(dev)
    pb = PtychoBatch(items)
    pb.cycles(1, algos, init_psi=True)
    best, _ = autotune(pb, algos, lanes=(1, 2), batch_frames=(0, 32), use_cache=False)
    pb.cycles(1, algos)
    torch.cuda.synchronize(dev)
    ms_one = _events_ms(lambda: pb.cycles(3, algos), 3, stream) / 3
    # the same problems as one persistent launch of their batch passes per cycle
    pb.set_param("persistent", 1)
    pb.cycles(1, algos)
    torch.cuda.synchronize(dev)
    ms_pers = _events_ms(lambda: pb.cycles(3, algos), 3, stream) / 3
    pb.close()
    handles = [Ptycho(it["obj"], it["probe"], it["iobs"], it["positions"], it["mask"], with_psi=True) for it in items]
    for h, a in zip(handles, algos):
        h.dm(1, init_psi=True) if a == "DM" else h.ap(1)

    def sep():
        for h, a in zip(handles, algos):
            h.dm(1) if a == "DM" else h.ap(1)
    sep()
    torch.cuda.synchronize(dev)
    ms_sep = _events_ms(sep, 3, stream)
    for h in handles:
        h.close()
    return {"workload": f"{len(specs)} scans, frame sizes {sorted(set(s.N for s in scans))}, {frames} frames "
                        f"(positions x{j_scale} of the full batched workload), AP and DM alternately",
            "ms_per_cycle_one_handle": ms_one, "frames_per_s_one_handle": frames * ws / (ms_one * 1e-3),
            "schedule": dict(zip(("lanes", "batch_frames", "tma", "bwd_slots"), best)),
            "ms_per_cycle_persistent": ms_pers, "frames_per_s_persistent": frames * ws / (ms_pers * 1e-3),
            "ms_per_cycle_separate_handles": ms_sep, "frames_per_s_separate": frames * ws / (ms_sep * 1e-3)}


def run_ours(args):
    import torch
    ws, rank, local = dist_init()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2008_11511_gb300 import Ptycho, _lib
    from synthetic import make_config
    s = make_config(args.workload) if not args.frames else make_config(args.workload, J=args.frames)
    obj = torch.tensor(s.obj0, device=dev)
    probe = torch.tensor(s.probe0, device=dev)
    iobs = torch.tensor(s.iobs, device=dev)
    pb = Ptycho(obj, probe, iobs, s.positions, s.mask, with_psi=True)
    params = []
    if args.lanes:
        params.append(("lanes", args.lanes))
    if args.batch_frames:
        params.append(("batch_frames", args.batch_frames))
    if args.persistent:
        params.append(("persistent", 1))
    if args.tma is not None:
        params.append(("tma", args.tma))
    if args.tma_gather is not None:
        params.append(("tma_gather", args.tma_gather))
    if args.tc:
        params.append(("tc", args.tc))
    if args.tc_rows:
        params.append(("tc_rows", 1))
    if args.pdl is not None:
        params.append(("pdl", args.pdl))
    for name, val in params:
        pb.set_param(name, val)
    stream = torch.cuda.current_stream(dev)
    llk_buf = torch.empty(max(args.steps, args.warmup, 1), dtype=torch.float64, device=dev)

    # warm-up (the first cycle initialises Psi and captures the CUDA graphs)
    pb.dm(args.warmup, init_psi=True, llk=llk_buf)
    pb.dm(1, llk=llk_buf)
    torch.cuda.synchronize(dev)
    import ctypes
    nk = ctypes.c_int64()
    _lib.call("ptx_cycle_kernels", pb._handle(), _lib.PTX_ALGO_DM, _lib.PTX_UPDATE_OBJ | _lib.PTX_UPDATE_PROBE,
              ctypes.byref(nk))
    cycle_kernels = int(nk.value)

    # timed region: K DM cycles (inputs ~3 GB >> 129 MB L2, so no flush is needed),
    # repeated; each repeat is bracketed by a barrier and a synchronise, the
    # max over ranks is taken per repeat and the median of the repeats reported
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    rep_ms = []
    for _ in range(max(1, args.repeats)):
        barrier(ws)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pb.dm(args.steps, llk=llk_buf)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(ws)
        rep_ms.append(max_over_ranks(e0.elapsed_time(e1), ws))
    clk = clocks.stop()
    ms_max = statistics.median(rep_ms)
    value = s.J * args.steps * ws / (ms_max / 1e3)
    ms_per_step = ms_max / args.steps

    if args.timing_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms_per_step,
                              "workload": args.workload, "frames": s.J, "steps": args.steps, "repeats_ms": rep_ms,
                              "timing_only": True}), flush=True)
        pb.close()
        return

    # the other form of the metric's comparison on the same box and data: the
    # split-precision tensor-core column pass (TF32 hi + lo DFT stages) when the
    # plain form was timed above, and the plain form otherwise
    other = None
    if not args.no_form_comparison and s.N == 256 and s.K == 1:
        other = []
        variants = [(f, 0) for f in range(4) if f != args.tc] + [(f, 1) for f in (1, 2, 3)]
        for tc_other, rows in variants:
            pb.set_param("tc", tc_other)
            pb.set_param("tc_rows", rows)
            pb.dm(2, llk=llk_buf)  # capture the other form's graph
            torch.cuda.synchronize(dev)
            n_other = max(1, min(args.steps, 10))
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            pb.dm(n_other, llk=llk_buf)
            f1.record(stream)
            torch.cuda.synchronize(dev)
            ms_o = max_over_ranks(f0.elapsed_time(f1), ws) / n_other
            other.append({"form": FORMS_ALL[tc_other] if rows else FORMS[tc_other], "value": s.J * ws / (ms_o / 1e3),
                          "ms_per_step": ms_o, "steps": n_other})
        pb.set_param("tc", args.tc)
        pb.set_param("tc_rows", 1 if args.tc_rows else 0)
        pb.dm(1, llk=llk_buf)
        torch.cuda.synchronize(dev)

    # per-kernel durations, live, with events on the launch stream (direct launches)
    _lib.call("ptx_profile_enable", pb._handle(), 1)
    pb.dm(args.steps, llk=llk_buf)
    torch.cuda.synchronize(dev)
    nk = len(_lib.KERNEL_KINDS)
    launches = (ctypes.c_int64 * nk)()
    tot = (ctypes.c_double * nk)()
    _lib.call("ptx_profile_read", pb._handle(), nk, launches, tot)
    _lib.call("ptx_profile_enable", pb._handle(), 0)
    kstats = {name: {"launches": int(launches[i]), "total_ms": float(tot[i]),
                     "avg_us": (1e3 * tot[i] / launches[i]) if launches[i] else None}
              for i, name in enumerate(_lib.KERNEL_KINDS)}
    tot_ms = sum(v["total_ms"] for v in kstats.values()) or 1.0
    for v in kstats.values():
        v["share"] = v["total_ms"] / tot_ms

    # end to end through the public API with host buffers: every step copies its
    # intensity stack in from pinned host memory and reads the cycle's LLK back.
    form = e2e_form(args, s)
    e2e_value, e2e_bytes, e2e_copies, e2e_runs = run_e2e(args, s, pb, obj, probe, iobs, params, llk_buf, stream,
                                                         dev, ws, form)
    # the same leg with the wider upload forms (what a caller that sends uint16
    # counts or float32 frames moves)
    e2e_other = {}
    if args.e2e_dtype == "auto":
        for f in (("u16", "f32") if form == "u8" else ("f32",) if form == "u16" else ()):
            v, b, c, r = run_e2e(args, s, pb, obj, probe, iobs, params, llk_buf, stream, dev, ws, f)
            e2e_other[f] = {"value": v, "unit": UNIT, "h2d_bytes_per_step": int(b), "d2h_bytes_per_step": 8,
                            "copies": c, "runs": r}

    # roofline: the dominant kernel by time share, against the measured FMA peak
    from paper_2008_11511_gb300 import fma_tflops
    fma_peak = fma_tflops(dev)
    pk = peaks()
    models = kernel_models(s)
    dom = max(("row_fwd", "col", "row_bwd", "obj_gather"), key=lambda k: kstats[k]["total_ms"])
    ks = kstats[dom]
    nframes_per_launch = s.J * args.steps / ks["launches"]
    traffic = ncu_traffic(dom)
    if dom == "obj_gather":
        gbs = models[dom]["bytes"] * nframes_per_launch / (ks["avg_us"] * 1e-6) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / pk["hbm_gbs"], "peak_src": pk["src"],
                "alg_bytes_per_launch": models[dom]["bytes"] * nframes_per_launch, "traffic": traffic}
    else:
        flops = models[dom]["flops"] * nframes_per_launch
        alu_derived = 152 * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
        achieved_tflops = flops / (ks["avg_us"] * 1e-6) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved_tflops, "peak": fma_peak,
                "unit": "TFLOP/s", "frac": achieved_tflops / fma_peak,
                "peak_src": "measured: FP32 FMA probe (ptx_fma_peak) on this GPU, best of 3",
                "peak_derived": alu_derived, "frac_of_derived": achieved_tflops / alu_derived,
                "flops_per_launch": flops, "alg_bytes_per_launch": models[dom]["bytes"] * nframes_per_launch,
                "traffic": traffic}
    # the cycle against the HBM roof, on the scope table's algorithmic bytes:
    # J K px 16 (Psi read + written) + J px 4 (I) + Ho Wo 16 (O) + K px 16 (P);
    # beside it the bytes of this design, whose object update re-reads Psi'
    px = s.N * s.N
    single = s.J * s.K * px * 16 + s.J * px * 4 + s.Ho * s.Wo * 16 + s.K * px * 16
    cyc_gbs = single / (ms_per_step * 1e-3) / 1e9
    cyc_bytes = alg_bytes_per_cycle(s, "DM")
    roof_cycle = {"bound": "hbm", "achieved": cyc_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                  "frac": cyc_gbs / pk["hbm_gbs"], "peak_src": pk["src"], "alg_bytes_per_cycle": single,
                  "bytes_src": "J K px 16 + J px 4 + Ho Wo 16 + K px 16 (Psi read and written once)",
                  "with_psi_reread": {"alg_bytes_per_cycle": cyc_bytes,
                                      "frac": cyc_bytes / (ms_per_step * 1e-3) / 1e9 / pk["hbm_gbs"]}}

    extras = None
    if not args.no_extras:
        pb.close()
        del pb
        torch.cuda.synchronize(dev)
        extras = {"ml256": run_extra_ml(dev, fma_peak, ws), "modes512": run_extra_modes(dev, pk, ws),
                  "batched16": run_extra_batched(dev, ws)}
        pb = None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, J, dt = oracle_sample_rate(s, seconds=args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": f"one FP64 DM cycle on {J} of {s.J} frames (evenly spaced), full object; {dt:.1f} s"}

    # kernels in the timed region: per repeat, `steps` replays of the cycle graph
    # (its kernel nodes, counted by the library) and the per-call control kernel
    gpu_launches = len(rep_ms) * (args.steps * cycle_kernels + 1)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "desc": workload_desc(s), "form": FORMS[args.tc],
                           "parallelism": f"replicas x{ws}",
                           "l2": "inputs larger than L2 (Psi 2.1 GB + I 1.05 GB per replica); no flush"},
                "roofline": roof, "roofline_cycle": roof_cycle, "kernels": kstats, "other_form": other,
                "repeats_ms": rep_ms, "fma_peak_tflops": fma_peak, "extra": extras, "e2e_u16": e2e_other.get("u16"),
                "e2e_f32": e2e_other.get("f32"),
                "kernels_note": ("per-kernel times from a pass with one batch lane and direct launches (sum "
                                 f"{sum(v['total_ms'] for v in kstats.values()) / args.steps:.3f} ms per cycle); the "
                                 f"timed graph cycle ({ms_per_step:.3f} ms) runs two lanes whose batches overlap"),
                "clocks": clk, "gpu_launches": gpu_launches,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(e2e_bytes),
                        "d2h_bytes_per_step": 8, "steps": max(1, min(args.steps, 50)), "copies": e2e_copies,
                        "runs": e2e_runs},
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if pb is not None:
        pb.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-repeats", type=int, default=3,
                    help="timed runs of the end-to-end leg (median reported)")
    ap.add_argument("--workload", choices=("dm256", "modes512"), default=WORKLOAD,
                    help="the scan the timed cycles run on (the JSON line's metric is defined on dm256; the other "
                         "workloads are for profiling with --timing-only)")
    ap.add_argument("--frames", type=int, default=0,
                    help="use only the first FRAMES frames of the workload (small cases for profiling)")
    ap.add_argument("--no-form-comparison", action="store_true",
                    help="skip timing the other number format (plain FP32 vs the tensor-core column pass)")
    ap.add_argument("--e2e-dtype", choices=("auto", "u8", "u16", "f32"), default="auto",
                    help="intensity upload of the end-to-end leg: auto = the smallest exact form (one-byte counts "
                         "with escapes, uint16 counts, else float32), reported with the wider forms beside it")
    ap.add_argument("--copy-streams", type=int, default=1,
                    help="streams the end-to-end leg splits each step's intensity upload over")
    ap.add_argument("--lanes", type=int, default=0,
                    help="batches in flight per cycle (library default when 0)")
    ap.add_argument("--tma", type=int, choices=(0, 1), default=None,
                    help="column pass staged by tensor copies (1) or the register column pass (0, the library default)")
    ap.add_argument("--tma-gather", type=int, choices=(0, 1), default=None,
                    help="object gather fed by tensor copies (1, the library default) or the plain gather (0)")
    ap.add_argument("--pdl", type=int, choices=(0, 1), default=None,
                    help="batch passes launched as programmatic dependents (1, the library default) or plainly (0)")
    ap.add_argument("--tc", type=int, choices=(0, 1, 2, 3), default=0,
                    help="number format of the column pass's DFT stages: 0 FP32 (CUDA cores), or on the tensor "
                         "cores 1 TF32 hi+lo, 2 BF16 hi+mid+lo, 3 BF16 hi+lo")
    ap.add_argument("--tc-rows", action="store_true",
                    help="with --tc F, the row passes' DFT stages on the tensor cores too (timing-only profiling)")
    ap.add_argument("--persistent", action="store_true",
                    help="the cycle's batch passes as one persistent launch (work list with bounded waits)")
    ap.add_argument("--batch-frames", type=int, default=0,
                    help="upper bound on frames per batch (library default when 0)")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed repeats of the K-step region (the median is reported)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary workloads (ML gradient and CG step, three-mode 512^2 DM cycle)")
    ap.add_argument("--timing-only", action="store_true",
                    help="stop after the timed region (no per-kernel pass, e2e or CPU baseline)")
    args = ap.parse_args()
    if args.workload != WORKLOAD and not args.timing_only:
        raise SystemExit("--workload other than dm256 needs --timing-only")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
