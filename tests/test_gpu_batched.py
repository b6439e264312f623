"""Batched uneven scans through one handle (ptx_cycles): problems of different
frame sizes and scan lengths, AP and DM alternately, each against its own FP64
oracle cycle; and the schedule autotuner restoring the state it tunes on."""
import numpy as np
import pytest

import oracle
from synthetic import make_scan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL1 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2008_11511_gb300 import build as b
    b.build()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


def _problems():
    specs = [(128, 150), (192, 60), (256, 90), (384, 30), (512, 20), (64, 300)]
    out = []
    for i, (N, J) in enumerate(specs):
        step = N / 10
        ext = int(2 * step / np.sqrt(np.pi) * np.sqrt(J)) + N + 8
        s = make_scan(f"b{i}", N=N, J=J, Ho=ext, Wo=ext + 4, seed=200 + i, photons=10 ** (4 + i % 3), step=step,
                      probe_radius=N * 0.16, mask_fraction=0.02 if i % 2 else 0.0)
        data = oracle.Data.make(s.iobs, s.positions, s.mask)
        o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
        out.append((s, data, o0.astype(np.complex64), p0.astype(np.complex64)))
    return out


def test_batched_cycles_match_oracle_per_problem():
    from paper_2008_11511_gb300 import PtychoBatch
    probs = _problems()
    algos = ["AP" if i % 2 == 0 else "DM" for i in range(len(probs))]
    items = [dict(obj=dev(o0), probe=dev(p0), iobs=dev(s.iobs), positions=s.positions, mask=s.mask)
             for s, data, o0, p0 in probs]
    pb = PtychoBatch(items)
    llk = pb.cycles(1, algos, init_psi=True).cpu().numpy()
    for i, ((s, data, o0, p0), a) in enumerate(zip(probs, algos)):
        if a == "AP":
            o, p, l = oracle.ap_cycle(o0, p0, data)
        else:
            o, p, psi, l = oracle.dm_cycle(o0, p0, None, data, init_psi=True)
            assert rel(pb.items[i]["psi"].cpu().numpy(), psi) < TOL1, i
        assert rel(pb.items[i]["obj"].cpu().numpy(), o) < TOL1, (i, a)
        assert rel(pb.items[i]["probe"].cpu().numpy(), p) < TOL1, (i, a)
        assert abs(llk[0, i] - l) < TOL1 * abs(l), (i, a, llk[0, i], l)
    pb.close()


def test_full_size_batched_workload_sampled():
    """The 16-scan batched workload at full size (22 245 frames, N from 128 to
    512, AP and DM alternately) through one handle, one cycle from the true
    objects and probes (DM from Psi = Phi): for each DM scan the new exit waves
    of four frames spread over the scan, for each AP scan of up to 1000 frames
    the cycle's LLK (the exact LLK at the truth), against the oracle."""
    from paper_2008_11511_gb300 import PtychoBatch
    from synthetic import batched_problem_specs
    specs = batched_problem_specs()
    scans = [make_scan(sp["name"], N=sp["N"], J=sp["J"], Ho=sp["Ho"], Wo=sp["Wo"], K=1, seed=sp["seed"],
                       photons=sp["photons"], step=sp["step"], probe_radius=sp["probe_radius"], mask_fraction=0.0)
             for sp in specs]
    algos = [sp["algorithm"] for sp in specs]
    truth = [(s.obj_true.astype(np.complex64), s.probe_true.astype(np.complex64)) for s in scans]
    items = [dict(obj=dev(o), probe=dev(p), iobs=dev(s.iobs), positions=s.positions, mask=s.mask)
             for s, (o, p) in zip(scans, truth)]
    pb = PtychoBatch(items)
    llk = pb.cycles(1, algos, init_psi=True).cpu().numpy()
    checked = 0
    for i, (s, (o, p), a) in enumerate(zip(scans, truth, algos)):
        if a == "DM":
            for j in np.linspace(0, s.J - 1, 4).astype(int):
                ref, _ = oracle.dm_frame_update(o, p, None, s.iobs[j], s.positions[j], s.mask, init_psi=True)
                assert rel(pb.items[i]["psi"][j].cpu().numpy(), ref) < TOL1, (i, j)
                checked += 1
        elif s.J <= 1000:
            data = oracle.Data.make(s.iobs, s.positions, s.mask)
            ref = oracle.frames_llk(o, p, data, np.arange(s.J))
            assert abs(llk[0, i] - ref) < TOL1 * abs(ref), (i, llk[0, i], ref)
            checked += 1
    assert checked >= 20
    pb.close()


def test_batched_equals_separate_handles_over_cycles():
    from paper_2008_11511_gb300 import Ptycho, PtychoBatch
    probs = _problems()[:3]
    algos = ["DM", "AP", "DM"]
    items = [dict(obj=dev(o0), probe=dev(p0), iobs=dev(s.iobs), positions=s.positions, mask=s.mask)
             for s, data, o0, p0 in probs]
    pb = PtychoBatch(items)
    pb.cycles(3, algos, init_psi=True)
    for i, (s, data, o0, p0) in enumerate(probs):
        one = Ptycho(dev(o0), dev(p0), dev(s.iobs), s.positions, s.mask)
        if algos[i] == "DM":
            one.dm(3, init_psi=True)
        else:
            one.ap(3)
        # the probe sums are FP32 atomic additions whose order varies between
        # runs (~1e-7 per cycle), amplified over three DM cycles
        assert rel(pb.items[i]["obj"].cpu().numpy(), one.obj.cpu().numpy()) < 1e-5
        assert rel(pb.items[i]["probe"].cpu().numpy(), one.probe.cpu().numpy()) < 1e-5
        one.close()
    pb.close()


def test_autotune_restores_state_and_sets_a_schedule():
    from paper_2008_11511_gb300 import Ptycho
    from paper_2008_11511_gb300.autotune import autotune
    s, data, o0, p0 = _problems()[2]
    pb = Ptycho(dev(o0), dev(p0), dev(s.iobs), s.positions, s.mask)
    pb.dm(1, init_psi=True)
    before = [t.clone() for t in (pb.obj, pb.probe, pb.psi)]
    best, times = autotune(pb, ["DM"], lanes=(1, 2), batch_frames=(0, 16), tma=(0, 1), bwd_slots=(0, 4),
                           use_cache=False)
    assert best in times and len(times) == 16
    for t, b in zip((pb.obj, pb.probe, pb.psi), before):
        assert torch.equal(t, b)
    # tuned schedule gives the same cycle as the default one
    ref = Ptycho(before[0].clone(), before[1].clone(), dev(s.iobs), s.positions, s.mask, psi=before[2].clone())
    pb.dm(1)
    ref.dm(1)
    assert rel(pb.obj.cpu().numpy(), ref.obj.cpu().numpy()) < 1e-6
    pb.close()
    ref.close()


def _cycle_kernels(pb, algo):
    import ctypes
    from paper_2008_11511_gb300 import _lib
    n = ctypes.c_int64()
    _lib.call("ptx_cycle_kernels", pb._handle(), algo, _lib.PTX_UPDATE_OBJ | _lib.PTX_UPDATE_PROBE, ctypes.byref(n))
    return n.value


def test_persistent_schedule_matches_oracle_per_problem():
    """The batch passes of five scans (128^2 to 512^2, AP and DM alternately) as
    one persistent launch per cycle: each problem against its own FP64 oracle
    cycle, and three cycles against the per-batch launches."""
    from paper_2008_11511_gb300 import PtychoBatch, _lib
    probs = _problems()[:5]
    algos = ["AP" if i % 2 == 0 else "DM" for i in range(len(probs))]
    items = [dict(obj=dev(o0), probe=dev(p0), iobs=dev(s.iobs), positions=s.positions, mask=s.mask)
             for s, data, o0, p0 in probs]
    pb = PtychoBatch(items)
    n_batches = _cycle_kernels(pb, _lib.PTX_ALGO_DM)
    pb.set_param("persistent", 1)
    n_pers = _cycle_kernels(pb, _lib.PTX_ALGO_DM)
    assert n_pers < n_batches  # one launch replaces the per-batch launches
    llk = pb.cycles(1, algos, init_psi=True).cpu().numpy()
    for i, ((s, data, o0, p0), a) in enumerate(zip(probs, algos)):
        if a == "AP":
            o, p, l = oracle.ap_cycle(o0, p0, data)
        else:
            o, p, psi, l = oracle.dm_cycle(o0, p0, None, data, init_psi=True)
            assert rel(pb.items[i]["psi"].cpu().numpy(), psi) < TOL1, i
        assert rel(pb.items[i]["obj"].cpu().numpy(), o) < TOL1, (i, a)
        assert rel(pb.items[i]["probe"].cpu().numpy(), p) < TOL1, (i, a)
        assert abs(llk[0, i] - l) < TOL1 * abs(l), (i, llk[0, i], l)
    pb.close()
    # three cycles, persistent against per-batch launches, with small batches (many slots reused)
    ref = PtychoBatch([dict(obj=dev(o0), probe=dev(p0), iobs=dev(s.iobs), positions=s.positions, mask=s.mask)
                       for s, data, o0, p0 in probs])
    per = PtychoBatch([dict(obj=dev(o0), probe=dev(p0), iobs=dev(s.iobs), positions=s.positions, mask=s.mask)
                       for s, data, o0, p0 in probs])
    per.set_param("persistent", 1)
    per.set_param("batch_frames", 7)
    l_ref = ref.cycles(3, algos, init_psi=True).cpu().numpy()
    l_per = per.cycles(3, algos, init_psi=True).cpu().numpy()
    np.testing.assert_allclose(l_per, l_ref, rtol=1e-5)
    for i in range(len(probs)):
        assert rel(per.items[i]["obj"].cpu().numpy(), ref.items[i]["obj"].cpu().numpy()) < 1e-5
        assert rel(per.items[i]["probe"].cpu().numpy(), ref.items[i]["probe"].cpu().numpy()) < 1e-5
    ref.close()
    per.close()


def test_persistent_schedule_wait_gives_up_and_reports():
    """A dependency that is never met (the self-test switch) makes the
    persistent launch's bounded wait give up: the next call reports
    PTX_ERR_TIMEOUT once, and the handle then runs correct cycles again."""
    from paper_2008_11511_gb300 import PtychoBatch, PtychoError
    probs = _problems()[2:3]
    s, data, o0, p0 = probs[0]
    pb = PtychoBatch([dict(obj=dev(o0), probe=dev(p0), iobs=dev(s.iobs), positions=s.positions, mask=s.mask)])
    pb.set_param("persistent", 1)
    pb.set_param("persistent_selftest", 1)
    pb.cycles(1, ["AP"])
    torch.cuda.synchronize()
    with pytest.raises(PtychoError, match="TIMEOUT"):
        pb.cycles(1, ["AP"])
    pb.set_param("persistent_selftest", 0)
    pb.items[0]["obj"].copy_(dev(o0))
    pb.items[0]["probe"].copy_(dev(p0))
    pb.cycles(1, ["AP"])
    o, p, _ = oracle.ap_cycle(o0, p0, data)
    assert rel(pb.items[0]["obj"].cpu().numpy(), o) < TOL1
    pb.close()
