"""Edge cases of the cycle on the GPU against the FP64 oracle: the maximum
number of probe modes, the largest frames with several modes, frames with no
photons and negative intensities, one-frame batches in three lanes, every
frame at one position, odd object widths at 256^2, and calls that do nothing."""
import numpy as np
import pytest

import oracle
from synthetic import make_config, make_scan

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
    return float(np.linalg.norm(np.ravel(np.asarray(a) - np.asarray(b))) / np.linalg.norm(np.ravel(b)))


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


def _problem(s, o, p, with_psi=True):
    from paper_2008_11511_gb300 import Ptycho
    return Ptycho(dev(o.astype(np.complex64)), dev(p.astype(np.complex64)), dev(s.iobs), s.positions, s.mask,
                  with_psi=with_psi)


def _warm(s):
    data = oracle.Data.make(s.iobs, s.positions, s.mask)
    o, p, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    return data, o.astype(np.complex64), p.astype(np.complex64)


def _check(s, pb, o, p, tol, psi=None):
    d = oracle.object_denominator(p, s.positions, (s.Ho, s.Wo))
    ill = d > 1e-3 * d.max()
    assert rel(pb.obj.cpu().numpy()[ill], o[ill]) < tol
    assert rel(pb.probe.cpu().numpy(), p) < tol
    if psi is not None:
        assert rel(pb.psi.cpu().numpy(), psi) < tol


@pytest.mark.parametrize("N,K,J", [(64, 8, 30), (128, 8, 12), (512, 8, 3)])
def test_maximum_modes_dm_cycle_llk_and_gradient(N, K, J):
    """PTX_MAX_MODES = 8 incoherent modes (512^2 frames included): one DM cycle,
    the exact LLK and its gradient against the oracle."""
    s = make_scan(f"k8_{N}", N=N, J=J, Ho=N + 40, Wo=N + 36, K=K, seed=500 + N, photons=1e6, step=N / 10,
                  probe="hg", probe_radius=N / 10, mode_powers=[0.5 ** i for i in range(K)], mask_fraction=0.02)
    data, o0, p0 = _warm(s)
    pb = _problem(s, o0, p0)
    l_gpu = float(pb.llk())
    l_ref = oracle.llk(o0, p0, data)
    assert abs(l_gpu - l_ref) < TOL1 * abs(l_ref)
    _, go, gp = pb.ml_grad()
    _, go_ref, gp_ref = oracle.ml_grad(o0, p0, data)
    assert rel(go.cpu().numpy(), go_ref) < 1e-4 and rel(gp.cpu().numpy(), gp_ref) < 1e-4
    llk = pb.dm(1, init_psi=True).cpu().numpy()
    o, p, psi, lr = oracle.cycles("DM", o0, p0, data, 1)
    _check(s, pb, o, p, TOL1 * 2, psi)
    assert abs(llk[0] - lr[0]) < TOL1 * abs(lr[0])
    pb.close()


def test_frames_without_photons_and_negative_intensities_dm():
    """Whole frames of zero photons (the projection sends their waves to zero,
    their LLK is sum I_c) and negative readings (treated as 0) in DM cycles."""
    s = make_config("ap64", J=40)
    s.iobs = s.iobs.copy()
    s.iobs[[3, 17, 31]] = 0.0
    s.iobs[5, 10:14, 20:30] = -3.0
    data, o0, p0 = _warm(s)
    pb = _problem(s, o0, p0)
    llk = pb.dm(2, init_psi=True).cpu().numpy()
    o, p, psi, lr = oracle.cycles("DM", o0, p0, data, 2)
    _check(s, pb, o, p, TOL1 * 2, psi)
    np.testing.assert_allclose(llk, lr, rtol=TOL1 * 2)
    pb.close()


def test_one_frame_batches_in_three_lanes():
    """Batches of a single frame spread over three lanes (the most launches per
    cycle and the smallest grids) give the oracle's DM cycles."""
    s = make_config("dm256", J=11, Ho=512, Wo=512)
    data, o0, p0 = _warm(s)
    pb = _problem(s, o0, p0)
    pb.set_param("lanes", 3)
    pb.set_param("batch_frames", 1)
    llk = pb.dm(2, init_psi=True).cpu().numpy()
    o, p, psi, lr = oracle.cycles("DM", o0, p0, data, 2)
    _check(s, pb, o, p, TOL1 * 2, psi)
    np.testing.assert_allclose(llk, lr, rtol=TOL1 * 2)
    pb.close()


def test_every_frame_at_one_position():
    """Degenerate overlap: all frames on the same patch (their exit waves differ
    only through their intensities); one AP and one DM cycle."""
    s = make_config("ap64", J=12)
    s.positions = np.tile(np.array([[70, 90]], dtype=np.int32), (12, 1))
    data, o0, p0 = _warm(s)
    pb = _problem(s, o0, p0)
    pb.ap(1)
    o, p, _ = oracle.ap_cycle(o0, p0, data)
    _check(s, pb, o, p, TOL1)
    pb.close()
    pb = _problem(s, o0, p0)
    pb.dm(1, init_psi=True)
    o, p, psi, _ = oracle.cycles("DM", o0, p0, data, 1)
    _check(s, pb, o, p, TOL1, psi)
    pb.close()


def test_odd_object_width_at_256_with_edge_and_odd_positions():
    """256^2 frames over a 517 x 521 object (odd width: the gather's tensor-copy
    windows start on the even column left of the tile) with frames flush with
    every edge and at odd columns; one DM cycle."""
    s = make_scan("odd256", N=256, J=14, Ho=517, Wo=521, seed=77, photons=1e6, step=24, probe_radius=40,
                  mask_fraction=0.02)
    edge = np.array([[0, 0], [0, 521 - 256], [517 - 256, 0], [517 - 256, 521 - 256], [0, 133], [131, 0],
                     [77, 265], [261, 1]], dtype=np.int32)
    s.positions[:len(edge)] = edge
    data, o0, p0 = _warm(s)
    pb = _problem(s, o0, p0)
    pb.dm(1, init_psi=True)
    o, p, psi, _ = oracle.cycles("DM", o0, p0, data, 1)
    _check(s, pb, o, p, TOL1, psi)
    pb.close()


def test_zero_cycles_do_nothing():
    """ncycles = 0 enqueues nothing: object, probe, exit waves and the LLK buffer
    are untouched."""
    from paper_2008_11511_gb300 import Ptycho
    s = make_config("ap64", J=10)
    o0, p0 = s.obj0.copy(), s.probe0.copy()
    pb = Ptycho(dev(o0), dev(p0), dev(s.iobs), s.positions, s.mask, with_psi=True)
    pb.dm(1, init_psi=True)
    before = [t.clone() for t in (pb.obj, pb.probe, pb.psi)]
    buf = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    pb.dm(0, llk=buf)
    pb.ap(0, llk=buf)
    torch.cuda.synchronize()
    for t, b in zip((pb.obj, pb.probe, pb.psi), before):
        assert torch.equal(t, b)
    assert buf.cpu().tolist() == [7.0, 7.0]
    pb.close()


def test_set_param_refuses_bad_names_and_values_and_keeps_the_handle():
    """ptx_set_param on a live handle: unknown names and values outside each
    parameter's range come back as PTX_ERR_INVALID_ARG, change nothing, and the
    handle then runs a cycle that matches the oracle."""
    from paper_2008_11511_gb300 import PtychoError
    s = make_config("ap64", J=10)
    data, o0, p0 = _warm(s)
    pb = _problem(s, o0, p0)
    bad = [("no_such_parameter", 1.0), ("lanes", 0.0), ("lanes", 5.0), ("lanes", 1.5), ("tc", 4.0),
           ("tc_rows", 2.0), ("persistent", 0.5), ("tma", 2.0), ("pdl", 0.5), ("batch_frames", 1.5),
           ("bwd_slots", 5000.0), ("alpha_obj", -1.0), ("alpha_probe", float("nan")), ("tc_selftest", 3.0)]
    for name, value in bad:
        with pytest.raises(PtychoError) as ei:
            pb.set_param(name, value)
        assert ei.value.status_name == "PTX_ERR_INVALID_ARG", (name, value)
    for name, value in [("lanes", 3.0), ("lanes", 2.0), ("tc", 0.0), ("tc_rows", 0.0), ("batch_frames", 0.0)]:
        pb.set_param(name, value)
    pb.ap(1)
    o, p, _ = oracle.ap_cycle(o0, p0, data)
    _check(s, pb, o, p, TOL1)
    pb.close()


def test_dependent_launches_match_plain_launches():
    """The batch passes launched as programmatic dependents (the default) and
    plainly ("pdl" 0), in batches of 24 frames over two lanes: both give the
    oracle's LLK and two DM cycles; the LLK (no atomics on its path) is
    bit-identical, the gradient and the cycles agree to FP32 rounding (the
    probe sums and the gradient scatter are atomic additions in arbitrary
    order).  The gradient is not compared with the oracle here: one AP cycle
    from the start leaves pixels of small I_c whose weight 2(1 - I_o/I_c)
    amplifies float32 rounding (the full-size gradient test covers the
    dependent chain of eight batches against the oracle)."""
    s = make_config("dm256", J=150, Ho=640, Wo=640)
    data, o0, p0 = _warm(s)
    l_ref = oracle.llk(o0, p0, data)
    o, p, psi, lr = oracle.cycles("DM", o0, p0, data, 2)
    out = {}
    for pdl in (1, 0):
        pb = _problem(s, o0, p0)
        pb.set_param("pdl", pdl)
        pb.set_param("batch_frames", 24)
        l0 = float(pb.llk())
        assert abs(l0 - l_ref) < TOL1 * abs(l_ref)
        _, go, gp = pb.ml_grad()
        llk = pb.dm(2, init_psi=True).cpu().numpy()
        _check(s, pb, o, p, TOL1 * 2, psi)
        np.testing.assert_allclose(llk, lr, rtol=TOL1 * 2)
        out[pdl] = dict(l0=l0, go=go.cpu().numpy(), gp=gp.cpu().numpy(), llk=llk, obj=pb.obj.cpu().numpy(),
                        probe=pb.probe.cpu().numpy(), psi=pb.psi.cpu().numpy())
        pb.close()
    a, b = out[1], out[0]
    assert a["l0"] == b["l0"]
    for k in ("go", "gp", "obj", "probe"):
        assert rel(a[k], b[k]) < 1e-6, k
    assert rel(a["psi"], b["psi"]) < 1e-5
    np.testing.assert_allclose(a["llk"], b["llk"], rtol=1e-6)
