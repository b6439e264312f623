"""Incoherent background (AP optimisation, LLK, gradient): CUDA path vs the
FP64 oracle through the C ABI, at the FP32 tolerances of test_gpu_parity."""
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
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


def _problem(N, J, nearfield=0.0, seed=70):
    """A scan whose intensities carry a smooth incoherent background (Poisson
    noise), the oracle's state after one background AP cycle as the common
    warm start, and a background guess 1.5x too high."""
    s = make_scan(f"bg{N}", N=N, J=J, Ho=2 * N + 20, Wo=2 * N + 26, seed=seed, photons=1e6, step=N / 8,
                  probe_radius=N * 0.16 if not nearfield else N * 0.35, mask_fraction=0.02, noise=False,
                  nearfield=nearfield, diffuser_phase=2.0 if nearfield else 0.0,
                  phase_coef=0.0 if nearfield else None)
    yy, xx = np.mgrid[0:N, 0:N]
    b_true = 20.0 * (1.0 + 0.5 * np.cos(2 * np.pi * yy / N) * np.cos(2 * np.pi * xx / N))
    iobs = np.random.default_rng(seed + 1).poisson(s.iobs.astype(np.float64) + b_true[None]).astype(np.float32)
    iobs[:, s.mask.astype(bool)] = 0.0
    data = oracle.Data.make(iobs, s.positions, s.mask, nearfield=nearfield)
    o, p, bg, _ = oracle.ap_cycle_background(s.obj0, s.probe0, 1.5 * b_true, data)
    return s, iobs, data, o.astype(np.complex64), p.astype(np.complex64), bg.astype(np.float32)


def _ptycho(s, iobs, o, p, bg, nearfield=0.0):
    from paper_2008_11511_gb300 import Ptycho
    return Ptycho(dev(o), dev(p), dev(iobs), s.positions, s.mask, background=dev(bg), nearfield=nearfield)


@pytest.mark.parametrize("N,J,nf", [(64, 60, 0.0), (256, 24, 0.0), (128, 30, 30.0)])
def test_background_ap_cycles_with_update(N, J, nf):
    """Two AP cycles updating O, P and the background, against the oracle."""
    s, iobs, data, o0, p0, b0 = _problem(N, J, nf)
    pb = _ptycho(s, iobs, o0, p0, b0, nf)
    llk = pb.ap(2, update_background=True).cpu().numpy()
    o, p, b = o0, p0, b0
    ls = []
    for _ in range(2):
        o, p, b, l = oracle.ap_cycle_background(o, p, b, data)
        ls.append(l)
    d = oracle.object_denominator(p, s.positions, o.shape)
    ill = d > 1e-3 * d.max()
    assert rel(pb.obj.cpu().numpy()[ill], o[ill]) < 2 * TOL1
    assert rel(pb.probe.cpu().numpy(), p) < 2 * TOL1
    assert rel(pb.background.cpu().numpy(), b) < 2 * TOL1
    np.testing.assert_allclose(llk, ls, rtol=2 * TOL1)
    pb.close()


def test_background_dm_llk_and_gradient():
    """DM and the exact LLK use I_c + B (background fixed), and so does the LLK
    gradient."""
    s, iobs, data, o0, p0, b0 = _problem(64, 60)
    d = oracle.Data.make(iobs, s.positions, s.mask, background=b0)
    pb = _ptycho(s, iobs, o0, p0, b0)
    l = float(pb.llk())
    ref = oracle.llk(o0, p0, d)
    assert abs(l - ref) < 1e-5 * ref
    llk = pb.dm(2, init_psi=True).cpu().numpy()
    o, p, psi, ls = oracle.cycles("DM", o0, p0, d, 2)
    assert rel(pb.probe.cpu().numpy(), p) < 2 * TOL1
    np.testing.assert_allclose(llk, ls, rtol=2 * TOL1)
    assert rel(pb.background.cpu().numpy(), b0) == 0.0  # not updated in DM
    pb.close()
    pb = _ptycho(s, iobs, o0, p0, b0)
    _, go, gp = oracle.ml_grad(o0, p0, d)
    _, g_o, g_p = pb.ml_grad()
    assert rel(g_o.cpu().numpy(), go) < 1e-4 and rel(g_p.cpu().numpy(), gp) < 1e-4
    pb.close()
