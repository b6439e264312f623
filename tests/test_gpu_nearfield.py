"""Near-field (PropagateNearField) AP / DM cycles and LLK: CUDA path vs the
FP64 oracle, element by element, through the C ABI.  Tolerances as in
test_gpu_parity: 1e-5 relative L2 per FP32 cycle."""
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
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


def data_of(s):
    return oracle.Data.make(s.iobs, s.positions, s.mask, nearfield=s.nearfield)


def _warm(s, n_ap=1):
    data = data_of(s)
    o, p = s.obj0.astype(complex), s.probe0.astype(complex)
    for _ in range(n_ap):
        o, p, _ = oracle.ap_cycle(o, p, data)
    return data, o.astype(np.complex64), p.astype(np.complex64)


def _problem(s, o, p, **kw):
    from paper_2008_11511_gb300 import Ptycho
    return Ptycho(dev(o), dev(p), dev(s.iobs), s.positions, s.mask, nearfield=s.nearfield, **kw)


def _check(s, pb, o_ref, p_ref, tol, psi_ref=None):
    o = pb.obj.cpu().numpy()
    d = oracle.object_denominator(p_ref, s.positions, o.shape)
    ill = d > 1e-3 * d.max()
    assert rel(o[ill], o_ref[ill]) < tol
    assert rel(pb.probe.cpu().numpy(), p_ref) < tol
    if psi_ref is not None:
        assert rel(pb.psi.cpu().numpy(), psi_ref) < tol


@pytest.mark.parametrize("N,J,c", [(256, 24, 200.0), (128, 40, 35.0), (64, 60, 6.0)])
def test_near_field_ap_and_dm_cycles(N, J, c):
    """One AP cycle and two DM cycles from a warm state, with the 2 % mask,
    several batches (J frames, batch size capped below J) and ragged tails."""
    if N == 256:
        s = make_config("nf256", J=J, Ho=520, Wo=520)
    else:
        s = make_scan(f"nf{N}", N=N, J=J, Ho=3 * N, Wo=3 * N + 6, seed=50 + N, photons=1e8, step=N * 0.12,
                      probe_radius=N * 0.35, phase_coef=0.0, diffuser_phase=2.0, mask_fraction=0.02, nearfield=c)
    data, o0, p0 = _warm(s)
    pb = _problem(s, o0, p0)
    pb.set_param("batch_frames", max(1, J // 3 + 1))
    l1 = pb.ap(1).cpu().numpy()
    o, p, l = oracle.ap_cycle(o0, p0, data)
    _check(s, pb, o, p, TOL1)
    assert abs(l1[0] - l) < TOL1 * abs(l)
    pb.close()
    pb = _problem(s, o0, p0)
    pb.set_param("batch_frames", max(1, J // 3 + 1))
    l2 = pb.dm(2, init_psi=True).cpu().numpy()
    o, p, psi, ls = oracle.cycles("DM", o0, p0, data, 2)
    _check(s, pb, o, p, 2 * TOL1, psi_ref=psi)
    np.testing.assert_allclose(l2, ls, rtol=2 * TOL1)
    pb.close()


def test_near_field_llk_and_fixed_point():
    """ptx_llk in the near field equals the oracle's LLK; noise-free near-field
    data of the true object and probe give a zero LLK and a DM step that leaves
    the exit waves in place."""
    s = make_config("nf256", J=16, Ho=480, Wo=480, noise=False)
    data = data_of(s)
    o, p = s.obj_true.astype(np.complex64), s.probe_true.astype(np.complex64)
    pb = _problem(s, o, p)
    l = float(pb.llk())
    assert l < 1e-6 * float(s.iobs.sum())
    rng = np.random.default_rng(3)
    o2 = (s.obj_true * (1 + 0.05 * (rng.standard_normal(s.obj_true.shape)))).astype(np.complex64)
    pb2 = _problem(s, o2, p)
    ref = oracle.llk(o2, p, data)
    assert abs(float(pb2.llk()) - ref) < 1e-5 * ref
    pb.dm(1, init_psi=True)
    phi = oracle.obj_probe_to_psi(s.obj_true, s.probe_true, s.positions)
    assert rel(pb.psi.cpu().numpy(), phi) < 1e-5
    pb.close()
    pb2.close()


def test_near_field_rejects_modes_and_ml():
    from paper_2008_11511_gb300 import Ptycho
    from paper_2008_11511_gb300._lib import PtychoError
    s = make_config("nf256", J=4, Ho=400, Wo=400)
    p2 = np.concatenate([s.probe0, 0.1 * s.probe0]).astype(np.complex64)
    with pytest.raises(PtychoError):
        Ptycho(dev(s.obj0), dev(p2), dev(s.iobs), s.positions, s.mask, nearfield=s.nearfield)
    pb = _problem(s, s.obj0, s.probe0)
    with pytest.raises(PtychoError):
        pb.ml_grad()
    pb.close()
