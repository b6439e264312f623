"""Position refinement: the per-frame shift estimate against the oracle on the
same inputs, ptx_set_positions against the oracle cycle at the new positions,
and the refinement loop recovering perturbed positions."""
import numpy as np
import pytest

import oracle
from synthetic import make_config, make_scan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("cfg,J", [("ap64", 60), ("dm256", 24)])
def test_position_shifts_match_oracle_on_the_same_inputs(cfg, J):
    from paper_2008_11511_gb300 import Ptycho
    s = make_config(cfg, J=J) if cfg == "ap64" else make_config(cfg, J=J, Ho=600, Wo=600)
    data = oracle.Data.make(s.iobs, s.positions, s.mask)
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    # the exit waves after one amplitude projection, from the oracle
    phi = oracle.obj_probe_to_psi(o0, p0, s.positions)
    psi = data.from_detector(oracle.apply_amplitude(data.to_detector(phi), data.iobs, data.mask))
    psi = psi.astype(np.complex64)
    pb = Ptycho(dev(o0), dev(p0), dev(s.iobs), s.positions, s.mask, psi=dev(psi))
    d = pb.position_shifts(0.1).cpu().numpy()
    ref = oracle.position_shifts(o0, p0, psi, s.positions, 0.1)
    assert np.abs(d - ref).max() < 1e-3 * max(np.abs(ref).max(), 1e-2), np.abs(d - ref).max()
    assert np.array_equal(d == 0, ref == 0)
    pb.close()


def test_set_positions_then_cycle_matches_oracle():
    from paper_2008_11511_gb300 import Ptycho
    s = make_config("ap64", J=50)
    data = oracle.Data.make(s.iobs, s.positions, s.mask)
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    pb = Ptycho(dev(o0), dev(p0), dev(s.iobs), s.positions, s.mask)
    rng = np.random.default_rng(5)
    new = np.clip(s.positions + rng.integers(-3, 4, size=s.positions.shape), 0, s.Ho - s.N).astype(np.int32)
    pb.set_positions(new)
    l = pb.ap(1).cpu().numpy()
    o, p, lr = oracle.ap_cycle(o0, p0, oracle.Data.make(s.iobs, new, s.mask))
    assert rel(pb.probe.cpu().numpy(), p) < 1e-5
    d = oracle.object_denominator(p, new, o.shape)
    ill = d > 1e-3 * d.max()
    assert rel(pb.obj.cpu().numpy()[ill], o[ill]) < 1e-5
    assert abs(l[0] - lr) < 1e-5 * abs(lr)
    from paper_2008_11511_gb300._lib import PtychoError
    with pytest.raises(PtychoError):
        pb.set_positions(np.full_like(new, s.Ho))
    pb.close()


def test_refinement_recovers_perturbed_positions():
    """Known object and probe, data from the true positions, the handle created
    with positions off by up to 2 px: AP projections (object and probe held)
    and refinement steps bring every frame back to its true position."""
    from paper_2008_11511_gb300 import Ptycho
    s = make_scan("posref", N=64, J=40, Ho=200, Wo=200, seed=90, photons=1e7, step=12.0,
                  probe_radius=14.0, phase_coef=0.02, noise=False)
    rng = np.random.default_rng(91)
    start = np.clip(s.positions + rng.integers(-2, 3, size=s.positions.shape), 0, 200 - 64).astype(np.int32)
    pb = Ptycho(dev(s.obj_true.astype(np.complex64)), dev(s.probe_true.astype(np.complex64)), dev(s.iobs),
                start, s.mask)
    err0 = np.abs(start - s.positions).sum()
    for _ in range(15):
        pb.ap(1, update_obj=False, update_probe=False)
        pb.refine_positions(filter_ratio=0.1, step=1.0)
    err = np.abs(pb.positions - s.positions).sum()
    assert err0 > 20 and err <= err0 // 10, (err0, err)
    pb.close()
