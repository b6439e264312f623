"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 norm ||x - x_ref|| / ||x_ref||, float32 path vs float64
oracle): 1e-5 for one cycle (object, probe, exit waves, log-likelihood), 1e-4
after 20 or 100 cycles.  The object error is also measured on the illuminated
region (D_O > 1e-3 max D_O) where the update acts.

Both sides start from the same complex64 state.  The configured start points
(flat object, Gaussian-blurred probe) put up to half of the detector pixels
below the float32 FFT resolution (model amplitude < 1e-7 of the peak), where
any single-precision transform returns rounding noise and the amplitude
projection gives the observed photons that noise's phase.  Cycle parity is
therefore checked from "warm" states (the oracle's state after one or more AP
cycles, where the spectrum is filled), and the configured start itself is
checked against an independent single-precision evaluation of the same cycle
(test_configured_start_is_at_the_float32_floor).
"""
import copy
import ctypes
import functools

import scipy.fft
import numpy as np
import pytest

import oracle
from synthetic import make_config, make_scan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL1 = 1e-5     # one float32 cycle
TOL20 = 1e-4    # many cycles


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


def to_dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


def gpu_problem(s, with_psi=True, obj=None, probe=None):
    from paper_2008_11511_gb300 import Ptycho
    o = to_dev((s.obj0 if obj is None else obj).astype(np.complex64))
    p = to_dev((s.probe0 if probe is None else probe).astype(np.complex64))
    return Ptycho(o, p, to_dev(s.iobs), s.positions, s.mask, with_psi=with_psi)


def data_of(s):
    return oracle.Data.make(s.iobs, s.positions, s.mask)


def illuminated(s, probe):
    d = oracle.object_denominator(probe, s.positions, (s.Ho, s.Wo))
    return d > 1e-3 * d.max()


def check_close(name, got, ref, tol):
    e = rel(got, ref)
    assert e < tol, f"{name}: rel err {e:.3e} >= {tol:.0e}"
    return e


@functools.lru_cache(maxsize=None)
def _warm_cached(cfg, J, n_ap, over):
    s = make_config(cfg, J=J, **dict(over))
    o, p = s.obj0.astype(complex), s.probe0.astype(complex)
    data = data_of(s)
    for _ in range(n_ap):
        o, p, _ = oracle.ap_cycle(o, p, data)
    return s, o.astype(np.complex64), p.astype(np.complex64)


def warm(cfg, J=None, n_ap=1, **over):
    """(scan, obj, probe): the oracle's state after n_ap AP cycles from the
    configured start, rounded to complex64 (the common start of both sides)."""
    s, o, p = _warm_cached(cfg, J, n_ap, tuple(sorted(over.items())))
    return copy.copy(s), o.copy(), p.copy()


# ------------------------------------------------------------------ FT / IFT

@pytest.mark.parametrize("N", [8, 12, 16, 32, 64, 80, 128, 160, 192, 224, 256, 384, 400, 448, 512])
def test_fft2_matches_oracle(N):
    from paper_2008_11511_gb300 import fft2
    rng = np.random.default_rng(N)
    nf = 5
    x = (rng.standard_normal((nf, N, N)) + 1j * rng.standard_normal((nf, N, N))).astype(np.complex64)
    X = to_dev(x)
    fft2(X, -1)
    ref = oracle.ft(x.astype(np.complex128))
    check_close(f"FT N={N}", X.cpu().numpy(), ref, 2e-6)
    fft2(X, +1)
    check_close(f"IFT(FT) N={N}", X.cpu().numpy(), x, 3e-6)


@pytest.mark.parametrize("N", [32, 80, 192, 224, 256, 400])
def test_fft2_special_inputs(N):
    from paper_2008_11511_gb300 import fft2
    d = np.zeros((3, N, N), np.complex64)
    d[0, 0, 0] = 1.0                                   # delta -> constant 1/N
    d[1] = 1.0                                          # constant -> N delta at DC
    yy, xx = np.mgrid[0:N, 0:N]
    d[2] = np.exp(2j * np.pi * (3 * yy + 5 * xx) / N)   # single frequency -> N delta at (3, 5)
    X = to_dev(d)
    fft2(X, -1)
    got = X.cpu().numpy()
    exp0 = np.full((N, N), 1.0 / N)
    exp1 = np.zeros((N, N)); exp1[0, 0] = N
    exp2 = np.zeros((N, N), complex); exp2[3, 5] = N
    assert np.abs(got[0] - exp0).max() < 1e-6
    assert np.abs(got[1] - exp1).max() < 1e-3
    assert np.abs(got[2] - exp2).max() < 2e-3


def test_fft2_direct_dft_small():
    from paper_2008_11511_gb300 import fft2
    rng = np.random.default_rng(3)
    for N in (8, 12, 16):
        x = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
        ref = np.zeros((N, N), complex)
        y = np.arange(N)
        for ky in range(N):
            for kx in range(N):
                ref[ky, kx] = (x * np.exp(-2j * np.pi * (ky * y[:, None] + kx * y[None, :]) / N)).sum() / N
        X = to_dev(x[None])
        fft2(X, -1)
        check_close(f"direct DFT N={N}", X.cpu().numpy()[0], ref, 1e-6)


# ------------------------------------------------------------------ LLK and gradient

@pytest.mark.parametrize("cfg,J", [("ap64", 100), ("ml32fd", 16), ("dm256", 40)])
def test_llk_exact_parity(cfg, J):
    s, o, p = warm(cfg, J=J)
    pb = gpu_problem(s, with_psi=False, obj=o, probe=p)
    g = float(pb.llk())
    ref = oracle.llk(o, p, data_of(s))
    assert abs(g - ref) / abs(ref) < TOL1, (g, ref)
    pb.close()


def test_llk_with_mask_and_negative_intensities():
    s, o, p = warm("ap64", J=30, mask_fraction=0.05)
    s.iobs = s.iobs.copy()
    s.iobs[0, 5, 7] = -2.0          # negative observations are clamped to 0
    s.iobs[3, 0, 1] = -0.5
    pb = gpu_problem(s, with_psi=False, obj=o, probe=p)
    g = float(pb.llk())
    ref = oracle.llk(o, p, data_of(s))
    assert abs(g - ref) / abs(ref) < TOL1
    pb.close()


def test_llk_zero_at_noise_free_truth():
    s = make_config("ap64", J=40, noise=False)
    pb = gpu_problem(s, with_psi=False, obj=s.obj_true, probe=s.probe_true)
    g = float(pb.llk())
    assert 0 <= g < 1e-6 * float(s.iobs.sum()), g
    pb.close()


@pytest.mark.parametrize("cfg,J,tol", [("ml32fd", 16, 1e-4), ("ml256", 60, 1e-4)])
def test_ml_grad_parity(cfg, J, tol):
    """The gradient weight 2(1 - I_o/I_c) amplifies float32 errors of small I_c, so
    the comparison starts after 3 AP cycles (ML follows DM/AP in the paper's chains)."""
    s, obj, probe = warm(cfg, J=J, n_ap=3)
    pb = gpu_problem(s, with_psi=False, obj=obj, probe=probe)
    L, go, gp = pb.ml_grad()
    ref_L, ref_go, ref_gp = oracle.ml_grad(obj, probe, data_of(s))
    assert abs(float(L) - ref_L) / abs(ref_L) < TOL1
    check_close("G_O", go.cpu().numpy(), ref_go, tol)
    check_close("G_P", gp.cpu().numpy(), ref_gp, tol)
    pb.close()


def test_ml_grad_autograd_function():
    from paper_2008_11511_gb300 import PtychoLLK
    s, obj, probe = warm("ml32fd", n_ap=3)
    pb = gpu_problem(s, with_psi=False)
    o = to_dev(obj).requires_grad_(True)
    p = to_dev(probe).requires_grad_(True)
    L = PtychoLLK.apply(o, p, pb)
    (3.0 * L).backward()
    ref_L, ref_go, ref_gp = oracle.ml_grad(obj, probe, data_of(s))
    assert abs(float(L.detach()) - ref_L) / abs(ref_L) < TOL1
    check_close("autograd G_O", o.grad.cpu().numpy(), 3.0 * ref_go, 1e-4)
    check_close("autograd G_P", p.grad.cpu().numpy(), 3.0 * ref_gp, 1e-4)
    pb.close()


# ------------------------------------------------------------------ AP / DM cycles

def _compare_cycle_state(s, pb, o_ref, p_ref, tol, psi_ref=None):
    o = pb.obj.cpu().numpy()
    p = pb.probe.cpu().numpy()
    ill = illuminated(s, p_ref)
    e = {"obj": check_close("obj", o, o_ref, tol),
         "obj_ill": check_close("obj (illuminated)", o[ill], o_ref[ill], tol),
         "probe": check_close("probe", p, p_ref, tol)}
    if psi_ref is not None:
        e["psi"] = check_close("psi", pb.psi.cpu().numpy(), psi_ref, tol)
    return e


def test_ap_one_cycle_parity():
    s, o0, p0 = warm("ap64")
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    llk = pb.ap(1).cpu().numpy()
    o, p, l = oracle.ap_cycle(o0, p0, data_of(s))
    _compare_cycle_state(s, pb, o, p, TOL1)
    assert abs(llk[0] - l) / abs(l) < TOL1
    pb.close()


def test_ap64_20_cycles_parity():
    """Plain AP, 64x64 probe, 256x256 object, 100 positions, 20 cycles."""
    s, o0, p0 = warm("ap64")
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    llk = pb.ap(20).cpu().numpy()
    o, p, _, llk_ref = oracle.cycles("AP", o0, p0, data_of(s), 20)
    _compare_cycle_state(s, pb, o, p, TOL20)
    np.testing.assert_allclose(llk, llk_ref, rtol=TOL20)
    assert llk[-1] < llk[0]
    pb.close()


@pytest.mark.parametrize("flags", [(True, True), (True, False), (False, True), (False, False)])
def test_ap_update_flags(flags):
    s, o0, p0 = warm("ap64", J=30)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    pb.ap(2, update_obj=flags[0], update_probe=flags[1])
    o, p, _, _ = oracle.cycles("AP", o0, p0, data_of(s), 2, update_obj=flags[0], update_probe=flags[1])
    _compare_cycle_state(s, pb, o, p, TOL1 * 2)
    if not flags[0]:
        assert np.array_equal(pb.obj.cpu().numpy(), o0)
    if not flags[1]:
        assert np.array_equal(pb.probe.cpu().numpy(), p0)
    pb.close()


def test_dm_cycles_parity_256_masked_ragged_batches():
    """DM on 256x256 frames with the 2% detector-gap mask; J = 300 spans three
    batches of the Fourier work stack with a ragged last batch."""
    s, o0, p0 = warm("dm256", J=300, Ho=768, Wo=768)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    llk = pb.dm(3, init_psi=True).cpu().numpy()
    o, p, psi, llk_ref = oracle.cycles("DM", o0, p0, data_of(s), 3)
    _compare_cycle_state(s, pb, o, p, TOL1 * 3, psi_ref=psi)
    np.testing.assert_allclose(llk, llk_ref, rtol=TOL1 * 3)
    pb.close()


def test_dm_one_cycle_parity_from_given_psi():
    s = make_config("ap64", J=50)
    rng = np.random.default_rng(5)
    phi = oracle.obj_probe_to_psi(s.obj0.astype(complex), s.probe0.astype(complex), s.positions)
    psi0 = (phi + 0.1 * (rng.standard_normal(phi.shape) + 1j * rng.standard_normal(phi.shape))).astype(np.complex64)
    from paper_2008_11511_gb300 import Ptycho
    pb = Ptycho(to_dev(s.obj0), to_dev(s.probe0), to_dev(s.iobs), s.positions, s.mask, psi=to_dev(psi0))
    llk = pb.dm(1).cpu().numpy()
    o, p, psi, l = oracle.dm_cycle(s.obj0, s.probe0, psi0, data_of(s))
    _compare_cycle_state(s, pb, o, p, TOL1, psi_ref=psi)
    assert abs(llk[0] - l) / abs(l) < TOL1
    pb.close()


def test_graph_and_direct_launch_agree():
    s, o0, p0 = warm("ap64", J=60)
    a = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    b = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    la = a.dm(3, init_psi=True, graph=True).cpu().numpy()
    lb = b.dm(3, init_psi=True, graph=False).cpu().numpy()
    assert rel(a.obj.cpu().numpy(), b.obj.cpu().numpy()) < 1e-6
    assert rel(a.probe.cpu().numpy(), b.probe.cpu().numpy()) < 1e-6
    np.testing.assert_allclose(la, lb, rtol=1e-6)
    a.close(); b.close()


# ------------------------------------------------------------------ modes

def test_multimode_dm_parity():
    """Three orthogonalised Hermite-Gauss modes (powers 0.7/0.2/0.1), 512x512 frames."""
    s, o0, p0 = warm("modes512", J=24, Ho=1024, Wo=1024)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    llk = pb.dm(2, init_psi=True).cpu().numpy()
    o, p, psi, llk_ref = oracle.cycles("DM", o0, p0, data_of(s), 2)
    _compare_cycle_state(s, pb, o, p, TOL1 * 2, psi_ref=psi)
    np.testing.assert_allclose(llk, llk_ref, rtol=TOL1 * 2)
    pb.close()


def test_multimode_dm_trajectory():
    """Six DM cycles of three modes at 512^2 from the oracle's warm state: the
    per-cycle LLK (of the reflected wave, which grows under DM here as it does
    in the oracle) and the final object and probe against the oracle."""
    s, o0, p0 = warm("modes512", J=40, Ho=1100, Wo=1100)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    llk = pb.dm(6, init_psi=True).cpu().numpy()
    o, p, psi, llk_ref = oracle.cycles("DM", o0, p0, data_of(s), 6)
    np.testing.assert_allclose(llk, llk_ref, rtol=1e-5)
    _compare_cycle_state(s, pb, o, p, 1e-5, psi_ref=psi)
    pb.close()


@pytest.mark.parametrize("N,K,J,algo", [
    (256, 2, 150, "DM"),   # several batches of (frame, mode) blocks, ragged last batch
    (384, 2, 10, "AP"),    # 16-column blocks, row backward with the 16-point factor second
    (448, 3, 8, "DM"),
    (160, 2, 20, "AP"),    # radix-5 factors
    (64, 3, 40, "DM"),     # several lines per thread
])
def test_multimode_register_passes(N, K, J, algo):
    """K Hermite-Gauss modes through the register-resident passes: one cycle
    (DM from Psi = Phi) from the oracle's warm state, object, probe, exit waves
    and LLK against the oracle."""
    s = make_scan(f"mm{N}", N=N, J=J, Ho=N + 6 * int(N / 8) + 8, Wo=N + 6 * int(N / 8) + 2, K=K, seed=N + K,
                  photons=1e6, step=N / 8, probe="hg", probe_radius=N / 10, mode_powers=[0.7, 0.2, 0.1][:K],
                  mask_fraction=0.02)
    data = data_of(s)
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    if algo == "DM":
        llk = pb.dm(1, init_psi=True).cpu().numpy()
        o, p, psi, l = oracle.cycles("DM", o0, p0, data, 1)
    else:
        llk = pb.ap(1).cpu().numpy()
        o, p, l = oracle.ap_cycle(o0, p0, data)
        psi = None
    _compare_cycle_state(s, pb, o, p, TOL1 * 2, psi_ref=psi)
    np.testing.assert_allclose(llk, np.atleast_1d(l), rtol=TOL1 * 2)
    pb.close()


@pytest.mark.parametrize("N,K,J", [(64, 2, 24), (256, 2, 12)])
def test_multimode_ml_grad_parity(N, K, J):
    s = make_scan(f"mg{N}", N=N, J=J, Ho=N + 5 * int(N / 8) + 4, Wo=N + 5 * int(N / 8) + 4, K=K, seed=3 * N + K,
                  photons=1e5, step=N / 8, probe="hg", probe_radius=N / 10, mode_powers=[0.8, 0.2],
                  mask_fraction=0.02)
    data = data_of(s)
    o, p = s.obj0, s.probe0
    for _ in range(3):
        o, p, _ = oracle.ap_cycle(o, p, data)
    o, p = o.astype(np.complex64), p.astype(np.complex64)
    pb = gpu_problem(s, with_psi=False, obj=o, probe=p)
    L, go, gp = pb.ml_grad()
    ref_L, ref_go, ref_gp = oracle.ml_grad(o, p, data)
    assert abs(float(L) - ref_L) / abs(ref_L) < TOL1
    check_close("G_O", go.cpu().numpy(), ref_go, 1e-4)
    check_close("G_P", gp.cpu().numpy(), ref_gp, 1e-4)
    pb.close()


def test_zero_extra_mode_equals_single_mode():
    s, o0, p0 = warm("ap64", J=30)
    p2 = np.concatenate([p0, np.zeros_like(p0)])
    a = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    b = gpu_problem(s, with_psi=True, obj=o0, probe=p2)
    a.ap(2, update_probe=False)
    b.ap(2, update_probe=False)
    assert rel(b.obj.cpu().numpy(), a.obj.cpu().numpy()) < 1e-6
    a.close(); b.close()


# ------------------------------------------------------------------ edge cases

@pytest.mark.parametrize("N", [32, 80, 160, 192, 224, 384, 400, 448])
def test_other_frame_sizes_ap(N):
    s = make_scan(f"n{N}", N=N, J=12, Ho=N + 40, Wo=N + 24, seed=N, photons=1e5, step=N / 12,
                  probe_radius=N * 0.18, mask_fraction=0.02)
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data_of(s))
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    llk = pb.ap(1).cpu().numpy()
    o, p, l = oracle.ap_cycle(o0, p0, data_of(s))
    _compare_cycle_state(s, pb, o, p, TOL1)
    assert abs(llk[0] - l) / abs(l) < TOL1
    pb.close()


def test_single_frame_object_equals_frame_corner_positions():
    """J = 1 and the object exactly one frame; then positions at both extreme corners."""
    s = make_scan("one", N=64, J=1, Ho=64, Wo=64, seed=11, photons=1e5, step=10, probe_radius=20)
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data_of(s))
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    pb.dm(2, init_psi=True)
    o, p, psi, _ = oracle.cycles("DM", o0, p0, data_of(s), 2)
    _compare_cycle_state(s, pb, o, p, TOL1 * 2, psi_ref=psi)
    pb.close()
    s2, o2, p2 = warm("ap64", J=4)
    s2.positions = np.array([[0, 0], [256 - 64, 256 - 64], [0, 256 - 64], [256 - 64, 0]], dtype=np.int32)
    o2, p2, _ = oracle.ap_cycle(o2, p2, data_of(s2))
    o2, p2 = o2.astype(np.complex64), p2.astype(np.complex64)
    pb = gpu_problem(s2, with_psi=True, obj=o2, probe=p2)
    pb.ap(1)
    o, p, _ = oracle.ap_cycle(o2, p2, data_of(s2))
    _compare_cycle_state(s2, pb, o, p, TOL1)
    pb.close()


def test_fully_masked_detector_leaves_waves_free():
    s, o0, p0 = warm("ap64", J=10)
    s.mask = np.ones_like(s.mask)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    llk = pb.ap(1).cpu().numpy()
    assert llk[0] == 0.0
    o, p, _ = oracle.ap_cycle(o0, p0, data_of(s))
    _compare_cycle_state(s, pb, o, p, TOL1)
    pb.close()


def test_zero_probe_region_gives_zero_not_nan():
    s, o0, p0 = warm("ap64", J=10)
    probe = np.zeros_like(p0)
    probe[0, 20:40, 20:40] = p0[0, 20:40, 20:40]
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=probe)
    llk = pb.ap(1).cpu().numpy()
    assert np.all(np.isfinite(pb.obj.cpu().numpy())) and np.all(np.isfinite(pb.probe.cpu().numpy()))
    o, p, l = oracle.ap_cycle(o0, probe, data_of(s))
    _compare_cycle_state(s, pb, o, p, TOL1)
    assert abs(llk[0] - l) / abs(l) < TOL1
    pb.close()


def test_out_of_bounds_position_is_rejected():
    from paper_2008_11511_gb300 import PtychoError
    s = make_config("ap64", J=5)
    s.positions[2] = [256 - 64 + 1, 3]
    with pytest.raises(PtychoError, match="OUT_OF_BOUNDS"):
        gpu_problem(s, with_psi=False)


def test_accumulators_and_external_normalise_match_internal():
    """Data-parallel form: cycles with normalise=False, then ptx_normalise, equal
    the fused cycle (the all-reduce of a multi-GPU split would sit in between)."""
    s, o0, p0 = warm("ap64", J=40)
    a = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    b = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    a.ap(1)
    b.ap(1, normalise=False)
    acc_o, acc_p = b.accumulators()
    assert float(acc_p[..., 2].max()) > 0
    assert float(acc_o.abs().max()) == 0.0  # the object sums are gathered after the probe update
    from paper_2008_11511_gb300.ptycho import PTX_STAGE_OBJ_GATHER, PTX_STAGE_OBJ_NORMALISE, PTX_STAGE_PROBE
    b.normalise(stages=PTX_STAGE_PROBE | PTX_STAGE_OBJ_GATHER)
    assert float(acc_o[..., 2].max()) > 0
    b.normalise(stages=PTX_STAGE_OBJ_NORMALISE)
    assert rel(b.obj.cpu().numpy(), a.obj.cpu().numpy()) < 1e-6
    assert rel(b.probe.cpu().numpy(), a.probe.cpu().numpy()) < 1e-6
    assert float(b.accumulators()[0].abs().max()) == 0.0
    a.close(); b.close()


# ------------------------------------------------------------------ long runs and conditioning

def test_dm_100_cycles_parity_noise_free():
    """DM, 100 cycles on noise-free 64x64-frame data from a start near the solution,
    where the iteration converges: <= 1e-4 after 100 float32 cycles."""
    s = make_config("ap64", noise=False)
    rng = np.random.default_rng(21)
    o0 = (s.obj_true * (1 + 0.02 * (rng.standard_normal(s.obj_true.shape)
                                     + 1j * rng.standard_normal(s.obj_true.shape)))).astype(np.complex64)
    p0 = (s.probe_true * (1 + 0.02 * (rng.standard_normal(s.probe_true.shape)
                                       + 1j * rng.standard_normal(s.probe_true.shape)))).astype(np.complex64)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    llk = pb.dm(100, init_psi=True).cpu().numpy()
    o, p, psi, llk_ref = oracle.cycles("DM", o0, p0, data_of(s), 100)
    _compare_cycle_state(s, pb, o, p, TOL20, psi_ref=psi)
    np.testing.assert_allclose(llk, llk_ref, rtol=TOL20)
    assert llk[-1] < llk[0]
    pb.close()


def _dm32_cycle(obj, probe, psi, data, init):
    """DM cycle with transforms and projection in complex64 (SciPy), overlap update
    as the oracle: an independent float32 evaluation."""
    obj32, probe32 = obj.astype(np.complex64), probe.astype(np.complex64)
    N = probe.shape[-1]
    phi = np.stack([probe32 * obj32[r:r + N, c:c + N][None] for r, c in data.positions])
    if init:
        psi = phi.copy()
    X = scipy.fft.fft2(2 * phi - psi, norm="ortho", axes=(-2, -1))
    ic = (np.abs(X) ** 2).sum(1)
    sc = np.where(data.mask, 1.0, np.sqrt(np.maximum(data.iobs, 0)) / np.maximum(np.sqrt(ic), 1e-20))
    psi = (psi + scipy.fft.ifft2(X * sc[:, None].astype(np.float32), norm="ortho", axes=(-2, -1)) - phi)
    psi = psi.astype(np.complex64)
    o, p = oracle.overlap_update(obj32.astype(complex), probe32.astype(complex), psi.astype(complex), data.positions)
    return o.astype(np.complex64), p.astype(np.complex64), psi


def test_dm_noisy_trajectory_per_cycle_and_drift():
    """On noisy data DM does not converge and its trajectory is sensitive to
    rounding: any float32 evaluation drifts from FP64 (about x1.8 per cycle here).
    Checked: one GPU cycle from the oracle's state at cycles 1, 10 and 30 matches
    to 1e-5, and over 20 cycles the GPU drifts no more than an independent
    single-precision implementation does."""
    s, o0, p0 = warm("ap64")
    data = data_of(s)
    from paper_2008_11511_gb300 import Ptycho
    o, p, psi = o0.astype(complex), p0.astype(complex), None
    for c in range(31):
        if c in (1, 10, 30):
            pb = Ptycho(to_dev(o.astype(np.complex64)), to_dev(p.astype(np.complex64)), to_dev(s.iobs), s.positions,
                        s.mask, psi=to_dev(psi.astype(np.complex64)))
            pb.dm(1)
            o1, p1, psi1, _ = oracle.dm_cycle(o.astype(np.complex64), p.astype(np.complex64),
                                              psi.astype(np.complex64), data)
            _compare_cycle_state(s, pb, o1, p1, TOL1, psi_ref=psi1)
            pb.close()
        o, p, psi, _ = oracle.dm_cycle(o, p, psi, data, init_psi=(c == 0))
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    pb.dm(20, init_psi=True)
    o64, p64, _, _ = oracle.cycles("DM", o0, p0, data, 20)
    o32, p32, psi32 = o0, p0, None
    for c in range(20):
        o32, p32, psi32 = _dm32_cycle(o32, p32, psi32, data, c == 0)
    e_gpu = rel(pb.obj.cpu().numpy(), o64)
    e_f32 = rel(o32, o64)
    assert e_gpu < 5 * e_f32 + TOL1, (e_gpu, e_f32)
    pb.close()


def _single_precision_ap_cycle(obj, probe, data):
    """The AP cycle with every transform and the projection in complex64 (SciPy's
    single-precision FFT), accumulation and normalisation as the oracle: an
    independent float32 evaluation used to measure the float32 floor."""
    obj32 = obj.astype(np.complex64)
    probe32 = probe.astype(np.complex64)
    N = probe.shape[-1]
    phi = np.stack([probe32 * obj32[r:r + N, c:c + N][None] for r, c in data.positions])
    X = scipy.fft.fft2(phi, norm="ortho", axes=(-2, -1))
    ic = (np.abs(X) ** 2).sum(1)
    sc = np.where(data.mask, 1.0, np.sqrt(np.maximum(data.iobs, 0)) / np.maximum(np.sqrt(ic), 1e-20))
    psi = scipy.fft.ifft2(X * sc[:, None].astype(np.float32), norm="ortho", axes=(-2, -1))
    return oracle.overlap_update(obj32.astype(complex), probe32.astype(complex), psi.astype(complex), data.positions)


@pytest.mark.parametrize("cfg,J", [("ap64", 100), ("dm256", 40)])
def test_configured_start_is_at_the_float32_floor(cfg, J):
    """From the configured start (flat object, blurred probe) one GPU AP cycle
    differs from FP64 by no more than an independent single-precision cycle does."""
    s = make_config(cfg, J=J)
    data = data_of(s)
    X = np.abs(oracle.ft(oracle.obj_probe_to_psi(s.obj0.astype(complex), s.probe0.astype(complex),
                                                 s.positions[:1])))[0, 0]
    assert (X < 1e-7 * X.max()).mean() > 0.01  # the start is ill-conditioned in float32
    pb = gpu_problem(s, with_psi=True)
    pb.ap(1)
    o64, p64, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    o32, p32 = _single_precision_ap_cycle(s.obj0, s.probe0, data)
    floor_o, floor_p = rel(o32, o64), rel(p32, p64)
    e_o, e_p = rel(pb.obj.cpu().numpy(), o64), rel(pb.probe.cpu().numpy(), p64)
    assert e_o < 2 * floor_o + TOL1 and e_p < 2 * floor_p + TOL1, (e_o, floor_o, e_p, floor_p)
    pb.close()


@pytest.mark.parametrize("N,J", [(64, 700), (80, 600), (128, 300), (160, 300), (192, 200), (224, 160), (384, 60),
                                 (400, 50), (448, 40), (512, 40)])
def test_several_frames_per_block_all_sizes(N, J):
    """Enough frames that every inverse-row block handles several frames (its
    staged rows are refilled between frames), for each register-kernel size:
    one AP and one DM cycle from a warm state."""
    step = N / 10
    ext = int(2 * step / np.sqrt(np.pi) * np.sqrt(J)) + N + 8
    s = make_scan(f"many{N}", N=N, J=J, Ho=ext, Wo=ext + 8, seed=100 + N, photons=1e5, step=step,
                  probe_radius=N * 0.16, mask_fraction=0.02)
    data = data_of(s)
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    llk = pb.ap(1).cpu().numpy()
    o, p, l = oracle.ap_cycle(o0, p0, data)
    _compare_cycle_state(s, pb, o, p, TOL1)
    assert abs(llk[0] - l) / abs(l) < TOL1
    pb.close()
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    pb.dm(1, init_psi=True)
    o, p, psi, _ = oracle.dm_cycle(o0, p0, None, data, init_psi=True)
    _compare_cycle_state(s, pb, o, p, TOL1, psi_ref=psi)
    pb.close()


TC_FORMS = {"register": 0, "tma": 0, "tc": 1, "bf16x3": 2}


@pytest.mark.parametrize("form", ["register", "tma", "tc", "bf16x3"])
@pytest.mark.parametrize("lanes,batch", [(1, 0), (2, 0), (2, 37)])
def test_dm256_column_pass_variants(form, lanes, batch):
    """The 256x256 column pass in its forms — FP32 registers, FP32 fed by tensor
    copies, DFT stages on the tensor cores (TF32 hi + lo, BF16 hi + mid + lo) —
    in one and two lanes and with a batch size (37 frames) that leaves ragged
    batches and a partial last wave of the persistent grid: three DM cycles and
    one AP cycle against the oracle, at the FP32 tolerance."""
    s, o0, p0 = warm("dm256", J=150, Ho=640, Wo=640)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    pb.set_param("tma", int(form == "tma"))
    pb.set_param("tc", TC_FORMS[form])
    pb.set_param("lanes", lanes)
    pb.set_param("batch_frames", batch)
    llk = pb.dm(3, init_psi=True).cpu().numpy()
    o, p, psi, llk_ref = oracle.cycles("DM", o0, p0, data_of(s), 3)
    _compare_cycle_state(s, pb, o, p, TOL1 * 3, psi_ref=psi)
    np.testing.assert_allclose(llk, llk_ref, rtol=TOL1 * 3)
    pb.close()
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    pb.set_param("tma", int(form == "tma"))
    pb.set_param("tc", TC_FORMS[form])
    pb.set_param("lanes", lanes)
    pb.set_param("batch_frames", batch)
    l1 = pb.ap(1).cpu().numpy()
    o, p, l = oracle.ap_cycle(o0, p0, data_of(s))
    _compare_cycle_state(s, pb, o, p, TOL1)
    assert abs(l1[0] - l) / abs(l) < TOL1
    pb.close()


def test_dm256_split_precision_forms_accuracy():
    """One DM cycle of each number format of the column pass's DFT stages,
    selected per call by the PTX_FORM_* flags, against the FP64 oracle: FP32,
    TF32 hi + lo and BF16 hi + mid + lo meet the single-cycle tolerance at the
    FP32 level (a few 1e-7); the two-term BF16 split (about 2^-16 per product)
    is measurably less accurate (here about 1e-6 to 7e-6 after one cycle, at
    least twice the FP32 distance) and is held to a bound of 1e-4.  The
    measured distances are printed."""
    from paper_2008_11511_gb300 import _lib
    s, o0, p0 = warm("dm256", J=60, Ho=512, Wo=512)
    o, p, psi, llk_ref = oracle.cycles("DM", o0, p0, data_of(s), 1)
    errs = {}
    for name, flag in (("fp32", 0), ("tf32x2", _lib.PTX_FORM_TF32X2), ("bf16x3", _lib.PTX_FORM_BF16X3),
                       ("bf16x2", _lib.PTX_FORM_BF16X2)):
        pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        f = _lib.PTX_UPDATE_OBJ | _lib.PTX_UPDATE_PROBE | _lib.PTX_DM_INIT_PSI | flag
        _lib.call("ptx_dm_cycles", pb._handle(), 1, f, ctypes.c_void_p(out.data_ptr()),
                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        ill = illuminated(s, p)
        errs[name] = (rel(pb.obj.cpu().numpy()[ill], o[ill]), rel(pb.probe.cpu().numpy(), p),
                      rel(pb.psi.cpu().numpy(), psi), abs(float(out.cpu()[0]) - llk_ref[0]) / abs(llk_ref[0]))
        pb.close()
        print(f"form {name}: obj {errs[name][0]:.2e} probe {errs[name][1]:.2e} psi {errs[name][2]:.2e} "
              f"llk {errs[name][3]:.2e}")
    for name in ("fp32", "tf32x2", "bf16x3"):
        assert max(errs[name]) < TOL1, (name, errs[name])
    assert 2 * max(errs["fp32"]) < max(errs["bf16x2"]) < 1e-4, errs


@pytest.mark.parametrize("form", [1, 2, 3])
@pytest.mark.parametrize("lanes,batch", [(2, 0), (1, 37)])
def test_dm256_all_dft_stages_on_tensor_cores(form, lanes, batch):
    """With "tc_rows" the forward and backward row passes run their DFT stages
    on the tensor cores too (every DFT stage of the cycle in the split form):
    three DM cycles and one AP cycle against the FP64 oracle, in two lanes and
    in one lane with ragged 37-frame batches; TF32 hi + lo and BF16 hi + mid +
    lo at the FP32 tolerance.  BF16 hi + lo keeps 16 significant bits per
    operand (about 2^-16 per product); with all eight DFT stages of a cycle in
    that form its distance after three DM cycles is about 1e-4, held to 3e-4."""
    tol = TOL1 * 3 if form in (1, 2) else 3e-4
    s, o0, p0 = warm("dm256", J=150, Ho=640, Wo=640)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    pb.set_param("tc", form)
    pb.set_param("tc_rows", 1)
    pb.set_param("lanes", lanes)
    pb.set_param("batch_frames", batch)
    llk = pb.dm(3, init_psi=True).cpu().numpy()
    o, p, psi, llk_ref = oracle.cycles("DM", o0, p0, data_of(s), 3)
    _compare_cycle_state(s, pb, o, p, tol, psi_ref=psi)
    np.testing.assert_allclose(llk, llk_ref, rtol=tol)
    pb.close()
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    pb.set_param("tc", form)
    pb.set_param("tc_rows", 1)
    pb.set_param("lanes", lanes)
    pb.set_param("batch_frames", batch)
    l1 = pb.ap(1).cpu().numpy()
    o, p, l = oracle.ap_cycle(o0, p0, data_of(s))
    _compare_cycle_state(s, pb, o, p, tol)
    assert abs(l1[0] - l) / abs(l) < tol
    pb.close()


@pytest.mark.parametrize("rows", [0, 1], ids=["column_pass", "every_stage"])
@pytest.mark.parametrize("K", [1, 3])
def test_modes512_split_precision_forms(K, rows):
    """The 512^2 column pass with its DFT stages on the tensor cores (a 16-point
    and a 32-point stage, the modes in two sweeps with the common factor), and
    with "tc_rows" the forward and backward row passes too (every DFT stage of
    the cycle), each number format against the FP64 oracle over one DM cycle
    and one AP cycle: TF32 hi + lo and BF16 hi + mid + lo at the single-cycle
    tolerance, BF16 hi + lo within its own bound.  The distances are printed."""
    from paper_2008_11511_gb300 import _lib
    s = make_scan(f"tc512_{K}", N=512, J=6, Ho=700, Wo=640, K=K, seed=90 + K, photons=1e7, step=51.2,
                  probe="hg", probe_radius=51.2, mode_powers=[0.7, 0.2, 0.1][:K], mask_fraction=0.02)
    data = data_of(s)
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    o, p, psi, llk_ref = oracle.cycles("DM", o0, p0, data, 1)
    oa, pa_, la = oracle.ap_cycle(o0, p0, data)
    errs = {}
    for name, flag in (("fp32", 0), ("tf32x2", _lib.PTX_FORM_TF32X2), ("bf16x3", _lib.PTX_FORM_BF16X3),
                       ("bf16x2", _lib.PTX_FORM_BF16X2)):
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
        pb.set_param("tc_rows", rows)
        f = _lib.PTX_UPDATE_OBJ | _lib.PTX_UPDATE_PROBE | flag
        _lib.call("ptx_dm_cycles", pb._handle(), 1, f | _lib.PTX_DM_INIT_PSI, ctypes.c_void_p(out.data_ptr()), stream)
        ill = illuminated(s, p)
        e_dm = (rel(pb.obj.cpu().numpy()[ill], o[ill]), rel(pb.probe.cpu().numpy(), p),
                rel(pb.psi.cpu().numpy(), psi), abs(float(out.cpu()[0]) - llk_ref[0]) / abs(llk_ref[0]))
        pb.close()
        pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
        pb.set_param("tc_rows", rows)
        _lib.call("ptx_ap_cycles", pb._handle(), 1, f, ctypes.c_void_p(out.data_ptr()), stream)
        e_ap = (rel(pb.obj.cpu().numpy()[ill], oa[ill]), rel(pb.probe.cpu().numpy(), pa_),
                abs(float(out.cpu()[0]) - la) / abs(la))
        pb.close()
        errs[name] = e_dm + e_ap
        print(f"512^2 K={K} rows={rows} form {name}: DM obj {e_dm[0]:.2e} probe {e_dm[1]:.2e} psi {e_dm[2]:.2e} "
              f"llk {e_dm[3]:.2e}; AP obj {e_ap[0]:.2e} probe {e_ap[1]:.2e} llk {e_ap[2]:.2e}")
    for name in ("fp32", "tf32x2", "bf16x3"):
        assert max(errs[name]) < 2 * TOL1, (name, errs[name])
    assert max(errs["bf16x2"]) < 1e-4, errs["bf16x2"]


@pytest.mark.parametrize("tg", [0, 1])
@pytest.mark.parametrize("case", ["corners64", "modes512"])
def test_object_gather_variants(tg, case):
    """The object update with the plain gather (0) and the gather fed by 3D
    tensor copies (1): frames flush with every object edge (their windows reach
    outside the frame on all sides) and, for three probe modes, several modes
    per frame.  One DM cycle against the oracle."""
    if case == "corners64":
        s = make_scan("corners64", N=64, J=60, Ho=200, Wo=203, seed=71, photons=1e5, step=9.0,
                      probe_radius=11, mask_fraction=0.02)
        edge = np.array([[0, 0], [0, 203 - 64], [200 - 64, 0], [200 - 64, 203 - 64], [0, 71], [99, 0]], dtype=np.int32)
        s.positions[:len(edge)] = edge
        s.iobs[:] = oracle.calc_intensity(oracle.ft(oracle.obj_probe_to_psi(s.obj_true, s.probe_true, s.positions)))
        data = data_of(s)
        o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
        o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    else:
        s, o0, p0 = warm("modes512", J=12, Ho=900, Wo=900)
        data = data_of(s)
    pb = gpu_problem(s, with_psi=True, obj=o0, probe=p0)
    pb.set_param("tma_gather", tg)
    pb.dm(1, init_psi=True)
    o, p, psi, _ = oracle.dm_cycle(o0, p0, None, data, init_psi=True)
    _compare_cycle_state(s, pb, o, p, TOL1, psi_ref=psi)
    pb.close()


def test_full_size_dm256_cycle_in_bench_configuration():
    """The headline workload at full size — 4000 frames of 256x256, 2048x2048 object,
    2 % mask — in bench.py's launch configuration (CUDA graph, two batch lanes):
    one DM cycle from an exit-wave stack Psi = P O + 10 % noise (well-conditioned
    in float32), against the FP64 oracle: every frame's Psi', the probe, the
    object (illuminated region) and the cycle's LLK.  The same cycle with every
    DFT stage on the tensor cores in the FP32-accurate splits (TF32 hi + lo,
    BF16 hi + mid + lo) meets the same tolerance."""
    s = make_config("dm256")
    data = data_of(s)
    rng = np.random.default_rng(30)
    phi = oracle.obj_probe_to_psi(s.obj0.astype(complex), s.probe0.astype(complex), s.positions)
    scale = 0.1 * np.sqrt(np.mean(np.abs(phi) ** 2))
    psi0 = (phi + scale * (rng.standard_normal(phi.shape) + 1j * rng.standard_normal(phi.shape))).astype(np.complex64)
    del phi
    from paper_2008_11511_gb300 import Ptycho
    o, p, psi, l = oracle.dm_cycle(s.obj0, s.probe0, psi0, data)
    for form, rows in ((0, 0), (1, 1), (2, 1)):
        pb = Ptycho(to_dev(s.obj0), to_dev(s.probe0), to_dev(s.iobs), s.positions, s.mask, psi=to_dev(psi0))
        pb.set_param("tc", form)
        pb.set_param("tc_rows", rows)
        llk = pb.dm(1).cpu().numpy()
        _compare_cycle_state(s, pb, o, p, TOL1, psi_ref=psi)
        assert abs(llk[0] - l) / abs(l) < TOL1, (form, llk[0], l)
        pb.close()



def test_full_size_modes512_cycle_sampled_frames():
    """The three-mode workload at full size — 10000 frames of 512x512, three
    modes, 6000x6000 object (Psi 62.9 GB on the device) — one DM cycle from
    Psi = Phi at the true object and probe (well conditioned: the model's far
    field carries the data's spectrum).  Every frame's new exit waves depend
    only on that frame, so the oracle computes a sample of 12 frames one by one."""
    s = make_config("modes512")
    o_t, p_t = s.obj_true.astype(np.complex64), s.probe_true.astype(np.complex64)
    pb = gpu_problem(s, with_psi=True, obj=o_t, probe=p_t)
    pb.dm(1, init_psi=True)
    for j in np.linspace(0, s.J - 1, 12).astype(int):
        ref, _ = oracle.dm_frame_update(o_t, p_t, None, s.iobs[j], s.positions[j], s.mask, init_psi=True)
        check_close(f"Psi' of frame {j}", pb.psi[j].cpu().numpy(), ref, TOL1)
    pb.close()


def test_full_size_ml256_gradient():
    """The ML workload at full size — 1000 frames of 256x256, 1536x1536 object —
    the LLK and its gradient at the true object and probe against the oracle."""
    s = make_config("ml256")
    o_t, p_t = s.obj_true.astype(np.complex64), s.probe_true.astype(np.complex64)
    pb = gpu_problem(s, with_psi=False, obj=o_t, probe=p_t)
    L, go, gp = pb.ml_grad()
    ref_L, ref_go, ref_gp = oracle.ml_grad(o_t, p_t, data_of(s))
    assert abs(float(L) - ref_L) / abs(ref_L) < TOL1
    check_close("G_O", go.cpu().numpy(), ref_go, 1e-4)
    check_close("G_P", gp.cpu().numpy(), ref_gp, 1e-4)
    pb.close()


# ------------------------------------------------------------------ ML conjugate gradient

def _oracle_direction(s, obj, probe, which):
    """Search direction (-G_O, -0.1 G_P) from the oracle's gradient, rounded to
    complex64; the part not in `which` is zero."""
    _, go, gp = oracle.ml_grad(obj, probe, data_of(s))
    d_o = (-go).astype(np.complex64) if which in ("obj", "both") else np.zeros_like(obj)
    d_p = (-0.1 * gp).astype(np.complex64) if which in ("probe", "both") else np.zeros_like(probe)
    return d_o, d_p


def _line_coeffs_fp32_bound(obj, probe, d_o, d_p, data, eta=1e-6):
    """First-order bound on how far single-precision waves can move (L'(0), L''(0)).

    The far-field waves A, B, C of a frame carry absolute errors of about
    eta * rms(wave) per pixel in single precision (a few ulp times log2 N).
    Near a zero of A the terms (1 - I_o/I_c) and I_o dI^2 / I_c^2 react
    strongly to that error, so the comparison allows, per pixel,
    |d term / dA| dA + |d term / dB| dB + |d term / dC| dC."""
    pos = data.positions
    A = data.to_detector(oracle.obj_probe_to_psi(obj, probe, pos))
    B = data.to_detector(oracle.obj_probe_to_psi(obj, d_p, pos) + oracle.obj_probe_to_psi(d_o, probe, pos))
    C = data.to_detector(oracle.obj_probe_to_psi(d_o, d_p, pos))

    def err(X):
        return eta * np.sqrt((np.abs(X) ** 2).mean(axis=(-1, -2), keepdims=True))

    eA, eB, eC = err(A), err(B), err(C)
    aA, aB, aC = np.abs(A), np.abs(B), np.abs(C)
    ic = np.maximum((aA ** 2).sum(axis=-3), oracle.ICALC_FLOOR)
    di = 2.0 * (np.conj(A) * B).real.sum(axis=-3)
    d2 = 2.0 * (aB ** 2 + 2.0 * (np.conj(A) * C).real).sum(axis=-3)
    e_ic = (2.0 * aA * eA + eA ** 2).sum(axis=-3)
    e_di = 2.0 * (aB * eA + aA * eB).sum(axis=-3)
    e_d2 = (4.0 * aB * eB + 4.0 * (aC * eA + aA * eC)).sum(axis=-3)
    io = np.maximum(data.iobs, 0.0)
    live = ~data.mask
    b1 = (io / ic ** 2 * e_ic * np.abs(di) + np.abs(1.0 - io / ic) * e_di)[..., live].sum()
    b2 = (io / ic ** 2 * e_ic * np.abs(d2) + np.abs(1.0 - io / ic) * e_d2
          + io * (2.0 * np.abs(di) * e_di / ic ** 2 + 2.0 * di ** 2 * e_ic / ic ** 3))[..., live].sum()
    return np.array([b1, b2])


@pytest.mark.parametrize("cfg,J,which,over", [
    ("ml32fd", 16, "both", ()),
    ("ml256", 60, "both", ()),
    ("ml256", 60, "obj", ()),             # object only (the ML default): two waves, no C term
    ("ml256", 60, "probe", ()),           # probe only
    ("ml256", 301, "obj", ()),            # several line-search batches and a ragged last one
    ("ml32fd", 16, "both", (("K", 2), ("probe", "hg"))),  # two probe modes: the shared-memory kernels
])
def test_ml_line_coeffs_parity(cfg, J, which, over):
    """(L'(0), L''(0)) for each kind of search direction against the oracle,
    within 1e-4 plus the single-precision bound above: a few pixels next to a
    zero of the model wave can hold most of L''(0)."""
    s, obj, probe = warm(cfg, J=J, n_ap=3, **dict(over))
    d_o, d_p = _oracle_direction(s, obj, probe, which)
    pb = gpu_problem(s, with_psi=False, obj=obj, probe=probe)
    got = pb.line_coeffs(to_dev(d_o) if which != "probe" else None,
                         to_dev(d_p) if which != "obj" else None).cpu().numpy()
    data = data_of(s)
    ref = np.array(oracle.ml_line_coeffs(obj, probe, d_o, d_p, data))
    bound = _line_coeffs_fp32_bound(obj, probe, d_o, d_p, data)
    assert bound[0] < 1e-3 * abs(ref[0]), (bound, ref)  # L'(0) is well conditioned
    assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + bound), (got, ref, bound)
    pb.close()


@pytest.mark.parametrize("cfg,J,both", [("ml32fd", 16, False), ("ml256", 60, False), ("ml256", 60, True)])
def test_ml_cg_parity(cfg, J, both):
    """ML CG steps on the GPU against the FP64 oracle CG (object only, as the
    paper's ML defaults, and object + probe)."""
    s, obj, probe = warm(cfg, J=J, n_ap=3)
    pb = gpu_problem(s, with_psi=False, obj=obj, probe=probe)
    llk = pb.ml(1, update_probe=both, restart=True).cpu().numpy()
    o1, p1, l1 = oracle.ml_cg(obj, probe, data_of(s), 1, update_probe=both)
    check_close("obj after 1 CG step", pb.obj.cpu().numpy(), o1, TOL1)
    check_close("probe after 1 CG step", pb.probe.cpu().numpy(), p1, TOL1)
    assert abs(llk[0] - l1[0]) < TOL1 * abs(l1[0])
    more = pb.ml(4, update_probe=both).cpu().numpy()
    o5, p5, l5 = oracle.ml_cg(obj, probe, data_of(s), 5, update_probe=both)
    check_close("obj after 5 CG steps", pb.obj.cpu().numpy(), o5, TOL20)
    check_close("probe after 5 CG steps", pb.probe.cpu().numpy(), p5, TOL20)
    np.testing.assert_allclose(np.concatenate([llk, more]), l5, rtol=TOL20)
    assert all(b < a for a, b in zip(l5[:-1], l5[1:]))
    pb.close()
