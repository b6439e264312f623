"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a direct
DFT sum, hand-derived closed forms (tests/golden/), invariants (Parseval,
idempotence, fixed points), scipy.stats' Poisson log-pmf, torch autograd and
central finite differences.  A plausible mistake (dropped term, wrong sign,
transposed index, wrong conjugate) fails at least one of them; the
``test_planted_*`` cases demonstrate that on mutated copies of the oracle.
"""
import math
import os

import numpy as np
import pytest
import scipy.stats

import oracle
from oracle import ptycho as orc
from synthetic import make_config, make_scan

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def direct_dft2(x):
    """X[ky,kx] = (1/N) sum_{y,x} x[y,x] exp(-2 pi i (ky y + kx x) / N), by explicit sums."""
    N = x.shape[-1]
    y = np.arange(N)
    out = np.zeros((N, N), dtype=np.complex128)
    for ky in range(N):
        for kx in range(N):
            ph = np.exp(-2j * np.pi * (ky * y[:, None] + kx * y[None, :]) / N)
            out[ky, kx] = (x * ph).sum() / N
    return out


def noise_free_intensity(obj, probe, positions):
    """Model intensities computed here (not with the oracle): sum_k |fft2(P_k O_patch)|^2 / N^2."""
    K, N, _ = probe.shape
    out = np.zeros((len(positions), N, N))
    for j, (r, c) in enumerate(positions):
        for k in range(K):
            f = np.fft.fft2(probe[k] * obj[r:r + N, c:c + N]) / N
            out[j] += np.abs(f) ** 2
    return out


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


# ---------------------------------------------------------------- FT / IFT

@pytest.mark.parametrize("N", [8, 12, 16, 32])
def test_ft_matches_direct_dft_sum(N):
    rng = np.random.default_rng(N)
    x = crandn(rng, N, N)
    assert rel(orc.ft(x), direct_dft2(x)) < 1e-13


def _read_golden_dft():
    cases = []
    with open(os.path.join(GOLDEN, "dft2x2.txt")) as f:
        cur = None
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                N = int(tok[1])
                cur = (N, np.zeros((N, N), complex), np.zeros((N, N), complex))
            elif tok[0] == "in":
                cur[1][int(tok[1]), int(tok[2])] = float(tok[3]) + 1j * float(tok[4])
            elif tok[0] == "out":
                cur[2][int(tok[1]), int(tok[2])] = float(tok[3]) + 1j * float(tok[4])
            elif tok[0] == "end":
                cases.append(cur)
    return cases


def test_ft_golden_closed_forms():
    cases = _read_golden_dft()
    assert len(cases) == 2
    for N, x, X in cases:
        np.testing.assert_allclose(orc.ft(x), X, atol=1e-15)
        np.testing.assert_allclose(orc.ift(X), x, atol=1e-15)


def test_ft_parseval_inverse_and_special_inputs():
    rng = np.random.default_rng(1)
    N = 64
    x = crandn(rng, 3, N, N)
    X = orc.ft(x)
    np.testing.assert_allclose((np.abs(X) ** 2).sum(), (np.abs(x) ** 2).sum(), rtol=1e-13)
    assert rel(orc.ift(X), x) < 1e-14
    d = np.zeros((N, N), complex)
    d[0, 0] = 1.0
    np.testing.assert_allclose(orc.ft(d), np.full((N, N), 1.0 / N), atol=1e-16)
    yy, xx = np.mgrid[0:N, 0:N]
    f = np.exp(2j * np.pi * (5 * yy + 11 * xx) / N)
    F = orc.ft(f)
    expect = np.zeros((N, N), complex)
    expect[5, 11] = N
    np.testing.assert_allclose(F, expect, atol=1e-11)


# ---------------------------------------------------------------- ApplyAmplitude

def test_apply_amplitude_modulus_phase_mask_idempotent():
    rng = np.random.default_rng(2)
    K, N = 2, 16
    ph = crandn(rng, 3, K, N, N)
    io = rng.uniform(0, 50, size=(3, N, N))
    io[0, 0, 0] = -3.0  # negative observation is clamped to 0
    mask = rng.uniform(size=(N, N)) < 0.2
    out = orc.apply_amplitude(ph, io, mask)
    ic_out = (np.abs(out) ** 2).sum(1)
    um = ~mask
    np.testing.assert_allclose(ic_out[:, um], np.maximum(io, 0)[:, um], rtol=1e-12, atol=1e-12)
    # common factor: the ratio out/in is the same real positive number for all modes
    ratio = out / ph
    np.testing.assert_allclose(ratio[:, 0], ratio[:, 1], rtol=1e-12)
    assert np.all(np.abs(ratio.imag) < 1e-12) and np.all(ratio.real >= 0)
    np.testing.assert_array_equal(out[:, :, mask], ph[:, :, mask])
    again = orc.apply_amplitude(out, io, mask)
    assert rel(again, out) < 1e-14


def test_apply_amplitude_zero_stays_zero():
    N = 8
    ph = np.zeros((1, 1, N, N), complex)
    io = np.ones((1, N, N))
    out = orc.apply_amplitude(ph, io, np.zeros((N, N), bool))
    assert np.all(out == 0) and np.all(np.isfinite(out))


# ---------------------------------------------------------------- LLK

def test_llk_golden_values():
    rows = np.loadtxt(os.path.join(GOLDEN, "llk_poisson.txt"), comments="#")
    ic, io, t = rows[:, 0], rows[:, 1], rows[:, 2]
    got = orc.llk_terms(ic, io, np.zeros_like(ic, dtype=bool))
    np.testing.assert_allclose(got, t, rtol=1e-15, atol=1e-15)


def test_llk_is_poisson_log_likelihood_ratio():
    """Deviance/2 = log Pois(Io | Io) - log Pois(Io | Ic) (scipy.stats definition)."""
    rng = np.random.default_rng(3)
    N = 16
    ic = rng.uniform(0.5, 40, size=(2, N, N))
    io = rng.poisson(ic).astype(float)
    mask = rng.uniform(size=(N, N)) < 0.1
    expect = (scipy.stats.poisson.logpmf(io, np.maximum(io, 1e-300)) - scipy.stats.poisson.logpmf(io, ic))
    expect = np.where(io == 0, ic, expect)  # logpmf(0 | 0) is 0 and logpmf(0 | Ic) = -Ic
    expect[:, mask] = 0
    np.testing.assert_allclose(orc.llk_terms(ic, io, mask), expect, rtol=1e-10, atol=1e-10)
    assert orc.llk_poisson(ic, io, mask) >= 0
    assert abs(orc.llk_poisson(io, io, mask)) < 1e-12


def test_llk_constant_arrays_closed_form():
    N = 8
    a, b = 3.5, 2.0
    got = orc.llk_poisson(np.full((1, N, N), a), np.full((1, N, N), b), np.zeros((N, N), bool))
    assert abs(got - N * N * (a - b + b * math.log(b / a))) < 1e-12


# ---------------------------------------------------------------- Psi2ObjProbe

def test_overlap_update_single_frame_closed_form():
    """One frame, Psi = P X, alpha -> 0: the object becomes X on the patch, unchanged elsewhere."""
    rng = np.random.default_rng(4)
    N, Ho, Wo = 16, 40, 48
    obj = crandn(rng, Ho, Wo)
    probe = crandn(rng, 1, N, N)
    X = crandn(rng, N, N)
    pos = np.array([[7, 21]])
    psi = (probe * X[None])[None]
    sums = orc.psi_to_obj_probe_sums(psi, obj, probe, pos, obj.shape)
    new_obj, new_probe = orc.normalise(obj, probe, sums, alpha_obj=1e-16, alpha_probe=1e-16,
                                       update_probe=False)
    np.testing.assert_allclose(new_obj[7:23, 21:37], X, rtol=1e-9)
    outside = np.ones((Ho, Wo), bool)
    outside[7:23, 21:37] = False
    np.testing.assert_allclose(new_obj[outside], obj[outside], rtol=1e-12)
    np.testing.assert_array_equal(new_probe, probe)


def test_probe_update_single_frame_closed_form():
    """One frame, Psi = Q O_patch, alpha -> 0: the probe becomes Q."""
    rng = np.random.default_rng(5)
    N = 12
    obj = crandn(rng, 30, 30)
    probe = crandn(rng, 1, N, N)
    Q = crandn(rng, 1, N, N)
    pos = np.array([[3, 9]])
    psi = (Q * obj[3:15, 9:21][None])[None]
    sums = orc.psi_to_obj_probe_sums(psi, obj, probe, pos, obj.shape)
    _, new_probe = orc.normalise(obj, probe, sums, alpha_obj=1e-16, alpha_probe=1e-16, update_obj=False)
    np.testing.assert_allclose(new_probe, Q, rtol=1e-9)


def test_split_positions_partial_sums_add_up():
    """Data-parallel split: per-subset numerators/denominators sum to the unsplit ones."""
    rng = np.random.default_rng(6)
    N, K = 16, 2
    obj = crandn(rng, 64, 64)
    probe = crandn(rng, K, N, N)
    pos = rng.integers(0, 64 - N + 1, size=(20, 2))
    psi = crandn(rng, 20, K, N, N)
    full = orc.psi_to_obj_probe_sums(psi, obj, probe, pos, obj.shape)
    parts = [orc.psi_to_obj_probe_sums(psi[s], obj, probe, pos[s], obj.shape)
             for s in (slice(0, 7), slice(7, 13), slice(13, 20))]
    for i in range(4):
        np.testing.assert_allclose(sum(p[i] for p in parts), full[i], rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- fixed points

def _exact_problem(seed=7, K=1, N=32, J=12, Ho=80, Wo=72):
    rng = np.random.default_rng(seed)
    obj = np.exp(0.3 * crandn(rng, Ho, Wo))
    probe = crandn(rng, K, N, N)
    pos = np.stack([rng.integers(0, Ho - N + 1, J), rng.integers(0, Wo - N + 1, J)], 1)
    iobs = noise_free_intensity(obj, probe, pos)
    mask = np.zeros((N, N), bool)
    mask[3, :] = True
    return obj, probe, pos, orc.Data.make(iobs, pos, mask)


@pytest.mark.parametrize("K", [1, 2])
def test_fixed_point_ap_and_dm(K):
    obj, probe, pos, data = _exact_problem(K=K)
    o1, p1, l1 = orc.ap_cycle(obj, probe, data)
    assert rel(o1, obj) < 1e-12 and rel(p1, probe) < 1e-12
    assert abs(l1) < 1e-12 * data.iobs.sum()
    psi0 = orc.obj_probe_to_psi(obj, probe, pos)
    o2, p2, psi2, l2 = orc.dm_cycle(obj, probe, psi0, data)
    assert rel(o2, obj) < 1e-12 and rel(p2, probe) < 1e-12 and rel(psi2, psi0) < 1e-12
    assert abs(l2) < 1e-12 * data.iobs.sum()
    assert abs(orc.llk(obj, probe, data)) < 1e-12 * data.iobs.sum()


def test_fixed_point_on_float32_stored_data():
    """The synthetic generator's noise-free intensities (stored as float32) are a fixed point
    of the oracle up to float32 storage rounding."""
    s = make_config("ap64", noise=False)
    data = orc.Data.make(s.iobs, s.positions, s.mask)
    l = orc.llk(s.obj_true, s.probe_true, data)
    assert 0 <= l < 1e-10 * data.iobs.sum()
    o1, p1, _ = orc.ap_cycle(s.obj_true, s.probe_true, data)
    assert rel(p1, s.probe_true) < 1e-6


# ---------------------------------------------------------------- DM special case

def test_dm_equals_ap_single_frame_object_only():
    """J = 1, object-only update, |P| > 0 on the whole object, alpha = 0: the overlap
    projection is the identity on Psi, so every DM cycle equals an AP (= ER) cycle."""
    rng = np.random.default_rng(8)
    N = 16
    probe = crandn(rng, 1, N, N)
    obj_true = np.exp(0.5 * crandn(rng, N, N))
    pos = np.array([[0, 0]])
    iobs = rng.poisson(noise_free_intensity(obj_true, probe, pos) * 50).astype(float) / 50.0
    data = orc.Data.make(iobs, pos)
    o_ap = np.ones((N, N), complex)
    o_dm = np.ones((N, N), complex)
    psi = None
    kw = dict(alpha_obj=0.0, update_probe=False)
    for i in range(4):
        o_ap, _, _ = orc.ap_cycle(o_ap, probe, data, **kw)
        o_dm, _, psi, _ = orc.dm_cycle(o_dm, probe, psi, data, init_psi=(i == 0), **kw)
        assert rel(o_dm, o_ap) < 1e-12
    # and both equal the error-reduction form P_S F^-1 P_m F (support = whole frame)
    o_er = np.ones((N, N), complex)
    for i in range(4):
        w = probe[0] * o_er
        W = np.fft.fft2(w) / N
        W = W * np.sqrt(iobs[0]) / np.maximum(np.abs(W), 1e-20)
        o_er = (np.fft.ifft2(W) * N) / probe[0]
    assert rel(o_ap, o_er) < 1e-11


# ---------------------------------------------------------------- modes

def test_zero_second_mode_equals_single_mode():
    s = make_config("ml32fd")
    data = orc.Data.make(s.iobs, s.positions, s.mask)
    p1 = s.probe0.astype(np.complex128)
    p2 = np.concatenate([p1, np.zeros_like(p1)])
    o = s.obj0.astype(np.complex128) * 0.9
    a = orc.ap_cycle(o, p1, data)
    b = orc.ap_cycle(o, p2, data, update_probe=False)
    c = orc.ap_cycle(o, p1, data, update_probe=False)
    assert rel(b[0], c[0]) < 1e-14 and abs(b[2] - a[2]) < 1e-9 * abs(a[2])
    g1 = orc.ml_grad(o, p1, data)
    g2 = orc.ml_grad(o, p2, data)
    assert rel(g2[1], g1[1]) < 1e-13 and abs(g2[0] - g1[0]) < 1e-9 * abs(g1[0])
    assert rel(g2[2][0], g1[2][0]) < 1e-13


def test_modes_add_incoherently():
    rng = np.random.default_rng(9)
    N = 16
    obj = crandn(rng, 20, 20)
    p = crandn(rng, 1, N, N)
    probe = np.concatenate([p, 1j * p, 2 * p])
    phi_hat = orc.ft(orc.obj_probe_to_psi(obj, probe, np.array([[2, 3]])))
    ic = orc.calc_intensity(phi_hat)
    single = np.abs(np.fft.fft2(p[0] * obj[2:18, 3:19]) / N) ** 2
    np.testing.assert_allclose(ic[0], 6.0 * single, rtol=1e-12)


# ---------------------------------------------------------------- ML gradient

def richardson_fd(f, h):
    """Central difference with one Richardson step (error O(h^4)); the LLK is very curved where
    I_c is tiny, so a plain central difference converges only as h^2."""
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


def _fd_problem():
    s = make_config("ml32fd")
    data = orc.Data.make(s.iobs, s.positions, s.mask)
    rng = np.random.default_rng(10)
    obj = s.obj0.astype(np.complex128) * (1 + 0.05 * crandn(rng, s.Ho, s.Wo))
    probe = s.probe0.astype(np.complex128)
    return s, data, obj, probe


def test_ml_grad_directional_finite_differences():
    s, data, obj, probe = _fd_problem()
    L, go, gp = orc.ml_grad(obj, probe, data)
    assert abs(L - orc.llk(obj, probe, data)) < 1e-9 * abs(L)
    rng = np.random.default_rng(11)
    for trial in range(3):
        do = crandn(rng, *obj.shape)
        dp = crandn(rng, *probe.shape)
        ho = 1e-6 * np.sqrt(np.mean(np.abs(obj) ** 2))
        hp = 1e-6 * np.sqrt(np.mean(np.abs(probe) ** 2))
        fd_o = richardson_fd(lambda t: orc.llk(obj + t * do, probe, data), ho)
        fd_p = richardson_fd(lambda t: orc.llk(obj, probe + t * dp, data), hp)
        an_o = float(np.real(np.vdot(go, do)))
        an_p = float(np.real(np.vdot(gp, dp)))
        assert abs(fd_o - an_o) < 1e-7 * max(abs(an_o), 1.0), (fd_o, an_o)
        assert abs(fd_p - an_p) < 1e-7 * max(abs(an_p), 1.0), (fd_p, an_p)


def test_ml_grad_per_pixel_finite_differences():
    s, data, obj, probe = _fd_problem()
    _, go, gp = orc.ml_grad(obj, probe, data)
    h = 1e-4  # a single pixel moves L (~1e6) little: larger steps keep rounding below 1e-8
    for (y, x) in [(20, 30), (33, 33), (40, 25)]:
        for unit in (1.0, 1j):
            d = np.zeros_like(obj)
            d[y, x] = unit
            fd = richardson_fd(lambda t: orc.llk(obj + t * d, probe, data), h)
            an = go[y, x].real if unit == 1.0 else go[y, x].imag
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (y, x, unit, fd, an)
    for (y, x) in [(16, 16), (10, 20)]:
        for unit in (1.0, 1j):
            d = np.zeros_like(probe)
            d[0, y, x] = unit
            fd = richardson_fd(lambda t: orc.llk(obj, probe + t * d, data), h)
            an = gp[0, y, x].real if unit == 1.0 else gp[0, y, x].imag
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (y, x, unit, fd, an)


def test_ml_grad_matches_torch_autograd():
    """Independent adjoint: torch autograd through torch.fft (complex128, CPU)."""
    torch = pytest.importorskip("torch")
    s, data, obj, probe = _fd_problem()
    L, go, gp = orc.ml_grad(obj, probe, data)
    to = torch.tensor(obj, requires_grad=True)
    tp = torch.tensor(probe, requires_grad=True)
    io = torch.tensor(data.iobs)
    um = torch.tensor(~data.mask)
    N = probe.shape[-1]
    total = 0
    for j, (r, c) in enumerate(data.positions):
        w = tp * to[r:r + N, c:c + N][None]
        f = torch.fft.fft2(w, norm="ortho")
        ic = (f.real ** 2 + f.imag ** 2).sum(0)
        total = total + ((ic - io[j] * torch.log(ic)) * um).sum()
    total.backward()
    assert rel(to.grad.numpy(), go) < 1e-10
    assert rel(tp.grad.numpy(), gp) < 1e-10


def test_ml_grad_zero_at_noise_free_truth():
    obj, probe, pos, data = _exact_problem(seed=12)
    _, go, gp = orc.ml_grad(obj, probe, data)
    scale = np.sqrt(data.iobs.sum())
    assert np.abs(go).max() < 1e-10 * scale and np.abs(gp).max() < 1e-10 * scale


# ---------------------------------------------------------------- behaviour over cycles

def test_ap_llk_decreases_on_ap64():
    s = make_config("ap64")
    data = orc.Data.make(s.iobs, s.positions, s.mask)
    _, _, _, llks = orc.cycles("AP", s.obj0, s.probe0, data, 8)
    assert llks[-1] < llks[0]
    assert np.mean(np.diff(llks)) < 0


def test_dm_sampled_frame_update_matches_full_cycle():
    s = make_config("ap64")
    data = orc.Data.make(s.iobs, s.positions, s.mask)
    obj, probe = s.obj0.astype(complex), s.probe0.astype(complex)
    _, _, psi, _ = orc.dm_cycle(obj, probe, None, data, init_psi=True)
    for j in (0, 37, 99):
        pj, _ = orc.dm_frame_update(obj, probe, None, data.iobs[j], data.positions[j], data.mask, init_psi=True)
        assert rel(pj, psi[j]) < 1e-14


# ---------------------------------------------------------------- planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Mutations of the oracle (a dropped conjugate, a transposed patch) break the pins
    above; the DM combination's mutations are in test_oracle_pins_dm_cg.py."""
    obj, probe, pos, data = _exact_problem(seed=13)

    def bad_sums(psi, probe_, positions, shape_obj):
        K, N, _ = probe_.shape
        n_o = np.zeros(shape_obj, complex); d_o = np.zeros(shape_obj)
        for j, (r, c) in enumerate(positions):
            n_o[r:r + N, c:c + N] += (probe_ * psi[j]).sum(0)  # conjugate dropped
            d_o[r:r + N, c:c + N] += (np.abs(probe_) ** 2).sum(0)
        return n_o, d_o

    with monkeypatch.context() as m:
        m.setattr(orc, "psi_to_obj_sums", bad_sums)
        o1, _, _ = orc.ap_cycle(obj, probe, data)
        assert rel(o1, obj) > 1e-3

    def transposed_patch(obj_, probe_, positions):
        K, N, _ = probe_.shape
        out = np.empty((len(positions), K, N, N), complex)
        for j, (r, c) in enumerate(positions):
            out[j] = probe_ * obj_[r:r + N, c:c + N].T[None]
        return out

    with monkeypatch.context() as m:
        m.setattr(orc, "obj_probe_to_psi", transposed_patch)
        assert orc.llk(obj, probe, data) > 1e-3 * data.iobs.sum()


# ---------------------------------------------------------------- overlap update order

def test_dm_stays_bounded_over_100_cycles():
    """Psi2ObjProbe updates the probe from the current object, then the object from
    the new probe: DM stays bounded on the 64x64 scan (100 cycles)."""
    s = make_config("ap64")
    data = orc.Data.make(s.iobs, s.positions, s.mask)
    o, p, _ = orc.ap_cycle(s.obj0, s.probe0, data)
    _, _, psi, _ = orc.cycles("DM", o, p, data, 100)
    assert np.abs(psi).max() < 1e2


def test_simultaneous_update_would_diverge_under_dm():
    """Why the update alternates: with both factors updated from the same (O, P), a
    scale error of Psi enters O and P alike, the product takes it twice, and DM
    grows geometrically (the same 64x64 scan, 20 cycles)."""
    s = make_config("ap64")
    data = orc.Data.make(s.iobs, s.positions, s.mask)
    o, p, _ = orc.ap_cycle(s.obj0, s.probe0, data)
    psi = None
    for c in range(20):
        phi = orc.obj_probe_to_psi(o, p, data.positions)
        if psi is None:
            psi = phi.copy()
        x_hat = orc.ft(2 * phi - psi)
        psi = psi + orc.ift(orc.apply_amplitude(x_hat, data.iobs, data.mask)) - phi
        o, p = orc.normalise(o, p, orc.psi_to_obj_probe_sums(psi, o, p, data.positions, o.shape))
    assert np.abs(psi).max() > 1e4


def test_overlap_update_is_probe_then_object():
    rng = np.random.default_rng(15)
    N = 16
    obj = crandn(rng, 40, 40)
    probe = crandn(rng, 2, N, N)
    pos = rng.integers(0, 40 - N + 1, size=(7, 2))
    psi = crandn(rng, 7, 2, N, N)
    o1, p1 = orc.overlap_update(obj, probe, psi, pos)
    n_p, d_p = orc.psi_to_probe_sums(psi, obj, pos)
    p_exp = (n_p + 1e-2 * d_p.max() * probe) / (d_p + 1e-2 * d_p.max())[None]
    n_o, d_o = orc.psi_to_obj_sums(psi, p_exp, pos, obj.shape)
    o_exp = np.where(d_o + 1e-2 * d_o.max() > 0, (n_o + 1e-2 * d_o.max() * obj) / (d_o + 1e-2 * d_o.max()), obj)
    assert rel(p1, p_exp) < 1e-14 and rel(o1, o_exp) < 1e-14


# ---------------------------------------------------------------- ML conjugate gradient

def test_ml_line_coeffs_match_gradient_and_finite_differences():
    """L'(0) of the line expansion equals the directional derivative Re<G, D> of the
    gradient; L''(0) matches a central second difference of L along D."""
    s, data, obj, probe = _fd_problem()
    obj, probe, _ = orc.ap_cycle(obj, probe, data)
    obj, probe, _ = orc.ap_cycle(obj, probe, data)
    rng = np.random.default_rng(31)
    do = 0.01 * crandn(rng, *obj.shape)
    dp = 0.01 * crandn(rng, *probe.shape)
    l1, l2 = orc.ml_line_coeffs(obj, probe, do, dp, data)
    _, go, gp = orc.ml_grad(obj, probe, data)
    assert abs(l1 - (orc._dot(go, do) + orc._dot(gp, dp))) < 1e-9 * abs(l1)
    f = lambda a: orc.llk(obj + a * do, probe + a * dp, data)
    h = 1e-3
    fd2 = (f(h) - 2 * f(0.0) + f(-h)) / h ** 2
    assert abs(fd2 - l2) < 1e-4 * abs(l2), (fd2, l2)


def test_ml_cg_decreases_llk_and_takes_the_model_step():
    """CG lowers the LLK every step; its first step is steepest descent with the
    step that minimises the second-order model a L'(0) + a^2 L''(0) / 2 (whose
    derivatives are pinned above).  The Poisson LLK is far from quadratic where
    I_c is small, so the model step undershoots the line minimum but descends."""
    s, data, obj, probe = _fd_problem()
    o, p, llks = orc.ml_cg(obj, probe, data, 6)
    assert all(b < a for a, b in zip(llks[:-1], llks[1:]))
    _, go, gp = orc.ml_grad(obj, probe, data)
    l1, l2 = orc.ml_line_coeffs(obj, probe, -go, np.zeros_like(gp), data)
    a = -l1 / l2
    assert a > 0 and orc.llk(obj - a * go, probe, data) < orc.llk(obj, probe, data)
    o1, p1, _ = orc.ml_cg(obj, probe, data, 1)
    assert rel(o1, obj - a * go) < 1e-12 and rel(p1, probe) == 0.0
    o2, p2, l2s = orc.ml_cg(obj, probe, data, 3, update_obj=True, update_probe=True)
    assert l2s[-1] < l2s[0]


# ---------------------------------------------------------------- near field

def test_near_field_propagates_a_gaussian_beam_like_fresnel():
    """A Gaussian exp(-r^2 / (2 s^2)) after a paraxial propagation over lambda z is
    exp(-r^2 / (2 s^2 (1 + i b))) / (1 + i b), b = lambda z / (2 pi s^2) (s in
    pixels, lambda z = c pixel^2): the closed form pins the sign and the scale of
    the transfer function.  The beam stays far from the frame edges, so the
    periodic discrete propagation matches the continuous one."""
    N, sig = 128, 4.0
    y = np.arange(N) - N // 2
    r2 = y[:, None] ** 2 + y[None, :] ** 2
    u0 = np.exp(-r2 / (2 * sig ** 2))
    for c in (10.0, 60.0, 150.0):
        b = c / (2 * np.pi * sig ** 2)
        expect = np.exp(-r2 / (2 * sig ** 2 * (1 + 1j * b))) / (1 + 1j * b)
        got = orc.propagate_near_field(u0, c, +1)
        assert rel(got, expect) < 1e-8, c
        # back propagation: the conjugate closed form
        assert rel(orc.propagate_near_field(u0, c, -1), np.conj(expect)) < 1e-8, c


def test_near_field_propagation_is_unitary_and_reversible():
    rng = np.random.default_rng(40)
    x = crandn(rng, 3, 48, 48)
    for c in (0.0, 7.5, 300.0):
        y = orc.propagate_near_field(x, c, +1)
        assert abs(np.linalg.norm(y) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
        assert rel(orc.propagate_near_field(y, c, -1), x) < 1e-13
    assert rel(orc.propagate_near_field(x, 0.0, +1), x) < 1e-14
    # direct transfer values: h = exp(-i pi c (ky^2 + kx^2) / N^2), k signed
    h = orc.near_field_transfer(8, 3.0)
    assert abs(h[0, 0] - 1) < 1e-15
    assert abs(h[1, 2] - np.exp(-1j * np.pi * 3.0 * 5 / 64)) < 1e-15
    assert abs(h[7, 6] - np.exp(-1j * np.pi * 3.0 * (1 + 4) / 64)) < 1e-15
    assert abs(h[4, 0] - np.exp(-1j * np.pi * 3.0 * 16 / 64)) < 1e-15


def test_near_field_at_zero_distance_projects_in_real_space():
    """With lambda z = 0 the detector sees the exit wave itself: one near-field AP
    step replaces |Phi| by sqrt(I) pixel by pixel (checked here without any
    transform), masked pixels unchanged."""
    rng = np.random.default_rng(41)
    N = 16
    obj = crandn(rng, 30, 30)
    probe = crandn(rng, 1, N, N)
    pos = np.array([[0, 0], [5, 9], [14, 3]])
    iobs = rng.uniform(0.5, 4.0, size=(3, N, N))
    mask = np.zeros((N, N), bool)
    mask[2, 5] = True
    data = orc.Data.make(iobs, pos, mask, nearfield=1e-300)
    phi = np.stack([probe[0] * obj[r:r + N, c:c + N] for r, c in pos])
    expect = np.where(mask, phi, np.sqrt(iobs) * np.exp(1j * np.angle(phi)))
    got = data.from_detector(orc.apply_amplitude(data.to_detector(phi[:, None]), data.iobs, data.mask))[:, 0]
    assert rel(got, expect) < 1e-12


def _near_field_problem(noise=False):
    s = make_scan("nf32", N=32, J=12, Ho=80, Wo=80, seed=43, photons=1e6, step=8.0,
                  probe_radius=11.0, phase_coef=0.0, diffuser_phase=1.5, mask_fraction=0.02,
                  nearfield=12.0, noise=noise)
    return s, orc.Data.make(s.iobs, s.positions, s.mask, nearfield=s.nearfield)


def test_near_field_fixed_point_ap_and_dm():
    """Noise-free near-field intensities of the true object and probe: one AP and
    one DM cycle leave both unchanged and the LLK is zero (up to the float32
    storage of the intensities)."""
    s, data = _near_field_problem()
    o, p = s.obj_true, s.probe_true
    assert 0 <= orc.llk(o, p, data) < 1e-9 * data.iobs.sum()
    o1, p1, l1 = orc.ap_cycle(o, p, data)
    assert rel(p1, p) < 1e-6 and rel(o1[orc.object_denominator(p, s.positions, o.shape) > 0],
                                      o[orc.object_denominator(p, s.positions, o.shape) > 0]) < 1e-6
    psi0 = orc.obj_probe_to_psi(o, p, s.positions)
    _, p2, psi2, _ = orc.dm_cycle(o, p, psi0, data)
    assert rel(p2, p) < 1e-6 and rel(psi2, psi0) < 1e-6
    # and the same scan read as far field is not a fixed point
    far = orc.Data.make(s.iobs, s.positions, s.mask)
    assert orc.llk(o, p, far) > 1e-3 * data.iobs.sum()


def test_near_field_ml_grad_directional_finite_differences():
    s, data = _near_field_problem(noise=True)
    rng = np.random.default_rng(44)
    obj = s.obj_true * (1 + 0.05 * crandn(rng, s.Ho, s.Wo))
    probe = s.probe_true * (1 + 0.05 * crandn(rng, *s.probe_true.shape))
    L, go, gp = orc.ml_grad(obj, probe, data)
    assert abs(L - orc.llk(obj, probe, data)) < 1e-9 * abs(L)
    do = crandn(rng, *obj.shape)
    dp = crandn(rng, *probe.shape)
    ho = 1e-6 * np.sqrt(np.mean(np.abs(obj) ** 2))
    hp = 1e-6 * np.sqrt(np.mean(np.abs(probe) ** 2))
    fd_o = richardson_fd(lambda t: orc.llk(obj + t * do, probe, data), ho)
    fd_p = richardson_fd(lambda t: orc.llk(obj, probe + t * dp, data), hp)
    assert abs(fd_o - float(np.real(np.vdot(go, do)))) < 1e-7 * max(abs(fd_o), 1.0)
    assert abs(fd_p - float(np.real(np.vdot(gp, dp)))) < 1e-7 * max(abs(fd_p), 1.0)


# ---------------------------------------------------------------- incoherent background

def _background_problem(bg_level=3.0, noise=False):
    """Far-field data whose intensities carry a known smooth background B_true
    (model: |FT(P O)|^2 + B_true, computed here with numpy, not the oracle)."""
    s = make_scan("bg32", N=32, J=16, Ho=64, Wo=64, seed=61, photons=1e5, step=6.0,
                  probe_radius=6.0, mask_fraction=0.0, noise=False)
    yy, xx = np.mgrid[0:32, 0:32]
    b_true = bg_level * (1.0 + 0.5 * np.cos(2 * np.pi * yy / 32) * np.cos(2 * np.pi * xx / 32))
    iobs = noise_free_intensity(s.obj_true, s.probe_true, s.positions) + b_true[None]
    if noise:
        iobs = np.random.default_rng(62).poisson(iobs).astype(np.float64)
    return s, iobs, b_true


def test_background_llk_is_poisson_with_the_added_rate():
    """With a background the LLK terms are the Poisson deviance at rate I_c + B
    (checked against scipy.stats)."""
    s, iobs, b = _background_problem(noise=True)
    data = orc.Data.make(iobs, s.positions, None, background=0.7 * b)
    rng = np.random.default_rng(63)
    obj = s.obj_true * (1 + 0.03 * crandn(rng, s.Ho, s.Wo))
    ic = noise_free_intensity(obj, s.probe_true, s.positions) + 0.7 * b[None]
    ref = float(-(scipy.stats.poisson.logpmf(iobs, ic) - scipy.stats.poisson.logpmf(iobs, iobs)).sum())
    assert abs(orc.llk(obj, s.probe_true, data) - ref) < 1e-9 * abs(ref)


def test_background_fixed_point_and_zero_llk():
    """Noise-free data with the true background: the background AP cycle leaves
    O, P and B unchanged and the LLK is zero."""
    s, iobs, b = _background_problem()
    data = orc.Data.make(iobs, s.positions, None)
    o1, p1, b1, l1 = orc.ap_cycle_background(s.obj_true, s.probe_true, b, data)
    assert abs(l1) < 1e-10 * iobs.sum()
    assert rel(b1, b) < 1e-12 and rel(p1, s.probe_true) < 1e-10
    ill = orc.object_denominator(s.probe_true, s.positions, s.obj_true.shape) > 0
    assert rel(o1[ill], s.obj_true[ill]) < 1e-10


def test_background_update_is_an_em_step_towards_the_true_background():
    """With O and P held at the truth the background update is the EM step of
    a Poisson mixture (component B in I_c + B): from a guess twice too high or
    four times too low the LLK never increases, and where the background
    dominates the model (I_c < B_true) B reaches B_true; everywhere it moves
    towards it."""
    s, iobs, b = _background_problem(bg_level=40.0)
    data = orc.Data.make(iobs, s.positions, None)
    ic_max = noise_free_intensity(s.obj_true, s.probe_true, s.positions).max(axis=0)
    dark = ic_max < b
    assert dark.sum() > 50
    for b0 in (2.0 * b, 0.25 * b):
        bg, llks = b0, []
        for _ in range(150):
            _, _, bg, l = orc.ap_cycle_background(s.obj_true, s.probe_true, bg, data,
                                                  update_obj=False, update_probe=False)
            llks.append(l)
        assert all(b2 <= b1 * (1 + 1e-12) for b1, b2 in zip(llks[:-1], llks[1:]))
        assert rel(bg[dark], b[dark]) < 1e-3, rel(bg[dark], b[dark])
        assert rel(bg, b) < 0.5 * rel(b0, b)


def test_background_gradient_finite_differences():
    s, iobs, b = _background_problem(noise=True)
    data = orc.Data.make(iobs, s.positions, None, background=b)
    rng = np.random.default_rng(64)
    obj = s.obj_true * (1 + 0.05 * crandn(rng, s.Ho, s.Wo))
    probe = s.probe_true.copy()
    L, go, gp = orc.ml_grad(obj, probe, data)
    do = crandn(rng, *obj.shape)
    ho = 1e-6 * np.sqrt(np.mean(np.abs(obj) ** 2))
    fd = richardson_fd(lambda t: orc.llk(obj + t * do, probe, data), ho)
    assert abs(fd - float(np.real(np.vdot(go, do)))) < 1e-7 * max(abs(fd), 1.0)


# ---------------------------------------------------------------- position refinement

def _fourier_shift(x, dy, dx):
    """x(r + (dy, dx)) for a periodic band-limited x, by a phase ramp (numpy FFT)."""
    H, W = x.shape
    ky = np.fft.fftfreq(H)[:, None]
    kx = np.fft.fftfreq(W)[None, :]
    return np.fft.ifft2(np.fft.fft2(x) * np.exp(2j * np.pi * (ky * dy + kx * dx)))


def _smooth_object(seed, H=96, W=96, sigma=4.0):
    rng = np.random.default_rng(seed)
    from scipy.ndimage import gaussian_filter
    a = gaussian_filter(rng.standard_normal((H, W)), sigma, mode="wrap")
    p = gaussian_filter(rng.standard_normal((H, W)), sigma, mode="wrap")
    return (1.0 + 0.3 * a / np.abs(a).max()) * np.exp(1j * 1.5 * p / np.abs(p).max())


def test_position_shift_recovers_a_known_subpixel_shift():
    """Psi_j built from the object shifted by a known sub-pixel amount (exact
    Fourier shift, computed here with numpy): the estimated shift matches it to
    first order, scales linearly with it, and is zero for Psi = Phi."""
    obj = _smooth_object(80)
    N = 24
    yy, xx = np.mgrid[0:N, 0:N] - N / 2
    probe = np.exp(-(yy ** 2 + xx ** 2) / (2 * 6.0 ** 2))[None].astype(np.complex128)
    pos = np.array([[20, 30], [40, 12], [55, 50], [10, 60]])
    deltas = np.array([[0.12, -0.08], [-0.1, 0.05], [0.06, 0.11], [-0.05, -0.12]])
    psi = np.stack([probe * _fourier_shift(obj, dy, dx)[r:r + N, c:c + N][None]
                    for (r, c), (dy, dx) in zip(pos, deltas)])
    d = orc.position_shifts(obj, probe, psi, pos, filter_ratio=0.0)
    assert np.abs(d - deltas).max() < 0.1 * np.abs(deltas).max(), (d, deltas)
    d2 = orc.position_shifts(obj, probe, np.stack([probe * _fourier_shift(obj, 2 * dy, 2 * dx)[r:r + N, c:c + N][None]
                                                   for (r, c), (dy, dx) in zip(pos, deltas)]), pos, filter_ratio=0.0)
    assert np.abs(d2 - 2 * d).max() < 0.1 * np.abs(d).max()
    phi = orc.obj_probe_to_psi(obj, probe, pos)
    assert np.abs(orc.position_shifts(obj, probe, phi, pos)).max() == 0.0


def test_position_shift_filter_keeps_flat_regions_in_place():
    """A frame over a flat part of the object (no gradient) is not shifted and
    gives no NaN; frames over structure still are."""
    obj = _smooth_object(81)
    obj[:, :40] = 1.0  # flat left part
    N = 24
    probe = np.ones((1, N, N), dtype=np.complex128)
    pos = np.array([[10, 5], [10, 60], [50, 65]])
    psi = np.stack([probe * _fourier_shift(obj, 0.1, 0.1)[r:r + N, c:c + N][None] for r, c in pos])
    d = orc.position_shifts(obj, probe, psi, pos, filter_ratio=0.1)
    assert np.all(np.isfinite(d)) and np.all(d[0] == 0.0)
    assert np.all(np.abs(d[1:]) > 0.02)


def test_object_gradient_central_differences():
    y = np.arange(10)[:, None] * np.ones((1, 8))
    x = np.ones((10, 1)) * np.arange(8)[None, :]
    o = (2.0 * y + 3j * x ** 2).astype(np.complex128)
    gy, gx = orc.object_gradient(o)
    assert np.allclose(gy, 2.0)
    assert np.allclose(gx[:, 1:-1], 3j * 2 * x[:, 1:-1]) and np.allclose(gx[:, 0], 3j) and np.allclose(gx[:, -1], 3j * 13)
