"""Pins of the oracle's DM combination away from the fixed point, and of the
Polak-Ribiere direction of its ML conjugate gradient (CPU only).

DM (paper Section 4: difference map after Elser, in its ptychographic form):
one step is Psi' = Psi + P_F(2 Phi - Psi) - Phi.  Two special cases fix every
term of it at a point where Psi != Phi, from the definition alone:

* every detector pixel masked: the Fourier projection P_F leaves masked pixels
  free, so it is the identity and Psi' = Psi + (2 Phi - Psi) - Phi = Phi;
* I_obs = 0 on every pixel, no mask: P_F maps every wave to 0, so
  Psi' = Psi - Phi, and the cycle's Poisson LLK (deviance, = I_c where
  I_obs = 0) is sum |FT(2 Phi - Psi)|^2 = ||2 Phi - Psi||^2 by Parseval.

ML (paper Section 4, after Thibault & Guizar-Sicairos): the search direction of
step n + 1 is -G_{n+1} + beta D_n with the Polak-Ribiere
beta = max(0, <G_{n+1}, G_{n+1} - G_n> / <G_n, G_n>); the gradients come from
``ml_grad``, which ``test_oracle_pins.py`` pins by finite differences and by
torch autograd.

Each pin is also run against mutations of the oracle's own source (a wrong
sign, a dropped term, the Fletcher-Reeves numerator) and must reject every one.
"""
import inspect
import textwrap

import numpy as np
import pytest

from oracle import ptycho as orc
from synthetic import make_config


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def exit_waves_here(obj, probe, pos):
    """Phi[j, k] = P_k(x) O(r_j + x), by explicit loops (not the oracle's routine)."""
    K, N, _ = probe.shape
    out = np.zeros((len(pos), K, N, N), complex)
    for j, (r, c) in enumerate(pos):
        for k in range(K):
            for y in range(N):
                for x in range(N):
                    out[j, k, y, x] = probe[k, y, x] * obj[r + y, c + x]
    return out


def mutant(func, old, new):
    """``func`` recompiled from its own source with ``old`` (which must occur
    once) replaced by ``new``, in a copy of the oracle module's namespace."""
    src = textwrap.dedent(inspect.getsource(func))
    assert src.count(old) == 1, old
    ns = dict(func.__globals__)
    exec(compile(src.replace(old, new), inspect.getsourcefile(func), "exec"), ns)
    return ns[func.__name__]


# ---------------------------------------------------------------- DM at Psi != Phi

def _dm_problem(K, seed=21, N=16, J=6, Ho=40, Wo=36):
    rng = np.random.default_rng(seed + K)
    obj = np.exp(0.3 * crandn(rng, Ho, Wo))
    probe = crandn(rng, K, N, N)
    pos = np.stack([rng.integers(0, Ho - N + 1, J), rng.integers(0, Wo - N + 1, J)], 1)
    psi = crandn(rng, J, K, N, N)  # arbitrary exit waves, far from Phi
    iobs = rng.uniform(0.5, 5.0, (J, N, N))
    return obj, probe, pos, psi, iobs


def check_masked_detector_gives_phi(dm_cycle, K):
    obj, probe, pos, psi, iobs = _dm_problem(K)
    N = probe.shape[-1]
    data = orc.Data.make(iobs, pos, np.ones((N, N), bool))
    phi = exit_waves_here(obj, probe, pos)
    assert rel(psi, phi) > 0.5
    o, p, psi1, l = dm_cycle(obj, probe, psi, data, update_obj=False, update_probe=False)
    assert rel(psi1, phi) < 1e-13
    assert l == 0.0  # no unmasked pixel contributes
    assert rel(o, obj) == 0.0 and rel(p, probe) == 0.0
    # with the overlap update on: Psi' = P O exactly, a fixed point of Psi2ObjProbe
    o, p, psi1, _ = dm_cycle(obj, probe, psi, data)
    assert rel(psi1, phi) < 1e-13
    assert rel(o, obj) < 1e-13 and rel(p, probe) < 1e-13


def check_zero_intensity_gives_psi_minus_phi(dm_cycle, K):
    obj, probe, pos, psi, iobs = _dm_problem(K)
    N = probe.shape[-1]
    data = orc.Data.make(np.zeros_like(iobs), pos, np.zeros((N, N), bool))
    phi = exit_waves_here(obj, probe, pos)
    o, p, psi1, l = dm_cycle(obj, probe, psi, data, update_obj=False, update_probe=False)
    assert rel(psi1, psi - phi) < 1e-13
    x = 2.0 * phi - psi
    energy = float((x.real ** 2 + x.imag ** 2).sum())
    assert abs(l - energy) < 1e-12 * energy


@pytest.mark.parametrize("K", [1, 2])
def test_dm_fully_masked_detector_returns_phi_for_any_psi(K):
    check_masked_detector_gives_phi(orc.dm_cycle, K)


@pytest.mark.parametrize("K", [1, 2])
def test_dm_zero_intensity_returns_psi_minus_phi_and_parseval_llk(K):
    check_zero_intensity_gives_psi_minus_phi(orc.dm_cycle, K)


DM_MUTATIONS = [
    ("x = 2.0 * phi - psi[lo:hi]", "x = phi"),                       # X = Phi (the AP wave)
    ("x = 2.0 * phi - psi[lo:hi]", "x = 2.0 * phi + psi[lo:hi]"),    # sign of Psi in X
    ("x = 2.0 * phi - psi[lo:hi]", "x = phi - psi[lo:hi]"),          # factor of Phi in X
    ("psi[lo:hi] + x_proj - phi", "psi[lo:hi] + x_proj + phi"),      # sign of Phi in the update
    ("psi[lo:hi] + x_proj - phi", "x_proj - phi"),                   # Psi dropped from the update
    ("psi[lo:hi] + x_proj - phi", "psi[lo:hi] + x_proj"),            # -Phi dropped
    ("llk_poisson(calc_intensity(x_hat)", "llk_poisson(calc_intensity(data.to_detector(phi))"),  # LLK of Phi
]


@pytest.mark.parametrize("old,new", DM_MUTATIONS)
def test_dm_pins_reject_each_planted_mutation_of_the_oracle(old, new):
    bad = mutant(orc.dm_cycle, old, new)
    caught = 0
    for check in (check_masked_detector_gives_phi, check_zero_intensity_gives_psi_minus_phi):
        try:
            check(bad, 1)
        except AssertionError:
            caught += 1
    assert caught >= 1, f"mutation {new!r} passed both DM pins"


# ---------------------------------------------------------------- ML CG direction

def _cg_problem():
    s = make_config("ml32fd")
    data = orc.Data.make(s.iobs, s.positions, s.mask)
    rng = np.random.default_rng(10)
    obj = s.obj0.astype(np.complex128) * (1 + 0.05 * crandn(rng, s.Ho, s.Wo))
    probe = s.probe0.astype(np.complex128)
    # four AP cycles first (ML follows AP / DM in the paper's chains): from there
    # the CG steps include both a clamped beta_PR < 0 and positive ones
    for _ in range(4):
        obj, probe, _ = orc.ap_cycle(obj, probe, data)
    return data, obj, probe


def _vdot(a, b):
    return float(np.real(np.vdot(a, b)))


def check_cg_directions_are_polak_ribiere(ml_cg):
    data, obj, probe = _cg_problem()
    trace = []
    ml_cg(obj, probe, data, 5, update_obj=True, update_probe=True, trace=trace)
    separated = clamped = positive = 0
    for n in range(1, len(trace)):
        t0, t1 = trace[n - 1], trace[n]
        # the iterate moved along the previous direction by the recorded step
        assert rel(t1["obj"], t0["obj"] + t0["alpha"] * t0["dir"][0]) < 1e-14
        _, g0o, g0p = orc.ml_grad(t0["obj"], t0["probe"], data)
        _, g1o, g1p = orc.ml_grad(t1["obj"], t1["probe"], data)
        gg0 = _vdot(g0o, g0o) + _vdot(g0p, g0p)
        beta_pr = (_vdot(g1o, g1o - g0o) + _vdot(g1p, g1p - g0p)) / gg0
        beta_fr = (_vdot(g1o, g1o) + _vdot(g1p, g1p)) / gg0
        if abs(beta_pr - beta_fr) > 0.1 * abs(beta_fr):
            separated += 1
        beta = max(0.0, beta_pr)
        clamped += beta_pr < 0
        positive += beta_pr > 0.05
        assert abs(t1["beta"] - beta) <= 1e-9 * max(abs(beta_fr), 1e-300), (n, t1["beta"], beta_pr, beta_fr)
        d_obj = -g1o + beta * t0["dir"][0]
        d_probe = -g1p + beta * t0["dir"][1]
        assert rel(t1["dir"][0], d_obj) < 1e-9 and rel(t1["dir"][1], d_probe) < 1e-9
    # the case tells Polak-Ribiere from Fletcher-Reeves at least once, and takes
    # both branches of max(0, beta_PR)
    assert separated >= 1 and clamped >= 1 and positive >= 1


def test_ml_cg_directions_follow_polak_ribiere_from_pinned_gradients():
    trace = []
    data, obj, probe = _cg_problem()
    orc.ml_cg(obj, probe, data, 1, trace=trace)
    _, go, _ = orc.ml_grad(obj, probe, data)
    assert trace[0]["beta"] == 0.0 and rel(trace[0]["dir"][0], -go) < 1e-14  # first step: steepest descent
    check_cg_directions_are_polak_ribiere(orc.ml_cg)


@pytest.mark.parametrize("old,new", [
    ("num = _dot(go, go - g_prev[0]) + _dot(gp, gp - g_prev[1])", "num = _dot(go, go) + _dot(gp, gp)"),  # FR
    ("d = (-go + beta * d[0], -gp + beta * d[1])", "d = (-go - beta * d[0], -gp - beta * d[1])"),         # sign
    ("d = (-go + beta * d[0], -gp + beta * d[1])", "d = (-go, -gp)"),                                     # no memory
    ("beta = max(0.0, num / den)", "beta = num / den"),                                                   # no clamp
])
def test_cg_pin_rejects_planted_mutations_of_the_oracle(old, new):
    bad = mutant(orc.ml_cg, old, new)
    with pytest.raises(AssertionError):
        check_cg_directions_are_polak_ribiere(bad)
