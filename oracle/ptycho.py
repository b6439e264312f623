"""FP64 CPU oracle for the ptychography projection cycle (far and near field).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product path (``paper_2008_11511_gb300``) never calls it and has
no CPU fallback.  It shares no code with the CUDA path; the only common input
source is the seeded generator in ``synthetic/``.

Everything is plain NumPy/SciPy in float64 / complex128, written to be checked
against the paper by eye.  The paper (PyNX, Favre-Nicolin et al. 2020) gives
the operators by name and definition; the algorithms it cites (DM: Elser 2007
and its ptychographic form by Thibault et al. 2008/2009; AP: Marchesini et al.
2013; ML: Thibault & Guizar-Sicairos 2012; incoherent modes: Thibault & Menzel
2013) are restated here from their mathematics.

Notation (paper, Section 4 and the ptychography operator table in the
appendix): J positions r_j, K probe modes P_k (N x N), object O (Ho x Wo),
exit waves Psi_jk.  ``FT`` is the orthonormal 2D DFT over the last two axes,
arrays in FFT order (zero frequency at [0, 0]).  A position (row, col) is the
top-left corner of the frame's object patch.

Readings of points the paper leaves open:
* FT normalisation: orthonormal, so IFT = FT^H and Parseval holds exactly.
* ObjProbe2Psi: Phi_jk(x) = P_k(x) O(r_j + x) (the paper writes
  Psi_j(r) = O(r) P(r - r_j); with integer top-left positions this is the same
  product on the patch).
* ApplyAmplitude with modes: one common factor sqrt(I_obs) / sqrt(sum_k |Psi_k|^2)
  for all modes; masked pixels left unchanged; I_obs clamped at 0; a zero
  calculated amplitude stays zero (denominator floored at 1e-20).
* LLK (Poisson): the deviance form sum over unmasked pixels of
  I_c - I_o + I_o ln(I_o / I_c) (= I_c where I_o = 0), I_c floored at 1e-30 in
  the log.  It is 0 on exact data and >= 0.
* DM: beta = 1 difference map, Psi <- Psi + P_F(2 P_O Psi - Psi) - P_O Psi, with
  P_O Psi = Phi formed from the current O, P; Psi starts at Phi.
* Psi2ObjProbe: one alternation of the two least-squares updates, probe first:
  P <- (N_P + d_P P) / (D_P + d_P) with N_P, D_P from the current object, then
  O <- (N_O + d_O O) / (D_O + d_O) with N_O, D_O from the new probe; inertia
  d = alpha max D.  (Updating both from the same pre-update O, P lets a scale
  error of Psi enter both factors, so P O absorbs it twice; under DM that
  doubling makes the iteration diverge, |Psi| x2.5 per cycle on the 64x64
  scan.)
* The per-cycle LLK is that of the wave being projected (Phi for AP, 2 Phi - Psi
  for DM); ``llk`` gives the exact L(O, P).
* Incoherent background (the Ptycho object's background, optimised in AP;
  the paper cites Marchesini et al. 2013 without a formula): one N x N array B
  >= 0 added to every frame's model intensity (LLK, projection, gradient);
  the projection scales it like a mode, and ``ap_cycle_background`` replaces B
  by the mean over frames of the scaled backgrounds.  B = 0 stays 0 (the update
  is multiplicative), so a reconstruction starts it at a positive guess.
* Position refinement (Psi2PosShift; the paper cites Odstrcil et al. 2018 and
  adds a filter against weak object gradients, without formulas): per frame
  the first-order least-squares shift between Phi_j and the projected Psi_j,
  object gradient by central differences; frames whose gradient norm is below
  a fraction of the mean over frames keep their position.  Positions stay
  integer in the cycle; the caller accumulates the shifts and moves a frame
  when its accumulated shift rounds to a new pixel.
* Near field (PropagateNearField; the paper names the operator and the near /
  far field flag but gives no formula): paraxial Fresnel propagation in
  Fourier space, IFT(FT(x) exp(-i pi lambda z q^2)), q = k / (N pixel) the
  signed spatial frequency, parametrised by c = lambda z / pixel^2; back
  propagation uses the conjugate transfer.  The near-field amplitude projection
  is PropagateNearField^-1 ApplyAmplitude PropagateNearField (the paper's
  PropagateApplyAmplitude), with intensities and mask in detector pixels.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np
import scipy.fft

ICALC_FLOOR = 1e-30   # floor of the calculated intensity inside log and ratio
AMP_FLOOR = 1e-20     # floor of the calculated amplitude in the projection
STACK = 64            # frames per stack (the paper processes Psi in stacks of 16-128 frames)


def _workers():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


@dataclass
class Data:
    """PtychoData (paper Section 4): observed intensities, positions, mask and
    the near / far field flag.  ``nearfield`` = 0 is the far field (the
    detector sees FT(Psi), intensities in FFT order); ``nearfield`` = c > 0 is
    the near field with propagation factor c = lambda z / pixel^2 (the detector
    sees PropagateNearField(Psi), intensities in real-space order)."""

    iobs: np.ndarray       # float64 (J, N, N)
    positions: np.ndarray  # int64 (J, 2) top-left (row, col)
    mask: np.ndarray       # bool (N, N), True = bad pixel (free)
    nearfield: float = 0.0
    background: np.ndarray | None = None  # float64 (N, N) incoherent background, or None

    @staticmethod
    def make(iobs, positions, mask=None, nearfield=0.0, background=None):
        iobs = np.asarray(iobs, dtype=np.float64)
        N = iobs.shape[-1]
        if mask is None:
            mask = np.zeros((N, N), dtype=bool)
        bg = None if background is None else np.asarray(background, dtype=np.float64).reshape(N, N)
        return Data(iobs=iobs, positions=np.asarray(positions, dtype=np.int64),
                    mask=np.asarray(mask).astype(bool), nearfield=float(nearfield), background=bg)

    @property
    def bg(self):
        """The incoherent background added to every frame's model intensity (0 if none)."""
        return 0.0 if self.background is None else self.background

    @property
    def J(self):
        return self.iobs.shape[0]

    @property
    def N(self):
        return self.iobs.shape[-1]

    def to_detector(self, x):
        """The wave at the detector: FT (far field) or PropagateNearField forward."""
        return ft(x) if self.nearfield == 0 else propagate_near_field(x, self.nearfield, +1)

    def from_detector(self, y):
        """Inverse (and adjoint) of ``to_detector``."""
        return ift(y) if self.nearfield == 0 else propagate_near_field(y, self.nearfield, -1)


# --------------------------------------------------------------------------
# Operators (paper appendix, "Ptychography operators")
# --------------------------------------------------------------------------

def ft(x):
    """FT: orthonormal 2D discrete Fourier transform over the last two axes."""
    return scipy.fft.fft2(x, axes=(-2, -1), norm="ortho", workers=_workers())


def ift(x):
    """IFT: inverse of ``ft`` (its adjoint, as ``ft`` is unitary)."""
    return scipy.fft.ifft2(x, axes=(-2, -1), norm="ortho", workers=_workers())


def near_field_transfer(N, c):
    """Fresnel (paraxial) transfer function on the N x N frequency grid in FFT
    order: h[ky, kx] = exp(-i pi c (ky^2 + kx^2) / N^2), k the signed integer
    frequency (k - N for k >= N / 2) and c = lambda z / pixel^2 (a plane wave of
    spatial frequency q = k / (N pixel) gains the phase -pi lambda z q^2)."""
    k = np.fft.fftfreq(N) * N
    q2 = k[:, None] ** 2 + k[None, :] ** 2
    return np.exp(-1j * np.pi * c * q2 / N ** 2)


def propagate_near_field(x, c, direction=+1):
    """PropagateNearField: IFT(FT(x) h) over the last two axes; direction -1
    propagates back (conj(h), the inverse and adjoint, as |h| = 1)."""
    h = near_field_transfer(x.shape[-1], c)
    if direction < 0:
        h = np.conj(h)
    return ift(ft(x) * h)


def obj_probe_to_psi(obj, probe, positions):
    """ObjProbe2Psi: Phi[j, k] = P_k * O[r_j : r_j + N, c_j : c_j + N]."""
    K, N, _ = probe.shape
    out = np.empty((len(positions), K, N, N), dtype=np.complex128)
    for j, (r, c) in enumerate(positions):
        out[j] = probe * obj[r:r + N, c:c + N][None]
    return out


def calc_intensity(psi_hat):
    """Incoherent sum over probe modes: I_c = sum_k |Psi_hat_k|^2 (modes on axis -3)."""
    return (psi_hat.real ** 2 + psi_hat.imag ** 2).sum(axis=-3)


def apply_amplitude(psi_hat, iobs, mask, background=0.0):
    """ApplyAmplitude: in Fourier space replace the modulus by the observed
    amplitude, with one common factor for all modes; masked pixels unchanged.
    An incoherent background B is one more incoherent component of the model
    intensity (Marchesini et al. 2013's augmented projection): the factor is
    sqrt(I_obs) / sqrt(sum_k |Psi_k|^2 + B).

    psi_hat: (..., K, N, N); iobs: (..., N, N); mask: (N, N) bool.
    """
    ic = calc_intensity(psi_hat) + background
    s = np.sqrt(np.maximum(iobs, 0.0)) / np.maximum(np.sqrt(ic), AMP_FLOOR)
    s = np.where(mask, 1.0, s)
    return psi_hat * s[..., None, :, :]


def llk_terms(icalc, iobs, mask):
    """Poisson log-likelihood per pixel (deviance form), 0 on masked pixels:
    I_c - I_o + I_o ln(I_o / I_c), which is I_c where I_o = 0."""
    io = np.maximum(iobs, 0.0)
    ic = icalc
    with np.errstate(divide="ignore", invalid="ignore"):
        t = ic - io + np.where(io > 0, io * np.log(np.where(io > 0, io, 1.0) / np.maximum(ic, ICALC_FLOOR)), 0.0)
    return np.where(mask, 0.0, t)


def llk_poisson(icalc, iobs, mask):
    """LLK operator: total Poisson log-likelihood (sum of ``llk_terms``)."""
    return float(llk_terms(icalc, iobs, mask).sum())


def psi_to_probe_sums(psi, obj, positions):
    """Psi2ObjProbe probe numerator and denominator from the object O:
      N_Pk(x) = sum_j conj(O(r_j + x)) Psi_jk(x),   D_P(x) = sum_j |O(r_j + x)|^2"""
    J, K, N, _ = psi.shape
    n_p = np.zeros((K, N, N), dtype=np.complex128)
    d_p = np.zeros((N, N), dtype=np.float64)
    for j, (r, c) in enumerate(positions):
        patch = obj[r:r + N, c:c + N]
        n_p += np.conj(patch)[None] * psi[j]
        d_p += patch.real ** 2 + patch.imag ** 2
    return n_p, d_p


def psi_to_obj_sums(psi, probe, positions, shape_obj):
    """Psi2ObjProbe object numerator and denominator from the probe P:
      N_O(r_j + x) += sum_k conj(P_k(x)) Psi_jk(x),   D_O(r_j + x) += sum_k |P_k(x)|^2"""
    K, N, _ = probe.shape
    n_o = np.zeros(shape_obj, dtype=np.complex128)
    d_o = np.zeros(shape_obj, dtype=np.float64)
    p_conj = np.conj(probe)
    p_pow = (probe.real ** 2 + probe.imag ** 2).sum(0)
    for j, (r, c) in enumerate(positions):
        n_o[r:r + N, c:c + N] += (p_conj * psi[j]).sum(0)
        d_o[r:r + N, c:c + N] += p_pow
    return n_o, d_o


def psi_to_obj_probe_sums(psi, obj, probe, positions, shape_obj):
    """All four sums from the same (O, P): (N_O, D_O, N_P, D_P)."""
    n_o, d_o = psi_to_obj_sums(psi, probe, positions, shape_obj)
    n_p, d_p = psi_to_probe_sums(psi, obj, positions)
    return n_o, d_o, n_p, d_p


def inertia_update(old, num, den, alpha):
    """(num + d old) / (den + d), d = alpha max(den) (inertia, Section 4 feature list).
    A pixel whose denominator den + d is zero (alpha = 0 and never illuminated)
    keeps its value (the paper is silent on this case).  ``den`` broadcasts over
    leading axes of ``old`` (probe modes)."""
    delta = alpha * den.max()
    d = den + delta
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(d > 0, (num + delta * old) / d, old)


def normalise(obj, probe, sums, alpha_obj=1e-2, alpha_probe=1e-2,
              update_obj=True, update_probe=True):
    """Normalisation of precomputed sums (N_O, D_O, N_P, D_P) with inertia."""
    n_o, d_o, n_p, d_p = sums
    if update_obj:
        obj = inertia_update(obj, n_o, d_o, alpha_obj)
    if update_probe:
        probe = inertia_update(probe, n_p, d_p[None], alpha_probe)
    return obj, probe


def overlap_update(obj, probe, psi, positions, alpha_obj=1e-2, alpha_probe=1e-2,
                   update_obj=True, update_probe=True):
    """Psi2ObjProbe: update the probe and/or the object from the exit waves Psi
    (paper: operator table): probe first from the current object, then the
    object from the new probe."""
    if update_probe:
        n_p, d_p = psi_to_probe_sums(psi, obj, positions)
        probe = inertia_update(probe, n_p, d_p[None], alpha_probe)
    if update_obj:
        n_o, d_o = psi_to_obj_sums(psi, probe, positions, obj.shape)
        obj = inertia_update(obj, n_o, d_o, alpha_obj)
    return obj, probe


def _stacks(J, stack=STACK):
    for lo in range(0, J, stack):
        yield lo, min(J, lo + stack)


# --------------------------------------------------------------------------
# Algorithms
# --------------------------------------------------------------------------

def ap_cycle(obj, probe, data: Data, alpha_obj=1e-2, alpha_probe=1e-2,
             update_obj=True, update_probe=True):
    """One Alternating Projections cycle (AP, Marchesini et al. 2013):
    Psi_j = IFT(ApplyAmplitude(FT(Phi_j))), Phi = ObjProbe2Psi(O, P), then
    Psi2ObjProbe.  In the near field FT / IFT are the forward and backward
    PropagateNearField (the paper's PropagateApplyAmplitude operator).
    Returns (obj, probe, llk of the detector wave of Phi)."""
    obj = np.asarray(obj, dtype=np.complex128)
    probe = np.asarray(probe, dtype=np.complex128)
    psi = np.empty((data.J,) + probe.shape, dtype=np.complex128)
    llk = 0.0
    for lo, hi in _stacks(data.J):
        pos = data.positions[lo:hi]
        phi = obj_probe_to_psi(obj, probe, pos)
        phi_hat = data.to_detector(phi)
        llk += llk_poisson(calc_intensity(phi_hat) + data.bg, data.iobs[lo:hi], data.mask)
        psi[lo:hi] = data.from_detector(apply_amplitude(phi_hat, data.iobs[lo:hi], data.mask, data.bg))
    obj, probe = overlap_update(obj, probe, psi, data.positions, alpha_obj, alpha_probe, update_obj, update_probe)
    return obj, probe, llk


def ap_cycle_background(obj, probe, background, data: Data, alpha_obj=1e-2, alpha_probe=1e-2,
                        update_obj=True, update_probe=True):
    """AP cycle with the incoherent background optimisation (paper Section 4:
    "incoherent background optimisation (AP)", Marchesini et al. 2013).  The
    background B is an incoherent component of every frame's model intensity,
    I_c + B; the augmented amplitude projection scales it with the frames' modes
    (B_j' = s_j^2 B, s_j = sqrt(I_o,j / (I_c,j + B))), and the new background is
    their least-squares common value, the mean over frames:
        B <- B * (1 / J) sum_j I_o,j / (I_c,j + B)     (unmasked pixels; masked keep B).
    The waves are projected with the current B; O, P are updated from them as in
    ``ap_cycle``.  Returns (obj, probe, background, llk)."""
    background = np.asarray(background, dtype=np.float64)
    d = Data(iobs=data.iobs, positions=data.positions, mask=data.mask, nearfield=data.nearfield, background=background)
    obj = np.asarray(obj, dtype=np.complex128)
    probe = np.asarray(probe, dtype=np.complex128)
    psi = np.empty((d.J,) + probe.shape, dtype=np.complex128)
    llk = 0.0
    ratio = np.zeros_like(background)
    for lo, hi in _stacks(d.J):
        phi = obj_probe_to_psi(obj, probe, d.positions[lo:hi])
        phi_hat = d.to_detector(phi)
        ic = calc_intensity(phi_hat) + background
        llk += llk_poisson(ic, d.iobs[lo:hi], d.mask)
        ratio += (np.maximum(d.iobs[lo:hi], 0.0) / np.maximum(ic, ICALC_FLOOR)).sum(axis=0)
        psi[lo:hi] = d.from_detector(apply_amplitude(phi_hat, d.iobs[lo:hi], d.mask, background))
    new_bg = np.where(d.mask, background, background * ratio / d.J)
    obj, probe = overlap_update(obj, probe, psi, d.positions, alpha_obj, alpha_probe, update_obj, update_probe)
    return obj, probe, new_bg, llk


def object_gradient(obj):
    """(dO/dy, dO/dx) of the object by central differences, one-sided on the
    object's first and last row / column."""
    gy = np.empty_like(obj)
    gx = np.empty_like(obj)
    gy[1:-1] = 0.5 * (obj[2:] - obj[:-2])
    gy[0] = obj[1] - obj[0]
    gy[-1] = obj[-1] - obj[-2]
    gx[:, 1:-1] = 0.5 * (obj[:, 2:] - obj[:, :-2])
    gx[:, 0] = obj[:, 1] - obj[:, 0]
    gx[:, -1] = obj[:, -1] - obj[:, -2]
    return gy, gx


def position_shifts(obj, probe, psi, positions, filter_ratio=0.1):
    """Position refinement (Psi2PosShift; paper Section 4, after Odstrcil et al.
    2018): for frame j the shift d = (d_y, d_x) that moves the model exit wave
    Phi_j = P O[r_j] towards the projected wave Psi_j in the least-squares
    sense, to first order in the shift: with chi = Psi_j - Phi_j and
    G_a = P dO/da (a = y, x) on the patch, summed over modes and pixels,
        [<G_y,G_y> <G_y,G_x>] [d_y]   [<G_y,chi>]
        [<G_x,G_y> <G_x,G_x>] [d_x] = [<G_x,chi>],   <u,v> = sum Re(conj(u) v).
    The paper adds a filter against shifting where the object gradient is
    weak: a frame whose gradient norm <G_y,G_y> + <G_x,G_x> is below
    ``filter_ratio`` times the mean over frames keeps its position (shift 0),
    as does a frame whose 2 x 2 system is singular.
    Returns float64 (J, 2) shifts (row, col) in pixels."""
    obj = np.asarray(obj, dtype=np.complex128)
    probe = np.asarray(probe, dtype=np.complex128)
    K, N, _ = probe.shape
    gy, gx = object_gradient(obj)
    J = len(positions)
    out = np.zeros((J, 2))
    norm = np.zeros(J)
    systems = []
    dot = lambda u, v: float((np.conj(u) * v).real.sum())
    for j, (r, c) in enumerate(positions):
        sl = (slice(r, r + N), slice(c, c + N))
        chi = psi[j] - probe * obj[sl][None]
        g_y = probe * gy[sl][None]
        g_x = probe * gx[sl][None]
        a = np.array([[dot(g_y, g_y), dot(g_y, g_x)], [dot(g_x, g_y), dot(g_x, g_x)]])
        systems.append((a, np.array([dot(g_y, chi), dot(g_x, chi)])))
        norm[j] = a[0, 0] + a[1, 1]
    for j, (a, b) in enumerate(systems):
        det = a[0, 0] * a[1, 1] - a[0, 1] * a[1, 0]
        if norm[j] >= filter_ratio * norm.mean() and det > 1e-12 * norm[j] ** 2:
            out[j] = np.linalg.solve(a, b)
    return out


def refine_positions_step(pos_subpixel, shifts, step, max_shift, max_row, max_col):
    """The host step of position refinement (paper Section 4, after Odstrcil et
    al. 2018; positions stay integer inside the cycle): each frame's shift,
    scaled by ``step`` and clipped to [-max_shift, max_shift] pixels per axis,
    is added to its sub-pixel position, which is kept inside [0, max_row] x
    [0, max_col] (max_row = Ho - N, max_col = Wo - N); the frame's integer
    position is the nearest integer, halves to even.
    Returns (sub-pixel positions float64 (J, 2), integer positions int64 (J, 2))."""
    pos = np.asarray(pos_subpixel, dtype=np.float64)
    d = np.clip(step * np.asarray(shifts, dtype=np.float64), -max_shift, max_shift)
    hi = np.array([max_row, max_col], dtype=np.float64)
    new = np.clip(pos + d, 0.0, hi)
    return new, np.rint(new).astype(np.int64)


def dm_cycle(obj, probe, psi, data: Data, alpha_obj=1e-2, alpha_probe=1e-2,
             update_obj=True, update_probe=True, init_psi=False):
    """One Difference Map cycle (beta = 1; Elser 2007, Thibault et al. 2008):
    Phi = ObjProbe2Psi(O, P); X = 2 Phi - Psi;
    Psi <- Psi + IFT(ApplyAmplitude(FT(X))) - Phi; then Psi2ObjProbe from the new Psi
    (near field: PropagateNearField forward / back in place of FT / IFT).
    ``init_psi`` sets Psi = Phi first.  Returns (obj, probe, psi, llk of FT(X))."""
    obj = np.asarray(obj, dtype=np.complex128)
    probe = np.asarray(probe, dtype=np.complex128)
    psi = np.array(psi, dtype=np.complex128, copy=True) if psi is not None else None
    J = data.J
    if init_psi or psi is None:
        psi = np.empty((J,) + probe.shape, dtype=np.complex128)
        init_psi = True
    llk = 0.0
    for lo, hi in _stacks(J):
        pos = data.positions[lo:hi]
        phi = obj_probe_to_psi(obj, probe, pos)
        if init_psi:
            psi[lo:hi] = phi
        x = 2.0 * phi - psi[lo:hi]
        x_hat = data.to_detector(x)
        llk += llk_poisson(calc_intensity(x_hat) + data.bg, data.iobs[lo:hi], data.mask)
        x_proj = data.from_detector(apply_amplitude(x_hat, data.iobs[lo:hi], data.mask, data.bg))
        psi[lo:hi] = psi[lo:hi] + x_proj - phi
    obj, probe = overlap_update(obj, probe, psi, data.positions, alpha_obj, alpha_probe, update_obj, update_probe)
    return obj, probe, psi, llk


def llk(obj, probe, data: Data):
    """Exact Poisson LLK of (O, P): LLK operator applied to FT(ObjProbe2Psi(O, P))."""
    obj = np.asarray(obj, dtype=np.complex128)
    probe = np.asarray(probe, dtype=np.complex128)
    total = 0.0
    for lo, hi in _stacks(data.J):
        phi_hat = data.to_detector(obj_probe_to_psi(obj, probe, data.positions[lo:hi]))
        total += llk_poisson(calc_intensity(phi_hat) + data.bg, data.iobs[lo:hi], data.mask)
    return total


def ml_grad(obj, probe, data: Data):
    """Gradient of the Poisson LLK (ML, Thibault & Guizar-Sicairos 2012).

    L(O, P) = sum_j sum_unmasked [I_c - I_o ln I_c] (+ a constant; same gradient
    as the deviance returned by ``llk``), I_c = sum_k |FT(Phi_jk)|^2.
    With z complex, the returned gradient is dL/dRe z + i dL/dIm z:

      G_O(r_j + x) = sum_jk conj(P_k(x)) IFT[w_j FT(Phi_jk)](x)
      G_Pk(x)      = sum_j  conj(O(r_j + x)) IFT[w_j FT(Phi_jk)](x)
      w_j = 2 (1 - I_o / I_c) on unmasked pixels, 0 on masked ones.

    In the near field FT / IFT are PropagateNearField forward / back (the
    adjoint of a unitary propagator is its inverse).
    Returns (llk deviance, G_O, G_P)."""
    obj = np.asarray(obj, dtype=np.complex128)
    probe = np.asarray(probe, dtype=np.complex128)
    K, N, _ = probe.shape
    g_o = np.zeros(obj.shape, dtype=np.complex128)
    g_p = np.zeros(probe.shape, dtype=np.complex128)
    total = 0.0
    for lo, hi in _stacks(data.J):
        pos = data.positions[lo:hi]
        phi_hat = data.to_detector(obj_probe_to_psi(obj, probe, pos))
        ic = calc_intensity(phi_hat) + data.bg
        io = np.maximum(data.iobs[lo:hi], 0.0)
        total += llk_poisson(ic, data.iobs[lo:hi], data.mask)
        w = np.where(data.mask, 0.0, 2.0 * (1.0 - io / np.maximum(ic, ICALC_FLOOR)))
        back = data.from_detector(phi_hat * w[:, None])
        for i, (r, c) in enumerate(pos):
            patch = obj[r:r + N, c:c + N]
            g_o[r:r + N, c:c + N] += (np.conj(probe) * back[i]).sum(0)
            g_p += np.conj(patch)[None] * back[i]
    return total, g_o, g_p


def ml_line_coeffs(obj, probe, d_obj, d_probe, data: Data):
    """Derivatives of L(alpha) = L(O + alpha dO, P + alpha dP) at alpha = 0 from the
    expansion of the far field along the direction (ML line search, Thibault &
    Guizar-Sicairos 2012):
      FT((P + a dP)(O + a dO)) = A + a B + a^2 C,
      A = FT(P O), B = FT(dP O + P dO), C = FT(dP dO);
      I_c(a) = sum_k |A + a B + a^2 C|^2 = I_c + a dI + a^2 d2I / 2 + O(a^3),
      dI = 2 sum_k Re(conj(A) B),  d2I = 2 sum_k (|B|^2 + 2 Re(conj(A) C));
      L'(0) = sum (1 - I_o / I_c) dI,
      L''(0) = sum [(1 - I_o / I_c) d2I + (I_o / I_c^2) dI^2]   (unmasked pixels).
    Returns (L'(0), L''(0))."""
    obj = np.asarray(obj, dtype=np.complex128)
    probe = np.asarray(probe, dtype=np.complex128)
    d_obj = np.asarray(d_obj, dtype=np.complex128)
    d_probe = np.asarray(d_probe, dtype=np.complex128)
    l1 = l2 = 0.0
    for lo, hi in _stacks(data.J):
        pos = data.positions[lo:hi]
        A = data.to_detector(obj_probe_to_psi(obj, probe, pos))
        B = data.to_detector(obj_probe_to_psi(obj, d_probe, pos) + obj_probe_to_psi(d_obj, probe, pos))
        C = data.to_detector(obj_probe_to_psi(d_obj, d_probe, pos))
        ic = calc_intensity(A) + data.bg
        di = 2.0 * (np.conj(A) * B).real.sum(axis=-3)
        d2i = 2.0 * ((B.real ** 2 + B.imag ** 2) + 2.0 * (np.conj(A) * C).real).sum(axis=-3)
        io = np.maximum(data.iobs[lo:hi], 0.0)
        icf = np.maximum(ic, ICALC_FLOOR)
        w1 = np.where(data.mask, 0.0, 1.0 - io / icf)
        w2 = np.where(data.mask, 0.0, io / icf ** 2)
        l1 += float((w1 * di).sum())
        l2 += float((w1 * d2i + w2 * di ** 2).sum())
    return l1, l2


def _dot(a, b):
    """Real inner product Re sum conj(a) b of complex arrays."""
    return float(np.real(np.vdot(a, b)))


def ml_cg(obj, probe, data: Data, n, update_obj=True, update_probe=False, trace=None):
    """n steps of maximum-likelihood conjugate gradient on the Poisson LLK (the ML
    operator; Thibault & Guizar-Sicairos 2012; the paper's ML defaults update the
    object only).  Polak-Ribiere direction with beta = max(0, beta_PR) (0 at the
    first step); step alpha = -L'(0) / L''(0) from ``ml_line_coeffs`` (no step
    when L''(0) <= 0).  If ``trace`` is a list, each step appends a dict with its
    start point, beta, search direction and alpha (for the tests).
    Returns (obj, probe, [LLK before each step])."""
    obj = np.asarray(obj, dtype=np.complex128).copy()
    probe = np.asarray(probe, dtype=np.complex128).copy()
    g_prev = d = None
    llks = []
    for it in range(n):
        l, go, gp = ml_grad(obj, probe, data)
        llks.append(l)
        go = go if update_obj else np.zeros_like(go)
        gp = gp if update_probe else np.zeros_like(gp)
        if g_prev is None:
            beta = 0.0
        else:
            den = _dot(g_prev[0], g_prev[0]) + _dot(g_prev[1], g_prev[1])
            num = _dot(go, go - g_prev[0]) + _dot(gp, gp - g_prev[1])
            beta = max(0.0, num / den) if den > 0 else 0.0
        if d is None:
            d = (-go, -gp)
        else:
            d = (-go + beta * d[0], -gp + beta * d[1])
        l1, l2 = ml_line_coeffs(obj, probe, d[0], d[1], data)
        alpha = -l1 / l2 if l2 > 0 else 0.0
        if trace is not None:
            trace.append({"obj": obj.copy(), "probe": probe.copy(), "beta": beta,
                          "dir": (d[0].copy(), d[1].copy()), "alpha": alpha})
        obj = obj + alpha * d[0]
        probe = probe + alpha * d[1]
        g_prev = (go, gp)
    return obj, probe, llks


def cycles(algorithm, obj, probe, data: Data, n, psi=None, init_psi=True, **kw):
    """Run ``n`` AP or DM cycles; returns (obj, probe, psi, [llk per cycle])."""
    llks = []
    for i in range(n):
        if algorithm == "AP":
            obj, probe, l = ap_cycle(obj, probe, data, **kw)
        elif algorithm == "DM":
            obj, probe, psi, l = dm_cycle(obj, probe, psi, data, init_psi=(init_psi and i == 0), **kw)
        else:
            raise ValueError(algorithm)
        llks.append(l)
    return obj, probe, psi, llks


# --------------------------------------------------------------------------
# Sampled outputs for full-size checks: values the oracle can compute one frame
# or one object pixel at a time.
# --------------------------------------------------------------------------

def dm_frame_update(obj, probe, psi_j, iobs_j, pos_j, mask, init_psi=False, nearfield=0.0):
    """New Psi_j and the LLK of frame j for one DM step (the frame's part of
    ``dm_cycle``).  Returns (psi_new_j, llk_j)."""
    obj = np.asarray(obj, dtype=np.complex128)
    probe = np.asarray(probe, dtype=np.complex128)
    d = Data.make(np.asarray(iobs_j, np.float64)[None], np.asarray([pos_j]), mask, nearfield)
    phi = obj_probe_to_psi(obj, probe, np.asarray([pos_j]))[0]
    psi_j = phi if init_psi else np.asarray(psi_j, dtype=np.complex128)
    x_hat = d.to_detector(2.0 * phi - psi_j)
    l = llk_poisson(calc_intensity(x_hat), d.iobs[0], d.mask)
    return psi_j + d.from_detector(apply_amplitude(x_hat, d.iobs[0], d.mask)) - phi, l


def frames_llk(obj, probe, data: Data, frames):
    """Exact LLK of a subset of frames."""
    obj = np.asarray(obj, dtype=np.complex128)
    probe = np.asarray(probe, dtype=np.complex128)
    frames = np.asarray(frames)
    phi_hat = data.to_detector(obj_probe_to_psi(obj, probe, data.positions[frames]))
    return llk_poisson(calc_intensity(phi_hat) + data.bg, data.iobs[frames], data.mask)


def object_denominator(probe, positions, shape_obj):
    """D_O = sum_j sum_k |P_k(x)|^2 placed at r_j + x (needs no transforms)."""
    K, N, _ = probe.shape
    p_pow = (np.abs(np.asarray(probe, np.complex128)) ** 2).sum(0)
    d_o = np.zeros(shape_obj, dtype=np.float64)
    for r, c in positions:
        d_o[r:r + N, c:c + N] += p_pow
    return d_o


def frames_covering(positions, N, pixel):
    """Indices j whose N x N patch contains object pixel (row, col)."""
    y, x = pixel
    p = np.asarray(positions)
    sel = (p[:, 0] <= y) & (y < p[:, 0] + N) & (p[:, 1] <= x) & (x < p[:, 1] + N)
    return np.nonzero(sel)[0]


__all__ = [
    "Data", "ft", "ift", "obj_probe_to_psi", "calc_intensity", "apply_amplitude", "llk_terms",
    "llk_poisson", "psi_to_probe_sums", "psi_to_obj_sums", "psi_to_obj_probe_sums", "inertia_update",
    "normalise", "overlap_update", "ap_cycle", "dm_cycle", "llk", "ml_grad",
    "cycles", "dm_frame_update", "frames_llk", "object_denominator", "frames_covering", "ml_line_coeffs", "ml_cg",
    "ap_cycle_background", "near_field_transfer", "propagate_near_field", "object_gradient", "position_shifts",
    "refine_positions_step", "ICALC_FLOOR", "AMP_FLOOR", "STACK",
]


def unit_count(data: Data) -> int:
    """Number of unmasked detector pixels over all frames (the LLK normaliser)."""
    return int((~data.mask).sum()) * data.J

