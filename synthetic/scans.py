"""Seeded synthetic scans shaped like the paper's far-field ptychography workloads.

The paper's Table 1 measures far-field ptychography on 1000 frames of 256x256
pixels (1 and 3 probe modes), its Fig. 7 uses 400x400 frames and its MPI runs
70k frames of 512x512 and 250k of 256x256 (Section 4, Table 1).  Its datasets
are not available, so every input here is synthetic: this module draws a
smooth random complex object, a disk (or Hermite-Gauss) probe with a quadratic
phase, Fermat-spiral positions, a detector-gap mask, and Poisson-noised
far-field intensities.  The intensities come from one application of the
far-field forward model |FT(P . O[r_j])|^2 through ``scipy.fft`` -- this is
data simulation (the paper's "functions to simulate data" feature, Section 4),
not any step of a reconstruction.

Conventions shared with both the oracle and the CUDA path:

* arrays are C-contiguous; the object is ``(Ho, Wo)``, the probe ``(K, N, N)``;
* a position ``(row, col)`` is the top-left corner of the frame's object patch:
  the exit wave of frame j, mode k is ``P_k(y, x) * O(row_j + y, col_j + x)``;
* intensities and the mask are stored in FFT order (zero frequency at [0, 0]);
* ``mask`` is uint8, 1 = bad pixel (left free by the projection);
* the 2D transform is orthonormal (``norm="ortho"``).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np
import scipy.fft
import scipy.ndimage

_GOLDEN_ANGLE_DEG = 137.508


@dataclass
class Scan:
    """One synthetic ptychography problem (inputs for a reconstruction)."""

    name: str
    N: int
    K: int
    J: int
    Ho: int
    Wo: int
    positions: np.ndarray  # int32 (J, 2): (row, col) top-left corners
    iobs: np.ndarray  # float32 (J, N, N): FFT order (far field) or detector pixels (near field)
    mask: np.ndarray  # uint8 (N, N), 1 = masked, FFT order
    obj_true: np.ndarray  # complex128 (Ho, Wo)
    probe_true: np.ndarray  # complex128 (K, N, N), scaled to the photon count
    obj0: np.ndarray  # complex64 (Ho, Wo): starting object
    probe0: np.ndarray  # complex64 (K, N, N): starting probe
    photons: float
    seed: int
    step_px: float  # achieved mean nearest-neighbour step of the spiral
    algorithm: str = "AP"
    cycles: int = 20
    nearfield: float = 0.0  # 0: far field; c = lambda z / pixel^2 > 0: near field
    meta: dict = field(default_factory=dict)


def fermat_spiral(J: int, step: float, Ho: int, Wo: int, N: int):
    """Integer top-left positions on a Fermat spiral centred in the object.

    r_m = c sqrt(m), theta_m = m * 137.508 deg, c = step / sqrt(pi), so each
    point owns an area of about step^2.  If the spiral does not fit inside
    [0, Ho - N] x [0, Wo - N] it is shrunk uniformly to fit; the object size is
    authoritative.  Returns (positions int32 (J, 2), achieved mean
    nearest-neighbour distance in pixels).
    """
    c = step / math.sqrt(math.pi)
    half_y = (Ho - N) / 2.0
    half_x = (Wo - N) / 2.0
    rmax = c * math.sqrt(max(J - 1, 1))
    lim = min(half_y, half_x)
    if rmax > lim:
        c *= lim / rmax * 0.999
    m = np.arange(J, dtype=np.float64)
    r = c * np.sqrt(m)
    th = np.deg2rad(_GOLDEN_ANGLE_DEG) * m
    y = half_y + r * np.sin(th)
    x = half_x + r * np.cos(th)
    pos = np.stack([np.rint(y), np.rint(x)], axis=1)
    pos[:, 0] = np.clip(pos[:, 0], 0, Ho - N)
    pos[:, 1] = np.clip(pos[:, 1], 0, Wo - N)
    pos = pos.astype(np.int32)
    if J > 1:
        sub = pos[: min(J, 2000)].astype(np.float64)
        d2 = ((sub[:, None, :] - sub[None, :, :]) ** 2).sum(-1)
        np.fill_diagonal(d2, np.inf)
        nn = float(np.sqrt(d2.min(axis=1)).mean())
    else:
        nn = 0.0
    return pos, nn


def smooth_random_object(Ho: int, Wo: int, rng: np.random.Generator, sigma: float = 3.0,
                         amp_range=(0.8, 1.0), phase_range=(-math.pi / 2, math.pi / 2)):
    """Complex object: amplitude and phase drawn uniform, smoothed by a periodic
    Gaussian of width ``sigma`` px, then rescaled linearly to the stated ranges."""

    def field_(lo, hi):
        u = rng.uniform(lo, hi, size=(Ho, Wo))
        s = scipy.ndimage.gaussian_filter(u, sigma, mode="wrap")
        smin, smax = s.min(), s.max()
        return lo + (hi - lo) * (s - smin) / max(smax - smin, 1e-300)

    amp = field_(*amp_range)
    ph = field_(*phase_range)
    return amp * np.exp(1j * ph)


def disk_probe(N: int, radius: float, phase_coef: float):
    """Disk aperture of ``radius`` px centred at (N/2, N/2) with phase
    ``phase_coef * r^2`` (r in px from the centre).  Unit amplitude inside."""
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    r2 = (yy - N / 2) ** 2 + (xx - N / 2) ** 2
    amp = (r2 <= radius * radius).astype(np.float64)
    return amp * np.exp(1j * phase_coef * r2)


def hermite_gauss_modes(N: int, K: int, waist: float, phase_coef: float, powers):
    """K Hermite-Gauss-shaped modes (HG00, HG10, HG01, HG11, ...) times a
    quadratic phase, Gram-Schmidt orthogonalised, then scaled so that the
    fraction of the total power in mode k is ``powers[k]``."""
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    y = (yy - N / 2) / waist
    x = (xx - N / 2) / waist
    g = np.exp(-(x * x + y * y)) * np.exp(1j * phase_coef * ((yy - N / 2) ** 2 + (xx - N / 2) ** 2))
    orders = [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 2), (2, 1), (1, 2), (2, 2), (3, 0)]
    herm = [lambda t: np.ones_like(t), lambda t: 2 * t, lambda t: 4 * t * t - 2, lambda t: 8 * t ** 3 - 12 * t]
    modes = []
    for k in range(K):
        ny, nx = orders[k]
        m = g * herm[ny](y) * herm[nx](x)
        for q in modes:
            m = m - np.vdot(q, m) * q
        m = m / np.sqrt(np.vdot(m, m).real)
        modes.append(m)
    p = np.asarray(powers, dtype=np.float64)
    p = p / p.sum()
    return np.stack([np.sqrt(p[k]) * modes[k] for k in range(K)])


def detector_gap_mask(N: int, fraction: float = 0.02, band: int = 4):
    """Bad-pixel mask shaped like detector gaps: a horizontal band ``band`` px
    high across the detector plus a vertical band of the same width, cut so
    that about ``fraction`` of the pixels are masked.  Built in centred
    detector coordinates, returned in FFT order (uint8, 1 = masked)."""
    m = np.zeros((N, N), dtype=np.uint8)
    if fraction <= 0:
        return m
    target = int(round(fraction * N * N))
    r0 = N // 2 + N // 8
    m[r0:r0 + band, :] = 1
    left = target - int(m.sum())
    if left > 0:
        c0 = N // 2 - N // 5
        h = min(N, (left + band - 1) // band)
        m[:h, c0:c0 + band] = 1
    return np.fft.ifftshift(m)


def _blur_complex(p: np.ndarray, sigma: float):
    if sigma <= 0:
        return p.copy()
    out = np.empty_like(p)
    for k in range(p.shape[0]):
        out[k] = (scipy.ndimage.gaussian_filter(p[k].real, sigma, mode="wrap")
                  + 1j * scipy.ndimage.gaussian_filter(p[k].imag, sigma, mode="wrap"))
    return out


def _workers():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _frame_intensities(obj, probe, positions, lo, hi, nearfield=0.0):
    """Noise-free detector intensities for frames lo..hi-1: sum_k |FT(P_k O[r_j])|^2
    in the far field; in the near field sum_k of |the wave after a Fresnel
    propagation over lambda z = nearfield * pixel^2|^2, the propagation being
    done in Fourier space with the paraxial transfer exp(-i pi lambda z q^2)."""
    N = probe.shape[-1]
    n = hi - lo
    out = np.zeros((n, N, N), dtype=np.float64)
    if nearfield:
        k = np.fft.fftfreq(N) * N
        transfer = np.exp(-1j * np.pi * nearfield * (k[:, None] ** 2 + k[None, :] ** 2) / N ** 2)
    for i in range(n):
        r, c = positions[lo + i]
        patch = obj[r:r + N, c:c + N]
        w = probe * patch[None]
        f = scipy.fft.fft2(w, norm="ortho", workers=_workers())
        if nearfield:
            f = scipy.fft.ifft2(f * transfer, norm="ortho", workers=_workers())
        out[i] = (f.real ** 2 + f.imag ** 2).sum(0)
    return out


def make_scan(name: str, N: int, J: int, Ho: int, Wo: int, *, K: int = 1, seed: int,
              photons: float, step: float, probe: str = "disk", probe_radius: float | None = None,
              phase_coef: float | None = None, mode_powers=None, mask_fraction: float = 0.0,
              noise: bool = True, probe0_blur: float = 2.0, algorithm: str = "AP",
              cycles: int = 20, chunk: int = 256, nearfield: float = 0.0,
              diffuser_phase: float = 0.0) -> Scan:
    """Draw one seeded scan.  The probe is scaled so that the mean total model
    intensity per frame equals ``photons`` before Poisson sampling; hence the
    noise-free intensities equal the model of (obj_true, probe_true) exactly."""
    ss = np.random.SeedSequence(seed)
    s_obj, s_noise = ss.spawn(2)
    rng = np.random.default_rng(s_obj)
    obj = smooth_random_object(Ho, Wo, rng)
    if probe_radius is None:
        probe_radius = N * 12.0 / 64.0
    if phase_coef is None:
        # same edge phase gradient (0.48 rad/px) as the 64x64, r=12 px, 0.02 r^2 probe
        phase_coef = 0.24 / probe_radius
    if probe == "disk":
        P = disk_probe(N, probe_radius, phase_coef)[None]
        if diffuser_phase:
            # a diffuser in the beam: smooth random phase of about +-diffuser_phase rad
            d = scipy.ndimage.gaussian_filter(rng.standard_normal((N, N)), 4.0, mode="wrap")
            P = P * np.exp(1j * diffuser_phase * d / max(np.abs(d).max(), 1e-300))
        if K > 1:
            raise ValueError("disk probe is single-mode; use probe='hg' for K > 1")
    elif probe == "hg":
        P = hermite_gauss_modes(N, K, probe_radius, phase_coef, mode_powers or [1.0] * K)
    else:
        raise ValueError(probe)
    positions, nn = fermat_spiral(J, step, Ho, Wo, N)
    # photon scaling from a sample of frames (all of them when J is small)
    sample = np.linspace(0, J - 1, num=min(J, 64)).astype(np.int64)
    tot = np.array([_frame_intensities(obj, P, positions[i:i + 1], 0, 1, nearfield)[0].sum() for i in sample])
    P = P * math.sqrt(photons / tot.mean())
    mask = detector_gap_mask(N, mask_fraction)
    iobs = np.empty((J, N, N), dtype=np.float32)
    chunk_seeds = s_noise.spawn((J + chunk - 1) // chunk)
    for ci, lo in enumerate(range(0, J, chunk)):
        hi = min(J, lo + chunk)
        lam = _frame_intensities(obj, P, positions, lo, hi, nearfield)
        if noise:
            crng = np.random.default_rng(chunk_seeds[ci])
            iobs[lo:hi] = crng.poisson(lam).astype(np.float32)
        else:
            iobs[lo:hi] = lam.astype(np.float32)
    iobs[:, mask.astype(bool)] = 0.0
    obj0 = np.ones((Ho, Wo), dtype=np.complex64)
    probe0 = _blur_complex(P, probe0_blur).astype(np.complex64)
    return Scan(name=name, N=N, K=K, J=J, Ho=Ho, Wo=Wo, positions=positions, iobs=iobs,
                mask=mask, obj_true=obj, probe_true=P, obj0=obj0, probe0=probe0,
                photons=photons, seed=seed, step_px=nn, algorithm=algorithm, cycles=cycles,
                nearfield=nearfield)


# Workload recipes.  Each stands in for one of the paper's workload shapes
# (far-field, 256^2 / 512^2 frames, 1 or 3 probe modes, Table 1 and Fig. 7).
CONFIGS = {
    # plain AP parity case: 64^2 probe, 256^2 object, 100 positions, 1e5 photons, 20 cycles
    "ap64": dict(N=64, J=100, Ho=256, Wo=256, K=1, seed=1, photons=1e5, step=20.0,
                 probe_radius=12.0, phase_coef=0.02, mask_fraction=0.0, algorithm="AP", cycles=20),
    # DM headline: 256^2 frames, 2048^2 object, 4000 positions, 1e6 photons, 2 % gap mask
    "dm256": dict(N=256, J=4000, Ho=2048, Wo=2048, K=1, seed=2, photons=1e6, step=40.0,
                  probe_radius=40.0, mask_fraction=0.02, algorithm="DM", cycles=100),
    # ML gradient workload: 256^2 frames, 1536^2 object, 1000 positions, 1e5 photons
    "ml256": dict(N=256, J=1000, Ho=1536, Wo=1536, K=1, seed=4, photons=1e5, step=40.0,
                  probe_radius=40.0, mask_fraction=0.0, algorithm="ML", cycles=50),
    # finite-difference copy: 32^2 frames, 16 positions
    "ml32fd": dict(N=32, J=16, Ho=64, Wo=64, K=1, seed=4, photons=1e5, step=6.0,
                   probe_radius=6.0, mask_fraction=0.0, algorithm="ML", cycles=50),
    # near field (Table 1's near-field row, 1 probe): 256^2 frames of a diffuser-modulated
    # beam, Fresnel propagation factor lambda z / pixel^2 = 200, 1e8 photons per frame
    "nf256": dict(N=256, J=64, Ho=640, Wo=640, K=1, seed=6, photons=1e8, step=30.0,
                  probe_radius=90.0, phase_coef=0.0, diffuser_phase=2.0, mask_fraction=0.02,
                  nearfield=200.0, algorithm="DM", cycles=100),
    # large multi-mode DM: 3 Hermite-Gauss modes 512^2, 6000^2 object, 10000 positions, 1e7 photons
    "modes512": dict(N=512, J=10000, Ho=6000, Wo=6000, K=3, seed=5, photons=1e7, step=60.0,
                     probe="hg", probe_radius=51.2, mode_powers=[0.7, 0.2, 0.1],
                     mask_fraction=0.0, algorithm="DM", cycles=100),
}


def make_config(name: str, *, J: int | None = None, Ho: int | None = None, Wo: int | None = None,
                noise: bool = True, **over) -> Scan:
    """Build a named workload; ``J``/``Ho``/``Wo`` override the sizes (to make a
    subset that the FP64 oracle finishes quickly)."""
    spec = dict(CONFIGS[name])
    spec.update(over)
    if J is not None:
        spec["J"] = J
    if Ho is not None:
        spec["Ho"] = Ho
    if Wo is not None:
        spec["Wo"] = Wo
    return make_scan(name, noise=noise, **spec)


def batched_problem_specs(seed: int = 3, nprob: int = 16, sizes=(128, 192, 256, 384, 512),
                          jmin: int = 200, jmax: int = 3000, border: int = 64,
                          photons_range=(1e4, 1e6), j_scale: float = 1.0):
    """Parameters of the batched workload: ``nprob`` independent scans with
    frame sizes drawn from ``sizes``, J ~ U[jmin, jmax] positions, objects sized
    to cover the scan plus a ``border`` px margin on each side, photons
    log-uniform in ``photons_range``, AP and DM alternately.  ``j_scale``
    shrinks every J (for subsets the oracle can run)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nprob):
        N = int(rng.choice(sizes))
        J = int(rng.integers(jmin, jmax + 1))
        J = max(2, int(round(J * j_scale)))
        logp = rng.uniform(math.log10(photons_range[0]), math.log10(photons_range[1]))
        step = 0.1 * N
        c = step / math.sqrt(math.pi)
        extent = 2 * c * math.sqrt(max(J - 1, 1))
        H = int(math.ceil(extent)) + N + 2 * border
        H += (-H) % 4
        out.append(dict(name=f"batched{i}", N=N, J=J, Ho=H, Wo=H, K=1, seed=seed * 1000 + i,
                        photons=float(10 ** logp), step=step, probe_radius=N * 40.0 / 256.0,
                        mask_fraction=0.0, algorithm="AP" if i % 2 == 0 else "DM", cycles=50))
    return out
