"""Long-run parity of the DM cycle on a noisy, headline-shaped case (GPU).

A subset of the 256^2 DM workload (100 frames of the spiral, 640^2 object,
1e6 photons, 2 % detector-gap mask, Poisson noise) runs 100 DM cycles on the
GPU from the FP64 oracle's state after one AP cycle, beside the oracle itself
and an independent single-precision evaluation (SciPy complex64 transforms and
projection, the oracle's overlap update).  At cycles 1, 10, 25, 50 and 100 the
relative L2 distance to FP64 of the object (illuminated region), the probe and
the per-cycle LLK is measured for both single-precision evaluations.  The
GPU side runs twice: the FP32 path, and the BF16 hi + mid + lo split-precision
form with every DFT stage on the tensor cores (an FP32-accurate form).

DM on noisy data does not converge to a fixed point and its trajectory
amplifies rounding differences: on this case both single-precision
evaluations stay near FP64 for ten cycles (about 2e-5) and then leave it
together (about 1.5e-2 at cycle 25, 0.15 at cycle 50, 0.4 - 1.3 at cycle 100),
so no single-precision evaluation meets 1e-4 after 100 noisy cycles.  The test
requires 1e-5 after the first cycle; 1e-4 for every quantity at the
checkpoints where the complex64 object and probe are still within 1e-4 of FP64;
after that divergence, an object and probe distance at most RATIO = 2 times
the complex64 evaluation's, and an LLK distance at most LLK_RATIO = 10 times
it (one scalar drawn from a chaotic trajectory varies more between
evaluations than the state does).
"""
import numpy as np
import pytest
import scipy.fft

import oracle
from synthetic import make_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL1, TOL100, RATIO, LLK_RATIO = 1e-5, 1e-4, 2.0, 10.0
CHECK = (1, 10, 25, 50, 100)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2008_11511_gb300 import build as b
    b.build()


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _dm_complex64(obj, probe, psi, data, init):
    """One DM cycle with the transforms and the projection in complex64 (SciPy)
    and the oracle's overlap update: an independent single-precision evaluation."""
    N = probe.shape[-1]
    o32, p32 = obj.astype(np.complex64), probe.astype(np.complex64)
    phi = np.stack([p32 * o32[r:r + N, c:c + N][None] for r, c in data.positions])
    if init:
        psi = phi.copy()
    X = scipy.fft.fft2(2 * phi - psi, norm="ortho", axes=(-2, -1))
    ic = (np.abs(X) ** 2).sum(1)
    sc = np.where(data.mask, 1.0, np.sqrt(np.maximum(data.iobs, 0)) / np.maximum(np.sqrt(ic), 1e-20))
    psi = (psi + scipy.fft.ifft2(X * sc[:, None].astype(np.float32), norm="ortho", axes=(-2, -1)) - phi)
    psi = psi.astype(np.complex64)
    llk = oracle.llk_poisson(ic.astype(np.float64), data.iobs, data.mask)
    o, p = oracle.overlap_update(o32.astype(complex), p32.astype(complex), psi.astype(complex), data.positions)
    return o.astype(np.complex64), p.astype(np.complex64), psi, llk


@pytest.fixture(scope="module")
def trajectory():
    """The case and its FP64 and complex64 trajectories at the checkpoints
    (computed once for the number formats tested below)."""
    s = make_config("dm256", J=100, Ho=640, Wo=640)
    data = oracle.Data.make(s.iobs, s.positions, s.mask)
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    o64, p64, psi64 = o0.astype(complex), p0.astype(complex), None
    o32, p32, psi32 = o0, p0, None
    ref = {}
    for c in range(1, 101):
        o64, p64, psi64, l64 = oracle.dm_cycle(o64, p64, psi64, data, init_psi=(c == 1))
        o32, p32, psi32, l32 = _dm_complex64(o32, p32, psi32, data, c == 1)
        if c in CHECK:
            d = oracle.object_denominator(p64, s.positions, (s.Ho, s.Wo))
            ill = d > 1e-3 * d.max()
            ref[c] = dict(o64=o64.copy(), p64=p64.copy(), l64=l64, ill=ill,
                          c64=(rel(o32[ill], o64[ill]), rel(p32, p64), abs(l32 - l64) / abs(l64)))
    return s, o0, p0, ref


@pytest.mark.parametrize("form,tc_rows", [(0, 0), (2, 1)], ids=["fp32", "bf16x3_every_stage"])
def test_dm256_subset_100_noisy_cycles_against_fp64(trajectory, form, tc_rows):
    """The FP32 path, and the BF16 hi + mid + lo form with every DFT stage on
    the tensor cores, against the bounds stated at the top of this file."""
    from paper_2008_11511_gb300 import Ptycho
    s, o0, p0, ref = trajectory
    dev = torch.device("cuda")
    pb = Ptycho(torch.tensor(o0, device=dev), torch.tensor(p0, device=dev), torch.tensor(s.iobs, device=dev),
                s.positions, s.mask, with_psi=True)
    pb.set_param("tc", form)
    pb.set_param("tc_rows", tc_rows)
    done = 0
    rows = []
    for c in CHECK:
        lg = pb.dm(c - done, init_psi=(done == 0)).cpu().numpy()[-1]
        done = c
        r = ref[c]
        ill = r["ill"]
        og, pg = pb.obj.cpu().numpy(), pb.probe.cpu().numpy()
        row = {"cycle": c, "gpu": (rel(og[ill], r["o64"][ill]), rel(pg, r["p64"]), abs(lg - r["l64"]) / abs(r["l64"])),
               "c64": r["c64"]}
        rows.append(row)
        print(f"dm256 subset [{form}, {tc_rows}] cycle {c:3d}: gpu obj {row['gpu'][0]:.2e} probe {row['gpu'][1]:.2e} "
              f"llk {row['gpu'][2]:.2e} | complex64 obj {row['c64'][0]:.2e} probe {row['c64'][1]:.2e} "
              f"llk {row['c64'][2]:.2e}")
    pb.close()
    import json
    import os
    out = os.environ.get("LONGRUN_JSON")
    if out:
        json.dump(rows, open(f"{out}.{form}{tc_rows}", "w"), default=float)
    assert max(rows[0]["gpu"]) < TOL1, rows[0]
    for row in rows:
        if max(row["c64"][:2]) < TOL100:  # before the trajectories diverge
            assert max(row["gpu"]) < TOL100, row
        else:
            assert row["gpu"][0] <= RATIO * row["c64"][0] and row["gpu"][1] <= RATIO * row["c64"][1], row
            assert row["gpu"][2] <= max(TOL100, LLK_RATIO * row["c64"][2]), row
