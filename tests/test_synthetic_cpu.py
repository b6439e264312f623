"""The seeded input generator (synthetic/): deterministic, shaped like the
paper's workloads as stated for each configuration, and holding none of the
method's arithmetic beyond the forward model used once to draw the data."""
import numpy as np

from synthetic import batched_problem_specs, make_config, make_scan
from synthetic.scans import detector_gap_mask, fermat_spiral, hermite_gauss_modes


def test_same_seed_same_scan_and_different_seed_differs():
    a = make_config("ap64", J=20)
    b = make_config("ap64", J=20)
    assert np.array_equal(a.iobs, b.iobs) and np.array_equal(a.positions, b.positions)
    assert np.array_equal(a.obj0, b.obj0) and np.array_equal(a.probe0, b.probe0)
    c = make_scan("ap64", N=64, J=20, Ho=256, Wo=256, seed=2, photons=1e5, step=20.0)
    assert not np.array_equal(a.iobs, c.iobs)


def test_shapes_types_and_positions_inside_the_object():
    s = make_config("ml32fd")
    assert s.iobs.shape == (s.J, s.N, s.N) and s.iobs.dtype == np.float32
    assert s.probe0.shape == (s.K, s.N, s.N) and s.probe0.dtype == np.complex64
    assert s.obj0.shape == (s.Ho, s.Wo) and s.obj0.dtype == np.complex64
    assert s.positions.dtype == np.int32 and s.positions.shape == (s.J, 2)
    assert s.positions.min() >= 0
    assert s.positions[:, 0].max() <= s.Ho - s.N and s.positions[:, 1].max() <= s.Wo - s.N


def test_photon_scaling_and_poisson_counts():
    """The probe is scaled so the mean model intensity per frame is the photon
    count; the noisy intensities are integer counts with that mean."""
    s = make_config("ap64")
    per_frame = s.iobs.reshape(s.J, -1).sum(axis=1)
    assert abs(per_frame.mean() / s.photons - 1.0) < 0.01
    assert np.array_equal(s.iobs, np.rint(s.iobs)) and s.iobs.min() >= 0


def test_fermat_spiral_fits_and_steps():
    pos, step = fermat_spiral(100, 20.0, 256, 256, 64)
    pos = np.asarray(pos)
    assert pos.shape == (100, 2)
    assert pos.min() >= 0 and pos.max() <= 256 - 64
    assert 5.0 < step <= 20.0 * 1.05


def test_detector_gap_mask_fraction_and_bands():
    m = detector_gap_mask(256, fraction=0.02, band=4)
    assert m.shape == (256, 256)
    assert 0.01 < m.mean() < 0.04


def test_hermite_gauss_modes_are_orthogonal_with_the_given_powers():
    P = hermite_gauss_modes(64, 3, waist=8.0, phase_coef=0.0, powers=[0.7, 0.2, 0.1])
    g = np.einsum("kxy,lxy->kl", np.conj(P), P)
    off = g - np.diag(np.diag(g))
    assert np.abs(off).max() < 1e-8 * np.abs(np.diag(g)).max()
    w = np.real(np.diag(g)) / np.real(np.trace(g))
    assert np.allclose(w, [0.7, 0.2, 0.1], atol=1e-6)


def test_batched_specs_match_the_stated_recipe():
    sp = batched_problem_specs()
    assert len(sp) == 16
    assert {x["N"] for x in sp} <= {128, 192, 256, 384, 512}
    assert all(200 <= x["J"] <= 3000 for x in sp)
    assert [x["algorithm"] for x in sp] == ["AP", "DM"] * 8
    assert all(1e4 <= x["photons"] <= 1e6 for x in sp)
