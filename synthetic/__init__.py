"""Seeded synthetic far-field ptychography scans.

This package is the one input source shared by the FP64 oracle (``oracle/``)
and the CUDA path (``paper_2008_11511_gb300``).  It simulates measured data the
way the paper's "functions to simulate data" feature does (Section 4 feature
list): a smooth random complex object, a disk probe with a quadratic phase,
Fermat-spiral scan positions, a detector-gap mask and Poisson-noised
far-field intensities.  It holds none of the reconstruction arithmetic
(no amplitude projection, log-likelihood, overlap update or normalisation).
"""
from .scans import (  # noqa: F401
    Scan,
    CONFIGS,
    make_scan,
    make_config,
    fermat_spiral,
    detector_gap_mask,
    smooth_random_object,
    disk_probe,
    hermite_gauss_modes,
    batched_problem_specs,
)
