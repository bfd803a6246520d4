"""Checks on the synthetic input generators (not the method)."""
import math

import numpy as np

from workloads import configs, ellipse_params, ellipse_sinogram, poisson_log_sinogram


def test_params_seeded_and_in_range():
    p1 = ellipse_params(512, 40, seed=3)
    p2 = ellipse_params(512, 40, seed=3)
    assert np.array_equal(p1, p2)
    assert np.all(np.abs(p1[:, :2]) <= 0.8 * 256)
    assert np.all((p1[:, 2:4] >= 2) & (p1[:, 2:4] <= 20))
    assert np.all((p1[:, 5] >= -0.5) & (p1[:, 5] <= 1.0))


def test_ellipse_projection_mass():
    # every view integrates to the phantom mass sum rho * pi * a * b
    p = ellipse_params(64, 3, seed=1)
    angles = np.array([0.0, 0.21, 0.5])
    lam = 0.05
    M = int(140 / lam)
    for zeta in (0.0, 1.0):
        s = ellipse_sinogram(p, angles, M, lam, zeta)
        mass = np.sum(p[:, 5] * math.pi * p[:, 2] * p[:, 3])
        assert np.max(np.abs(s.sum(axis=1) * lam - mass)) < 1e-3 * abs(mass) + 1e-3


def test_poisson_noise_unbiased_in_the_mean():
    s = np.full((4, 200), 3.0)
    g = poisson_log_sinogram(s, 1e5, seed=0)
    assert abs(g.mean() - 3.0) < 0.01 and g.std() > 0


def test_batch_slices():
    sl = configs.batch_slices(16, seed=0)
    assert len(sl) == 16 and all(s["N"] in configs.BATCH_SIZES_N for s in sl)
