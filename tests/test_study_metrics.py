"""Host-side metrics of the accuracy study (SNR in dB, SSIM) - CPU only.

SSIM is pinned by its closed form on constant images, by a brute-force evaluation of
the windowed statistics, and by its identities; SNR by its definition's special values.
"""
import math

import numpy as np
import pytest

from paper_2005_13471_gb300 import study


def test_snr_special_values():
    t = np.random.default_rng(0).standard_normal((16, 16))
    assert study.snr_db(t, t) == math.inf
    assert study.snr_db(t, np.zeros_like(t)) == pytest.approx(0.0, abs=1e-12)
    e = np.random.default_rng(1).standard_normal(t.shape)
    e *= 0.1 * np.linalg.norm(t) / np.linalg.norm(e)
    assert study.snr_db(t, t + e) == pytest.approx(20.0, abs=1e-9)


def test_ssim_identity_and_symmetry():
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal((24, 24)), rng.standard_normal((24, 24))
    assert study.ssim(a, a) == pytest.approx(1.0, abs=1e-12)
    assert study.ssim(a, b, data_range=3.0) == pytest.approx(study.ssim(b, a, data_range=3.0), abs=1e-14)
    assert study.ssim(a, b) < 0.5


def test_ssim_constant_images_closed_form():
    # zero local variances: SSIM = (2 u v + C1) / (u^2 + v^2 + C1)
    u, v, L = 0.7, 0.2, 1.0
    c1 = (0.01 * L) ** 2
    got = study.ssim(np.full((20, 20), u), np.full((20, 20), v), data_range=L)
    assert got == pytest.approx((2 * u * v + c1) / (u * u + v * v + c1), rel=1e-12)


def test_ssim_brute_force_windows():
    rng = np.random.default_rng(3)
    a = rng.uniform(0, 1, (15, 14))
    b = a + 0.2 * rng.standard_normal(a.shape)
    L = float(a.max() - a.min())
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    k = np.arange(-5, 6)
    w1 = np.exp(-0.5 * (k / 1.5) ** 2)
    W = np.outer(w1, w1) / np.outer(w1, w1).sum()
    vals = []
    for i in range(5, a.shape[0] - 5):
        for j in range(5, a.shape[1] - 5):
            pa, pb = a[i - 5:i + 6, j - 5:j + 6], b[i - 5:i + 6, j - 5:j + 6]
            ma, mb = np.sum(W * pa), np.sum(W * pb)
            va, vb = np.sum(W * pa * pa) - ma * ma, np.sum(W * pb * pb) - mb * mb
            cab = np.sum(W * pa * pb) - ma * mb
            vals.append((2 * ma * mb + c1) * (2 * cab + c2) / ((ma * ma + mb * mb + c1) * (va + vb + c2)))
    assert study.ssim(a, b) == pytest.approx(float(np.mean(vals)), rel=1e-12)


def test_detector_covers_image():
    for N, lam, z in ((64, 0.25, 1.0), (256, 2.0, 0.0), (100, 1.0, 1.0)):
        M = study.detector_bins(N, lam, z)
        assert (M - 1) / 2 * lam >= N / math.sqrt(2.0) + 1.0 + z / 2
