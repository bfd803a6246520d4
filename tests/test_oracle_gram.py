"""Pins for the oracle's Gram filter and Gram apply (Sec. 4) - CPU only."""
import math

import numpy as np
import pytest

from oracle import boxspline as bs
from oracle import gram
from oracle.geometry import cospi_sinpi, pixel_projections, uniform_angles


def test_single_view_axis_aligned_filter():
    # theta = 0: G[d] = A(d1) for every d2; delta without blur, [1/6, 2/3, 1/6] with zeta = 1
    N = 5
    G0 = gram.gram_taps(N, np.array([0.0]), 0.0)
    assert np.allclose(G0[:, N - 1], 1.0) and np.allclose(np.delete(G0, N - 1, axis=1), 0.0)
    G1 = gram.gram_taps(N, np.array([0.0]), 1.0)
    row = G1[3, N - 3:N + 2]
    assert np.max(np.abs(row - np.array([0, 1 / 6, 2 / 3, 1 / 6, 0]))) < 1e-15
    # theta = pi/2: same along the other axis
    G2 = gram.gram_taps(N, np.array([0.5]), 1.0)
    assert np.max(np.abs(G2.T - G1)) < 1e-15


def test_single_view_45_degrees():
    # theta = pi/4: G[d] = sqrt(2) beta_3(d1 + d2)
    N = 4
    G = gram.gram_taps(N, np.array([0.25]), 0.0)
    d = np.arange(-(N - 1), N)
    D = d[None, :] + d[:, None]
    beta3 = np.where(np.abs(D) < 1, 2 / 3 - D ** 2 + np.abs(D) ** 3 / 2,
                     np.where(np.abs(D) < 2, (2 - np.abs(D)) ** 3 / 6, 0.0))
    assert np.max(np.abs(G - math.sqrt(2) * beta3)) < 1e-14


def test_centre_tap_sum():
    angles = uniform_angles(4)
    G = gram.gram_taps(6, angles, 0.0)
    c, s = cospi_sinpi(angles)
    mx, mn = np.maximum(np.abs(c), np.abs(s)), np.minimum(np.abs(c), np.abs(s))
    assert abs(G[5, 5] - np.sum(1 / mx - mn / (3 * mx ** 2))) < 1e-14
    assert abs(G[5, 5] - 3.8856180831641267) < 1e-12  # sum over 0, 45, 90, 135 degrees


@pytest.mark.parametrize("zeta", [0.0, 1.0])
def test_symmetries(zeta):
    N = 9
    G = gram.gram_taps(N, uniform_angles(12), zeta)
    assert np.max(np.abs(G - G[::-1, ::-1])) < 1e-15        # G[d] = G[-d]
    assert np.max(np.abs(G - G[::-1, :])) < 1e-14           # uniform angles: mirror in d2
    assert np.max(np.abs(G - G.T)) < 1e-14                   # and swap of axes (n multiple of 4)


@pytest.mark.parametrize("zeta", [0.0, 1.0])
def test_quadrature_equals_truncated_power_well_conditioned(zeta):
    # two independent evaluations of the same taps: exact quadrature vs Sec. 4 box spline
    angles = np.array([0.11, 0.19, 0.3, 0.37, 0.62, 0.8])
    Gq = gram.gram_taps(8, angles, zeta, method="quadrature")
    Gb = gram.gram_taps(8, angles, zeta, method="boxspline")
    assert np.max(np.abs(Gq - Gb)) < 1e-12


@pytest.mark.parametrize("zeta", [0.0, 1.0])
def test_explicit_HtH_is_toeplitz_and_equals_filter(zeta):
    # Sec. 4 closing remark: the N^2 x N^2 Gram matrix is a (2N-1)^2 filter
    N = 4
    angles = np.array([0.0, 0.13, 0.25, 0.5, 0.71])
    Gm = gram.explicit_gram_matrix(N, angles, zeta)
    G = gram.gram_taps(N, angles, zeta)
    for i in range(N * N):
        i2, i1 = divmod(i, N)
        for j in range(N * N):
            j2, j1 = divmod(j, N)
            assert abs(Gm[i, j] - G[i2 - j2 + N - 1, i1 - j1 + N - 1]) < 1e-14
    assert np.max(np.abs(Gm - Gm.T)) < 1e-15


@pytest.mark.parametrize("N,zeta", [(8, 0.0), (13, 1.0), (32, 1.0)])
def test_fft_apply_equals_direct(N, zeta):
    rng = np.random.default_rng(N)
    G = gram.gram_taps(N, uniform_angles(10), zeta)
    x = rng.standard_normal((N, N))
    yd = gram.gram_apply_direct(G, x)
    yf = gram.gram_apply_fft(G, x)
    assert np.linalg.norm(yd - yf) / np.linalg.norm(yd) < 1e-14
    pts = [(0, 0), (N - 1, N - 1), (N // 2, 3), (1, N - 2)]
    assert np.max(np.abs(gram.gram_apply_sampled(G, x, pts) - np.array([yd[p] for p in pts]))) < 1e-12


def test_direct_apply_brute_force():
    # against the explicit matrix-vector product on a tiny grid
    N = 4
    angles = np.array([0.05, 0.3, 0.55])
    Gm = gram.explicit_gram_matrix(N, angles, 1.0)
    G = gram.gram_taps(N, angles, 1.0)
    x = np.random.default_rng(1).standard_normal((N, N))
    assert np.max(np.abs(gram.gram_apply_direct(G, x).reshape(-1) - Gm @ x.reshape(-1))) < 1e-13


def test_psd_restricted_operator_and_projection_energy():
    # x^T G x = sum_theta ||P_theta f_x||^2 >= 0 (energy of the projections)
    N = 6
    angles = np.array([0.07, 0.33, 0.58])
    G = gram.gram_taps(N, angles, 0.0)
    x = np.random.default_rng(3).standard_normal((N, N))
    quad = float(np.sum(x * gram.gram_apply_direct(G, x)))
    energy = 0.0
    for th in angles:
        c, s = cospi_sinpi(th)
        t = pixel_projections(N, c, s).reshape(-1)
        bp = bs.footprint_breakpoints(c, s, 0.0)
        edges = np.unique(np.concatenate([bp + tk for tk in t]))[None, :]
        f = lambda y: (bs.pixel_projection(y[..., None] - t, c, s) @ x.reshape(-1)) ** 2
        energy += bs.gl3_integrate(edges, f)[0]
    assert quad > 0 and abs(quad - energy) < 1e-12 * energy


def test_spectrum_real_and_reported_sign():
    # the circulant embedding's spectrum is real (G[d] = G[-d]); dense angle sets keep it >= 0
    G = gram.gram_taps(16, uniform_angles(90), 0.0)
    re, im = gram.gram_spectrum(G)
    assert np.max(np.abs(im)) <= 1e-12 * np.max(re)
    assert np.min(re) / np.max(re) > 0
    G1 = gram.gram_taps(8, np.array([0.1]), 0.0)
    re1, _ = gram.gram_spectrum(G1)
    assert np.min(re1) < 0  # not PSD for a single view: the embedding is not the operator


def test_sampled_taps_match_the_full_filter():
    # the per-offset evaluation used by the large-N GPU checks against the full filter
    N = 12
    angles = np.array([0.0, 0.11, 0.25, 0.47, 0.5, 0.73])
    rng = np.random.default_rng(21)
    offs = [(int(a), int(b)) for a, b in rng.integers(-(N - 1), N, (15, 2))] + [(0, 0), (N - 1, -(N - 1))]
    for zeta in (0.0, 1.0):
        for method in ("quadrature", "boxspline"):
            G = gram.gram_taps(N, angles, zeta, method)
            vals = gram.gram_tap_values(offs, angles, zeta, method)
            ref = np.array([G[d2 + N - 1, d1 + N - 1] for d1, d2 in offs])
            assert np.max(np.abs(vals - ref)) < 1e-14 * np.max(np.abs(G))
