"""Pins for the oracle's correction filter, interpolation and back projection (Sec. 5)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import backproject as bp
from oracle import boxspline as bs
from oracle import gram
from oracle.geometry import bin_centres, cospi_sinpi, interp_degree, pixel_projections

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def test_q40_printed_value():
    # Sec. 5 prints q[40] = 3.38e-31 for the degree-2 correction filter
    gold = json.load(open(GOLDEN))["q40_degree2"]
    q = bp.correction_filter(2)
    assert abs(q[80] - gold["value"]) <= gold["relative_tolerance"] * gold["value"]
    assert q[80] == q[0]
    # the formula as printed, without sqrt(2), does not give the printed value
    assert abs((2 * math.sqrt(2) - 3) ** 40 - gold["value"]) > 0.2 * gold["value"]


def test_correction_filter_inverts_sampled_bspline():
    # Eq. 5: q * b = delta with b[m] = beta_2(m) = [1/8, 3/4, 1/8]
    q = bp.correction_filter(2)
    full = np.convolve(q, [bs.bspline(-1, 2), bs.bspline(0, 2), bs.bspline(1, 2)])
    mid = full[1:-1]
    e = np.zeros_like(mid)
    e[40] = 1.0
    assert np.max(np.abs(mid - e)) < 1e-15
    assert np.all(bp.correction_filter(1) == bp.correction_filter(0))
    assert bp.correction_filter(1)[40] == 1.0 and bp.correction_filter(1).sum() == 1.0


def test_interpolant_reproduces_samples():
    # the oblique interpolant with the correction filter passes through the samples
    rng = np.random.default_rng(0)
    g = rng.standard_normal(50)
    lam = 0.7
    ym = bin_centres(50, lam)
    for d in (0, 1, 2):
        c = np.convolve(g, bp.correction_filter(d))[40:90]
        val = bp.interpolant(c, ym[10:40], lam, d)
        assert np.max(np.abs(val - g[10:40])) < 1e-12


@pytest.mark.parametrize("zeta", [0.0, 1.0])
def test_exact_recovery_axis_aligned(zeta):
    # Sec. 5: with views {0, pi/2}, even N and M, lambda_y = 1, sampling points include
    # every k_theta, so H^T g_hat = G c exactly
    N, M = 6, 10
    angles = np.array([0.0, 0.5])
    c = np.random.default_rng(5).standard_normal((N, N))
    sino = bp.forward_sample(c, angles, M, 1.0, zeta)
    b = bp.backproject(sino, N, angles, 1.0, zeta)
    Gc = gram.gram_apply_direct(gram.gram_taps(N, angles, zeta), c)
    assert np.max(np.abs(b - Gc)) < 1e-13


@pytest.mark.parametrize("zeta,lam", [(0.0, 1.0), (1.0, 1.0), (1.0, 0.6), (0.0, 1.7)])
def test_quadrature_equals_box_spline_closed_form(zeta, lam):
    N, M = 7, 13
    angles = np.array([0.0, 0.12, 0.27, 0.5, 0.66, 0.9])
    sino = np.random.default_rng(2).standard_normal((len(angles), M))
    b_q = bp.backproject(sino, N, angles, lam, zeta, method="quadrature")
    b_b = bp.backproject(sino, N, angles, lam, zeta, method="boxspline")
    assert np.max(np.abs(b_q - b_b)) < 1e-12 * np.max(np.abs(b_q))
    pts = [(0, 0), (6, 6), (3, 1)]
    assert np.max(np.abs(bp.backproject_sampled(sino, N, angles, lam, zeta, pts)
                         - np.array([b_q[p] for p in pts]))) < 1e-13


def test_orientation():
    # theta = pi/2 projects onto x2: b depends on the row index k2 only, and the
    # bin ordering follows +x2 (a sample on the last bin lights the last row)
    N, M = 5, 7
    sino = np.zeros((1, M))
    sino[0, 5] = 1.0
    b = bp.backproject(sino, N, np.array([0.5]), 1.0, 0.0)
    assert np.max(np.abs(b - b[:, :1])) < 1e-15
    assert np.argmax(b[:, 0]) == 4
    b0 = bp.backproject(sino, N, np.array([0.0]), 1.0, 0.0)
    assert np.max(np.abs(b0 - b0[:1, :])) < 1e-15 and np.argmax(b0[0]) == 4


def test_adjoint_identity():
    # <H x, g_hat> (continuous) = <x, H^T g_hat>
    N, M, lam, zeta = 5, 9, 0.9, 1.0
    angles = np.array([0.08, 0.41])
    rng = np.random.default_rng(7)
    x = rng.standard_normal((N, N))
    sino = rng.standard_normal((2, M))
    b = bp.backproject(sino, N, angles, lam, zeta)
    coef = bp.prefilter(sino, angles, zeta)
    lhs = 0.0
    for j, th in enumerate(angles):
        c, s = cospi_sinpi(th)
        d = interp_degree(c, s, zeta)
        t = pixel_projections(N, c, s).reshape(-1)
        knots = bin_centres(M, lam)[0] + lam * (np.arange(-4, M + 4) + (0.5 if d % 2 == 0 else 0.0))
        edges = np.unique(np.concatenate([knots] + [bs.footprint_breakpoints(c, s, zeta) + tk for tk in t]))[None, :]
        f = lambda y: bp.interpolant(coef[j], y, lam, d) * (bs.blurred_footprint(y[..., None] - t, c, s, zeta) @ x.reshape(-1))
        lhs += bs.gl3_integrate(edges, f)[0]
    assert abs(lhs - np.sum(x * b)) < 1e-12 * abs(lhs)


def test_prefilter_only_on_degree_two_views():
    sino = np.random.default_rng(4).standard_normal((3, 30))
    angles = np.array([0.0, 0.2, 0.5])
    out = bp.prefilter(sino, angles, 1.0)
    assert np.array_equal(out[0], sino[0]) and np.array_equal(out[2], sino[2])
    assert not np.allclose(out[1], sino[1])
    assert np.array_equal(bp.prefilter(sino, angles, 0.0), sino)


def test_forward_partition_of_unity():
    # zeta = 1 and lambda_y = 1: the footprint M_[|c|,|s|,1] contains a unit box, whose
    # integer shifts sum to one, so every view's samples add up to the sum of the
    # coefficients (the detector covers the whole image)
    N, M = 9, 17
    angles = np.array([0.0, 0.07, 0.25, 0.31, 0.5, 0.83])
    c = np.random.default_rng(11).standard_normal((N, N))
    sino = bp.forward_sample(c, angles, M, 1.0, 1.0)
    assert np.max(np.abs(sino.sum(axis=1) - c.sum())) < 1e-12 * np.abs(c).sum()


def test_forward_axis_views_are_line_sums():
    # theta = 0 without blur, lambda_y = 1, M = N: bin m sees exactly column m (a unit
    # box of the detector coordinate); theta = pi/2 sees row m
    N = 8
    c = np.random.default_rng(12).standard_normal((N, N))
    sino = bp.forward_sample(c, np.array([0.0, 0.5]), N, 1.0, 0.0)
    assert np.max(np.abs(sino[0] - c.sum(axis=0))) < 1e-13
    assert np.max(np.abs(sino[1] - c.sum(axis=1))) < 1e-13


def test_forward_sample_points_match_full_views():
    N, M, lam, zeta = 11, 19, 0.8, 0.5
    angles = np.array([0.13, 0.5, 0.77])
    c = np.random.default_rng(13).standard_normal((N, N))
    full = bp.forward_sample(c, angles, M, lam, zeta)
    pts = [(0, 0), (0, 9), (1, 4), (2, 18), (2, 10)]
    got = bp.forward_sample_points(c, angles, M, lam, zeta, pts)
    assert np.max(np.abs(got - np.array([full[p] for p in pts]))) < 1e-14 * np.abs(full).max()
