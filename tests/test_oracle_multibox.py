"""Pins for the oracle's detector kernel made of several boxes (Sec. 2) - CPU only.

Sec. 2 models the detector cell as a convolution of boxes and uses one; a sequence of
widths gives the convolution of unit-mass boxes.  The footprint is then the box spline
M_[|c|, |s|, w1, w2, ...], the Gram kernel M_[c, c, s, s, w1, w1, w2, w2, ...] and the
interpolation degree one more per box.  Pins: the geometric footprint against the
truncated-power closed form, unit mass, the one-box case, the partition of unity of a
unit box, the Gram taps and the back projection by both evaluations, the cubic
correction filter, exact recovery on axis views (Sec. 5) and the adjoint identity.
"""
import numpy as np
import pytest

from oracle import backproject as bp
from oracle import boxspline as bs
from oracle import gram
from oracle.geometry import bin_centres, cospi_sinpi, interp_degree, pixel_projections

ANGLES = np.array([0.0, 0.07, 0.25, 0.31, 0.5, 0.83])


@pytest.mark.parametrize("widths", [(1.0, 0.6), (0.5, 0.8, 1.3)])
def test_footprint_matches_truncated_power(widths):
    y = np.random.default_rng(1).uniform(-2.5, 2.5, 400)
    for a in ANGLES:
        c, s = cospi_sinpi(a)
        h = bs.blurred_footprint(y, c, s, widths)
        ref = bs.truncated_power(y, [abs(c), abs(s)] + list(widths))
        assert np.max(np.abs(h - ref)) < 1e-12
        edges = bs.footprint_breakpoints(c, s, widths)[None, :]
        assert bs.gl6_integrate(edges, lambda t: bs.blurred_footprint(t, c, s, widths))[0] == pytest.approx(1.0, abs=1e-13)


def test_one_box_sequence_is_the_scalar_path():
    y = np.linspace(-2, 2, 101)
    for a in ANGLES:
        c, s = cospi_sinpi(a)
        assert np.array_equal(bs.blurred_footprint(y, c, s, (0.7,)), bs.blurred_footprint(y, c, s, 0.7))
        assert np.array_equal(bs.blurred_footprint(y, c, s, (0.7, 0.0)), bs.blurred_footprint(y, c, s, 0.7))
    assert interp_degree(0.6, 0.8, (0.5, 1.0)) == 3 and interp_degree(1.0, 0.0, (0.5, 1.0)) == 2


def test_partition_of_unity_with_a_unit_box():
    N, M = 9, 19
    c = np.random.default_rng(2).standard_normal((N, N))
    sino = bp.forward_sample(c, ANGLES, M, 1.0, (1.0, 0.6))
    assert np.max(np.abs(sino.sum(axis=1) - c.sum())) < 1e-12 * np.abs(c).sum()


def test_gram_taps_two_evaluations():
    # views away from the axes: the degree-7 truncated-power form cancels badly when a
    # direction is short (|sin| = 0.09 cost it 6e-7 relative on the smallest taps)
    angles = np.array([0.15, 0.21, 0.5, 0.64])
    Gq = gram.gram_taps(6, angles, (0.5, 0.8), method="quadrature")
    Gb = gram.gram_taps(6, angles, (0.5, 0.8), method="boxspline")
    assert np.max(np.abs(Gq - Gb)) < 1e-12 * np.max(np.abs(Gq))
    assert np.allclose(Gq, Gq[::-1, ::-1], rtol=0, atol=1e-15)  # G[d] = G[-d]


def test_gram_kernel_near_axis_against_mpmath():
    # the quadrature (no cancellation) against 60-digit truncated powers where FP64
    # truncated powers fail: a view 5 degrees from the axis, two boxes
    c, s = cospi_sinpi(0.03)
    widths = (0.5, 0.8)
    t = np.array([0.0, 0.3, 0.9, 1.4, 1.9])
    a = bs.footprint_autocorrelation(t, c, s, widths)
    dirs = bs.directions_gram(c, s, widths)
    ref = np.array([float(bs.truncated_power_mp(ti, dirs)) for ti in t])
    assert np.max(np.abs(a - ref)) < 1e-13 * np.max(ref)


def test_cubic_correction_filter_and_spline():
    q = bp.correction_filter(3)
    b3 = np.array([1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0])
    conv = np.convolve(q, b3)
    centre = len(conv) // 2
    delta = np.zeros_like(conv)
    delta[centre] = 1.0
    assert np.max(np.abs(conv - delta)[5:-5]) < 1e-15
    scipy_bs = pytest.importorskip("scipy.interpolate")
    x = np.linspace(-2.5, 2.5, 201)
    ref = scipy_bs.BSpline.basis_element(np.arange(-2, 3), extrapolate=False)(x)
    assert np.max(np.abs(bs.bspline(x, 3) - np.nan_to_num(ref))) < 1e-14


def test_back_projection_two_evaluations():
    N, M = 6, 14
    angles = np.array([0.0, 0.12, 0.27, 0.5, 0.9])
    sino = np.random.default_rng(3).standard_normal((len(angles), M))
    bq = bp.backproject(sino, N, angles, 0.9, (0.7, 1.0), method="quadrature")
    bb = bp.backproject(sino, N, angles, 0.9, (0.7, 1.0), method="boxspline")
    # the truncated-power side sums degree-7 terms (c, s, two boxes and four lambda
    # directions) and keeps about 11 digits here
    assert np.max(np.abs(bq - bb)) < 1e-11 * np.max(np.abs(bq))


def test_exact_recovery_axis_views_two_boxes():
    # views {0, pi/2}, N and M even, lambda_y = 1, two unit boxes: the footprint
    # M_[1, 1, 1] is the quadratic B-spline, so each view's projection lies in the
    # degree-2 interpolation space and H^T g_hat = G c exactly (the argument of Sec. 5)
    N, M = 6, 12
    angles = np.array([0.0, 0.5])
    widths = (1.0, 1.0)
    c = np.random.default_rng(4).standard_normal((N, N))
    sino = bp.forward_sample(c, angles, M, 1.0, widths)
    b = bp.backproject(sino, N, angles, 1.0, widths)
    Gc = gram.gram_apply_direct(gram.gram_taps(N, angles, widths), c)
    assert np.max(np.abs(b - Gc)) < 1e-13 * np.max(np.abs(Gc))


def test_adjoint_identity_two_boxes():
    # <H x, g_hat> (continuous) = <x, H^T g_hat> with cubic interpolation on oblique views
    N, M, lam, widths = 5, 11, 0.9, (0.7, 1.0)
    angles = np.array([0.08, 0.41])
    rng = np.random.default_rng(7)
    x = rng.standard_normal((N, N))
    sino = rng.standard_normal((2, M))
    b = bp.backproject(sino, N, angles, lam, widths)
    coef = bp.prefilter(sino, angles, widths)
    lhs = 0.0
    for j, th in enumerate(angles):
        c, s = cospi_sinpi(th)
        d = interp_degree(c, s, widths)
        assert d == 3
        t = pixel_projections(N, c, s).reshape(-1)
        knots = bin_centres(M, lam)[0] + lam * (np.arange(-4, M + 4) + (0.5 if d % 2 == 0 else 0.0))
        edges = np.unique(np.concatenate([knots] + [bs.footprint_breakpoints(c, s, widths) + tk for tk in t]))[None, :]
        f = lambda y: bp.interpolant(coef[j], y, lam, d) * (bs.blurred_footprint(y[..., None] - t, c, s, widths) @ x.reshape(-1))
        lhs += bs.gl6_integrate(edges, f)[0]
    assert abs(lhs - np.sum(x * b)) < 1e-12 * abs(lhs)


def test_explicit_gram_matrix_is_the_filter_two_boxes():
    # H^T H entry by entry (integrals over both footprints' kinks, no Toeplitz
    # assumption) against the filter applied by shifted sums (Sec. 4)
    N = 3
    angles = np.array([0.1, 0.37, 0.5])
    widths = (0.6, 0.9)
    Gm = gram.explicit_gram_matrix(N, angles, widths)
    G = gram.gram_taps(N, angles, widths)
    for k in range(N * N):
        e = np.zeros(N * N)
        e[k] = 1.0
        col = gram.gram_apply_direct(G, e.reshape(N, N)).reshape(-1)
        assert np.max(np.abs(Gm[:, k] - col)) < 1e-13 * np.max(np.abs(Gm))
