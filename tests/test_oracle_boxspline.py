"""Pins for the oracle's box splines (Sec. 3, Eq. 1-2) against closed forms, libraries,
high precision and brute force.  CPU only."""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import boxspline as bs
from oracle.geometry import cospi_sinpi, interp_degree


def _bspline_scipy(x, d):
    knots = np.arange(d + 2) - (d + 1) / 2.0
    return BSpline.basis_element(knots, extrapolate=False)(x)


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_equal_directions_give_cardinal_bspline(d):
    # M_[1 x (d+1)] is the centred cardinal B-spline of degree d (library routine pin)
    x = np.linspace(-(d + 1) / 2 + 1e-3, (d + 1) / 2 - 1e-3, 257)
    ref = np.nan_to_num(_bspline_scipy(x, d))
    assert np.max(np.abs(bs.truncated_power(x, [1.0] * (d + 1)) - ref)) < 1e-13
    if d <= 2:
        assert np.max(np.abs(bs.bspline(x, d) - ref)) < 1e-14


def test_scaled_directions_scale_the_argument():
    # M_[a x n](x) = beta_{n-1}(x / a) / a  (unit mass under dilation)
    a = 0.37
    x = np.linspace(-0.7, 0.7, 101)
    ref = np.nan_to_num(_bspline_scipy(x / a, 3)) / a
    assert np.max(np.abs(bs.truncated_power(x, [a] * 4) - ref)) < 1e-12


@pytest.mark.parametrize("th", [0.03, 0.1, 0.2, 0.25, 0.31, 0.45, 0.6, 0.77])
def test_pixel_chord_equals_two_direction_box_spline(th):
    # Eq. 2 / Fig. 1: the X-ray transform of the unit pixel is M_[|cos|, |sin|]
    c, s = cospi_sinpi(th)
    y = np.linspace(-0.8, 0.8, 333) + 1e-7
    chord = bs.pixel_projection(y, c, s)
    assert np.max(np.abs(chord - bs.truncated_power(y, [c, s]))) < 1e-12


def test_pixel_chord_brute_force():
    # chord length by dense sampling of the line through the unit square
    c, s = cospi_sinpi(0.137)
    for y in [-0.6, -0.31, 0.0, 0.22, 0.55]:
        tt = np.linspace(-2, 2, 2_000_001)
        px = y * c - tt * s
        py = y * s + tt * c
        inside = (np.abs(px) <= 0.5) & (np.abs(py) <= 0.5)
        brute = inside.sum() * (tt[1] - tt[0])
        assert abs(brute - bs.pixel_projection(y, c, s)) < 1e-5


@pytest.mark.parametrize("th,zeta", [(0.0, 0.0), (0.0, 1.0), (0.13, 0.0), (0.13, 1.0), (0.25, 0.5), (0.5, 1.0)])
def test_unit_mass(th, zeta):
    c, s = cospi_sinpi(th)
    for f, bpfun in [
        (lambda y: bs.blurred_footprint(y, c, s, zeta), lambda: bs.footprint_breakpoints(c, s, zeta)),
        (lambda y: bs.footprint_autocorrelation(y, c, s, zeta),
         lambda: np.sort(np.concatenate([bs.footprint_breakpoints(c, s, zeta) + b
                                         for b in bs.footprint_breakpoints(c, s, zeta)]))),
    ]:
        edges = np.unique(bpfun())[None, :]
        assert abs(bs.gl3_integrate(edges, f)[0] - 1.0) < 1e-13


@pytest.mark.parametrize("th", [0.02, 0.1, 0.25, 0.4, 0.49, 0.7])
@pytest.mark.parametrize("zeta", [0.0, 1.0, 0.3])
def test_autocorrelation_equals_gram_box_spline_mp(th, zeta):
    # Sec. 4: the per-view Gram kernel is M_[c,c,s,s(,zeta,zeta)]; checked at 60 digits
    c, s = cospi_sinpi(th)
    dirs = bs.directions_gram(c, s, zeta)
    assert len(dirs) == (6 if zeta > 0 else 4)
    t = np.linspace(-2.2, 2.2, 17) + 1e-3
    A = bs.footprint_autocorrelation(t, c, s, zeta)
    ref = np.array([float(bs.truncated_power_mp(x, dirs)) for x in t])
    assert np.max(np.abs(A - ref)) < 5e-16 * 4


def test_fp64_truncated_power_cancellation_is_real():
    # the FP64 truncated power loses digits near axis-aligned views; quadrature does not
    c, s = cospi_sinpi(0.002)
    t = np.linspace(-1.5, 1.5, 31)
    ref = np.array([float(bs.truncated_power_mp(x, bs.directions_gram(c, s, 1.0))) for x in t])
    err_tp = np.max(np.abs(bs.truncated_power(t, bs.directions_gram(c, s, 1.0)) - ref))
    err_q = np.max(np.abs(bs.footprint_autocorrelation(t, c, s, 1.0) - ref))
    assert err_q < 1e-15 and err_tp > 1e-12


def test_centre_tap_closed_form():
    # A(0) = int P^2 = 1/max - min/(3 max^2) for the unblurred trapezoid
    for th in [0.05, 0.13, 0.25, 0.41]:
        c, s = cospi_sinpi(th)
        mx, mn = max(abs(c), abs(s)), min(abs(c), abs(s))
        assert abs(bs.footprint_autocorrelation(np.array([0.0]), c, s, 0.0)[0]
                   - (1 / mx - mn / (3 * mx * mx))) < 1e-15


def test_axis_aligned_kernels():
    # theta = 0: P = unit box, A = hat (no blur) or cubic B-spline (zeta = 1)
    t = np.linspace(-2.4, 2.4, 97) + 1e-4
    A0 = bs.footprint_autocorrelation(t, 1.0, 0.0, 0.0)
    assert np.max(np.abs(A0 - np.clip(1 - np.abs(t), 0, None))) < 1e-15
    A1 = bs.footprint_autocorrelation(t, 1.0, 0.0, 1.0)
    assert np.max(np.abs(A1 - np.nan_to_num(_bspline_scipy(t, 3)))) < 1e-15
    # 45 degrees: four equal directions 1/sqrt(2) -> sqrt(2) beta_3(sqrt(2) t)
    c, s = cospi_sinpi(0.25)
    A45 = bs.footprint_autocorrelation(t, c, s, 0.0)
    ref = math.sqrt(2.0) * np.nan_to_num(_bspline_scipy(math.sqrt(2.0) * t, 3))
    assert np.max(np.abs(A45 - ref)) < 1e-14


def test_degree_rule():
    assert interp_degree(1.0, 0.0, 0.0) == 0
    assert interp_degree(0.6, 0.8, 0.0) == 1
    assert interp_degree(1.0, 0.0, 1.0) == 1
    assert interp_degree(0.6, 0.8, 1.0) == 2
    c, s = cospi_sinpi(np.array([0.0, 0.5, 1.0]))
    assert np.all(s[[0, 2]] == 0.0) and c[1] == 0.0


def test_backprojection_kernel_is_interpolant_footprint_correlation():
    # lambda * M_[c, s, zeta, lambda^(d+1)](y_m - t) = int beta_d((y - y_m)/lambda) h(y - t) dy
    lam = 0.8
    for th, zeta in [(0.17, 0.0), (0.17, 1.0), (0.0, 1.0), (0.5, 0.0)]:
        c, s = cospi_sinpi(th)
        d = interp_degree(c, s, zeta)
        dirs = bs.directions_backprojection(c, s, zeta, lam, d)
        for u in [-1.3, -0.4, 0.05, 0.61, 1.7]:
            kn = lam * (np.arange(-3, 4) + (0.5 if d % 2 == 0 else 0.0))
            edges = np.sort(np.concatenate([kn, bs.footprint_breakpoints(c, s, zeta) - u]))[None, :]
            val = bs.gl3_integrate(edges, lambda y: bs.bspline(y / lam, d) * bs.blurred_footprint(y - (-u), c, s, zeta))[0]
            # y_m = 0, t = -u  => argument y_m - t = u
            ref = float(bs.truncated_power_mp(u, dirs)) * lam
            assert abs(val - ref) < 1e-14
