"""Sinogram interpolation and back projection H^T g (Sec. 5) - oracle, FP64.

For each view theta the sampled sinogram g_s[m] is turned into a continuous signal

    g_hat(y) = sum_m c~[m] beta_d((y - y_m) / lambda_y)

(the oblique-projection interpolant of Sec. 5) with c~ = g_s * q, q the correction
filter of Eq. 5 (identity for degree 0 and 1).  The back projection is the exact
adjoint of the continuous forward model applied to it:

    b_k = sum_theta int g_hat_theta(y) h_theta(y - x_k . u_theta) dy.

Readings: d is chosen per view by ``geometry.interp_degree``; the degree-2 correction
filter is q[m] = sqrt(2) (2 sqrt(2) - 3)^|m| truncated at |m| <= 40 (the value the
paper prints for q[40] carries the sqrt(2) factor that its formula omits); the
sinogram is zero outside the detector; c~ is kept for m in [0, M) only.
"""
import math

import numpy as np

from . import boxspline as bs
from .geometry import bin_centres, cospi_sinpi, interp_degree, pixel_projections

Q_RADIUS = 40


def correction_filter(degree, radius=Q_RADIUS):
    """Taps q[-radius..radius] of Q(z) = 1 / sum_m b[m] z^-m (Eq. 5) for beta_degree.

    b[m] = beta_d(m).  For d = 0, 1, b = delta so q = delta.  For d = 2,
    b = [1/8, 3/4, 1/8] whose inverse is the symmetric exponential
    sqrt(2) * z1^|m| with z1 = 2 sqrt(2) - 3 (the root of z + 6 + 1/z = 0 inside
    the unit circle).
    """
    m = np.arange(-radius, radius + 1)
    if degree in (0, 1):
        return (m == 0).astype(np.float64)
    if degree == 2:
        z1 = 2.0 * math.sqrt(2.0) - 3.0
        return math.sqrt(2.0) * z1 ** np.abs(m)
    if degree == 3:
        # b = [1/6, 2/3, 1/6]: root of z + 4 + 1/z = 0 inside the unit circle, and the
        # gain that makes q * b = delta (several detector boxes, oblique views)
        z1 = math.sqrt(3.0) - 2.0
        return math.sqrt(3.0) * z1 ** np.abs(m)
    raise ValueError("degree must be 0, 1, 2 or 3")


def prefilter(sino, angles_pi, zeta):
    """c~ = g_s * q per view (zero extension beyond both detector ends), shape [n_angles, M]."""
    sino = np.asarray(sino, dtype=np.float64)
    c_all, s_all = cospi_sinpi(angles_pi)
    out = np.empty_like(sino)
    M = sino.shape[1]
    for j, (c, s) in enumerate(zip(np.atleast_1d(c_all), np.atleast_1d(s_all))):
        d = interp_degree(c, s, zeta)
        q = correction_filter(d)
        full = np.convolve(sino[j], q)  # length M + 2R
        out[j] = full[Q_RADIUS:Q_RADIUS + M]
    return out


def interpolant(coef, y, lam, degree):
    """g_hat(y) = sum_m coef[m] beta_d((y - y_m)/lambda) for one view (coef zero outside [0, M))."""
    M = coef.shape[0]
    y = np.asarray(y, dtype=np.float64)
    y0 = -(M - 1) / 2.0 * lam
    u = (y - y0) / lam  # position in bin units
    mc = np.round(u).astype(np.int64)
    out = np.zeros_like(y)
    for off in range(-2, 3):
        m = mc + off
        ok = (m >= 0) & (m < M)
        w = bs.bspline(u - m, degree)
        out = out + np.where(ok, coef[np.clip(m, 0, M - 1)] * w, 0.0)
    return out


def _bp_view_quadrature(coef, t, c, s, zeta, lam, degree):
    """int g_hat(y) h(y - t) dy for an array of pixel positions t (one view), exact GL."""
    M = coef.shape[0]
    half = bs.footprint_support(c, s, zeta)
    bp = bs.footprint_breakpoints(c, s, zeta)
    y0 = -(M - 1) / 2.0 * lam
    # knots of the interpolant: y0 + lam * (j + delta), delta = 1/2 for even degree
    delta = 0.5 if degree % 2 == 0 else 0.0
    lo = t - half
    hi = t + half
    jlo = np.floor((lo - y0) / lam - delta)
    nk = int(math.ceil(2 * half / lam)) + 3
    knots = y0 + lam * (jlo[..., None] + np.arange(nk) + delta)
    knots = np.clip(knots, lo[..., None], hi[..., None])
    edges = np.sort(np.concatenate([knots, bp + t[..., None], lo[..., None], hi[..., None]], axis=-1), axis=-1)
    edges = np.clip(edges, lo[..., None], hi[..., None])
    f = lambda y: interpolant(coef, y, lam, degree) * bs.blurred_footprint(y - t[..., None], c, s, zeta)
    # several detector boxes raise both degrees past what 3-point GL integrates exactly
    return bs.gl6_integrate(edges, f) if len(bs.blur_widths(zeta)) >= 2 else bs.gl3_integrate(edges, f)


def backproject(sino, N, angles_pi, lam, zeta, method="quadrature"):
    """b = H^T g_hat on the N x N grid (Sec. 5), FP64.

    method="quadrature": integral definition with the interpolant and footprint;
    method="boxspline":  the closed form sum_m c~[m] lambda M_[c, s, zeta, lambda^(d+1)](y_m - t),
                         truncated-power evaluation.
    """
    sino = np.asarray(sino, dtype=np.float64)
    M = sino.shape[1]
    coef_all = prefilter(sino, angles_pi, zeta)
    c_all, s_all = cospi_sinpi(angles_pi)
    ym = bin_centres(M, lam)
    b = np.zeros((N, N))
    for j, (c, s) in enumerate(zip(np.atleast_1d(c_all), np.atleast_1d(s_all))):
        d = interp_degree(c, s, zeta)
        t = pixel_projections(N, c, s)
        if method == "quadrature":
            b += _bp_view_quadrature(coef_all[j], t.reshape(-1), c, s, zeta, lam, d).reshape(N, N)
        elif method == "boxspline":
            dirs = bs.directions_backprojection(c, s, zeta, lam, d)
            half = 0.5 * sum(abs(x) for x in dirs)
            tt = t.reshape(-1)
            acc = np.zeros_like(tt)
            mlo = np.floor((tt - half - ym[0]) / lam).astype(np.int64)
            for off in range(0, int(math.ceil(2 * half / lam)) + 2):
                m = mlo + off
                ok = (m >= 0) & (m < M)
                mm = np.clip(m, 0, M - 1)
                acc += np.where(ok, coef_all[j][mm] * lam * bs.truncated_power(ym[mm] - tt, dirs), 0.0)
            b += acc.reshape(N, N)
        else:
            raise ValueError(method)
    return b


def backproject_sampled(sino, N, angles_pi, lam, zeta, points):
    """b at selected pixels (k2, k1) only, by the quadrature definition (large-N parity)."""
    sino = np.asarray(sino, dtype=np.float64)
    coef_all = prefilter(sino, angles_pi, zeta)
    c_all, s_all = cospi_sinpi(angles_pi)
    pts = np.asarray(points, dtype=np.int64).reshape(-1, 2)
    xk1 = pts[:, 1] - (N - 1) / 2.0
    xk2 = pts[:, 0] - (N - 1) / 2.0
    out = np.zeros(len(pts))
    for j, (c, s) in enumerate(zip(np.atleast_1d(c_all), np.atleast_1d(s_all))):
        d = interp_degree(c, s, zeta)
        out += _bp_view_quadrature(coef_all[j], xk1 * c + xk2 * s, c, s, zeta, lam, d)
    return out


def forward_sample(coeffs, angles_pi, M, lam, zeta):
    """g_s[theta, m] = S H f: point samples at y_m of the blurred projection of f_psi (Sec. 2, Eq. 4)."""
    coeffs = np.asarray(coeffs, dtype=np.float64)
    N = coeffs.shape[0]
    c_all, s_all = cospi_sinpi(angles_pi)
    ym = bin_centres(M, lam)
    out = np.zeros((len(np.atleast_1d(c_all)), M))
    for j, (c, s) in enumerate(zip(np.atleast_1d(c_all), np.atleast_1d(s_all))):
        t = pixel_projections(N, c, s).reshape(-1)
        w = coeffs.reshape(-1)
        nz = w != 0.0
        h = bs.blurred_footprint(ym[:, None] - t[None, nz], c, s, zeta)
        out[j] = h @ w[nz]
    return out


def forward_sample_points(coeffs, angles_pi, M, lam, zeta, points):
    """g_s[j, m] = (S H f)(theta_j, y_m) at selected (view index j, bin m) pairs only.

    The same sum over every pixel as ``forward_sample`` (Sec. 2, Eq. 4), evaluated one
    detector sample at a time so that large images can be checked at a few samples.
    """
    coeffs = np.asarray(coeffs, dtype=np.float64)
    N = coeffs.shape[0]
    c_all, s_all = cospi_sinpi(np.atleast_1d(angles_pi))
    ym = bin_centres(M, lam)
    w = coeffs.reshape(-1)
    out = []
    for j, m in points:
        c, s = c_all[j], s_all[j]
        t = pixel_projections(N, c, s).reshape(-1)
        half = bs.footprint_support(c, s, zeta)
        near = np.abs(ym[m] - t) < half
        out.append(float(bs.blurred_footprint(ym[m] - t[near], c, s, zeta) @ w[near]))
    return np.array(out)
