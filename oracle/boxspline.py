"""Univariate box splines and the pixel footprint (Sec. 3, Eq. 1 and Eq. 2) - oracle, FP64.

Two independent evaluations are kept on purpose:

1. ``truncated_power`` - the closed form of a centred, unit-mass univariate box
   spline M_Xi as an alternating sum of truncated powers over all subsets of the
   direction list (the standard expansion of the convolution of Eq. 1).  FP64 and
   an mpmath version (``truncated_power_mp``) for spot checks at high precision.
2. ``pixel_projection`` / ``blurred_footprint`` / ``footprint_autocorrelation`` -
   the same functions built from the geometry alone: the X-ray transform of the
   unit pixel as the chord length of a line through the unit square (Fig. 1,
   Eq. 2), the detector box (Sec. 2) applied by exact midpoint integration of that
   piecewise-linear chord, and the autocorrelation integral of Sec. 4 by
   Gauss-Legendre quadrature over merged breakpoints.  Every integrand is a
   non-negative piecewise polynomial integrated exactly, so there is no
   cancellation anywhere on this path.

Reading (the paper defines M_xi on [0, xi]): all box splines here are centred and
unit-mass; zero-length directions are dropped (they act as a Dirac delta).
"""
import math
import numpy as np

# 3-point Gauss-Legendre on [0, 1]: exact for polynomials of degree <= 5.
_GL3_X = np.array([0.5 - math.sqrt(15.0) / 10.0, 0.5, 0.5 + math.sqrt(15.0) / 10.0])
_GL3_W = np.array([5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0])
# 6-point Gauss-Legendre on [0, 1] (numpy's nodes): exact for degree <= 11, used where
# several detector boxes raise the degree of the integrands.
_GL6_X, _GL6_W = np.polynomial.legendre.leggauss(6)
_GL6_X, _GL6_W = 0.5 * (_GL6_X + 1.0), 0.5 * _GL6_W


def blur_widths(zeta):
    """The detector kernel's box widths: a number (one box, none if 0) or a sequence.

    Sec. 2 models the detector cell as a convolution of boxes and uses one; a sequence
    gives the convolution of unit-mass boxes of those widths (zeros dropped).
    """
    if np.ndim(zeta) == 0:
        return (float(zeta),) if float(zeta) > 0.0 else ()
    return tuple(float(w) for w in zeta if float(w) > 0.0)


def _multi(zeta):
    return np.ndim(zeta) != 0 and len(blur_widths(zeta)) >= 2


def _clean_dirs(dirs):
    a = [abs(float(d)) for d in dirs]
    return [d for d in a if d != 0.0]


def truncated_power(x, dirs):
    """Centred unit-mass box spline M_[dirs](x) by the truncated-power formula, FP64.

    M(x) = 1 / ((n-1)! prod a_i) * sum_{S subset} (-1)^{|S|} (x + sum(a)/2 - sum_S a)_+^{n-1}

    Plain 2^n loop over subsets; no grouping of repeated directions.
    """
    a = _clean_dirs(dirs)
    n = len(a)
    if n == 0:
        raise ValueError("box spline needs at least one non-zero direction")
    x = np.asarray(x, dtype=np.float64)
    half = 0.5 * sum(a)
    acc = np.zeros_like(x)
    for mask in range(1 << n):
        off = 0.0
        bits = 0
        for i in range(n):
            if (mask >> i) & 1:
                off += a[i]
                bits += 1
        z = x + half - off
        if n == 1:
            term = (z > 0.0).astype(np.float64)
        else:
            term = np.where(z > 0.0, z, 0.0) ** (n - 1)
        acc = acc + (-term if bits & 1 else term)
    return acc / (math.factorial(n - 1) * math.prod(a))


def truncated_power_mp(x, dirs, dps=60):
    """Same formula in mpmath at ``dps`` decimal digits (scalar x); returns mpf.

    The FP64 direction values are converted exactly, so this measures the rounding
    error of the FP64 evaluation of the same function.
    """
    import mpmath as mp

    with mp.workdps(dps):
        a = [mp.mpf(abs(float(d))) for d in dirs if float(d) != 0.0]
        n = len(a)
        xm = mp.mpf(float(x)) if not isinstance(x, mp.mpf) else x
        half = sum(a) / 2
        acc = mp.mpf(0)
        for mask in range(1 << n):
            off = mp.mpf(0)
            bits = 0
            for i in range(n):
                if (mask >> i) & 1:
                    off += a[i]
                    bits += 1
            z = xm + half - off
            if n == 1:
                term = mp.mpf(1) if z > 0 else mp.mpf(0)
            else:
                term = z ** (n - 1) if z > 0 else mp.mpf(0)
            acc += -term if bits & 1 else term
        return acc / (mp.factorial(n - 1) * mp.fprod(a))


# ----------------------------------------------------------------------------------
# Geometric path (no box-spline algebra)
# ----------------------------------------------------------------------------------

def pixel_projection(y, c, s):
    """X-ray transform of the unit pixel [-1/2, 1/2]^2 along direction u = (c, s) (Fig. 1).

    Returns the length of the chord {x in pixel : x . u = y}.  The chord is
    parametrised along the coordinate axis with the larger |u| component; the
    pixel is symmetric under x1 -> -x1 and x2 -> -x2, so only |c|, |s| matter.
    Requires c^2 + s^2 = 1.
    """
    y = np.asarray(y, dtype=np.float64)
    a, b = abs(float(c)), abs(float(s))
    if b < a:  # swap roles: parametrise along x2
        a, b = b, a
    # line: a*x1 + b*x2 = y with b >= a > = 0, x1 in [-1/2, 1/2], |x2| <= 1/2
    if a == 0.0:
        inside = np.abs(y) < 0.5 * b
        return np.where(inside, 1.0 / b, 0.0)
    lo = (y - 0.5 * b) / a
    hi = (y + 0.5 * b) / a
    dx1 = np.clip(np.minimum(hi, 0.5) - np.maximum(lo, -0.5), 0.0, None)
    return dx1 / b  # chord length = dx1 * sqrt(1 + a^2/b^2) = dx1 / b


def projection_breakpoints(c, s):
    """Kinks of the pixel's projection: +-(|c|+|s|)/2 and +-||c|-|s||/2."""
    a, b = abs(float(c)), abs(float(s))
    return np.array([-(a + b) / 2, -abs(a - b) / 2, abs(a - b) / 2, (a + b) / 2])


def blurred_footprint(y, c, s, zeta):
    """Detector-blurred projection h(y) = (1/zeta) int_{|v|<zeta/2} P(y - v) dv (Sec. 2).

    The detector box is read as a unit-mass average (a detector cell averages the
    signal over its width).  zeta = 0 returns the unblurred chord.  The integral is
    exact: the window is split at the chord's four kinks and each linear piece is
    integrated by its midpoint value.
    """
    y = np.asarray(y, dtype=np.float64)
    if _multi(zeta):
        return _footprint_boxes(y, c, s, blur_widths(zeta))
    if np.ndim(zeta) != 0:
        zeta = blur_widths(zeta)[0] if blur_widths(zeta) else 0.0
    if zeta == 0.0:
        return pixel_projection(y, c, s)
    bp = projection_breakpoints(c, s)
    lo = y - 0.5 * zeta
    hi = y + 0.5 * zeta
    edges = np.concatenate(
        [lo[..., None], np.clip(bp, lo[..., None], hi[..., None]), hi[..., None]], axis=-1
    )
    edges = np.sort(edges, axis=-1)
    length = np.diff(edges, axis=-1)
    mid = 0.5 * (edges[..., 1:] + edges[..., :-1])
    vals = pixel_projection(mid, c, s)
    return np.sum(length * vals, axis=-1) / zeta


def _footprint_boxes(y, c, s, widths):
    """P averaged successively over boxes of the given widths: each average is the exact
    integral of a piecewise polynomial over its window, split at the previous level's
    kinks and summed by 6-point Gauss-Legendre (exact for the degrees that arise)."""
    if not widths:
        return pixel_projection(y, c, s)
    w = widths[-1]
    inner = widths[:-1]
    bp = footprint_breakpoints(c, s, inner) if inner else projection_breakpoints(c, s)
    lo = y - 0.5 * w
    hi = y + 0.5 * w
    edges = np.sort(np.concatenate([lo[..., None], np.clip(bp, lo[..., None], hi[..., None]), hi[..., None]],
                                   axis=-1), axis=-1)
    a = edges[..., :-1]
    ln = edges[..., 1:] - a
    total = 0.0
    for xg, wg in zip(_GL6_X, _GL6_W):
        total = total + np.sum(wg * ln * _footprint_boxes(a + xg * ln, c, s, inner), axis=-1)
    return total / w


def footprint_breakpoints(c, s, zeta):
    bp = projection_breakpoints(c, s)
    if _multi(zeta):
        for w in blur_widths(zeta):
            bp = np.unique(np.concatenate([bp - 0.5 * w, bp + 0.5 * w]))
        return bp
    if np.ndim(zeta) != 0:
        zeta = blur_widths(zeta)[0] if blur_widths(zeta) else 0.0
    if zeta == 0.0:
        return bp
    return np.sort(np.concatenate([bp - 0.5 * zeta, bp + 0.5 * zeta]))


def footprint_support(c, s, zeta):
    """Half-width of h's support: (|c| + |s| + zeta) / 2 (zeta: the sum of the box widths)."""
    return 0.5 * (abs(float(c)) + abs(float(s)) + float(sum(blur_widths(zeta))))


def gl3_integrate(edges, f):
    """Sum over consecutive pieces of ``edges`` (last axis) of 3-point Gauss-Legendre of f.

    Exact for piecewise polynomials of degree <= 5 whose kinks are all in ``edges``.
    """
    lo = edges[..., :-1]
    w = edges[..., 1:] - lo
    total = 0.0
    for xg, wg in zip(_GL3_X, _GL3_W):
        total = total + np.sum(wg * w * f(lo + xg * w), axis=-1)
    return total


def footprint_autocorrelation(t, c, s, zeta):
    """A(t) = int h(y) h(y - t) dy (the per-view Gram kernel of Sec. 4), exact quadrature.

    h is piecewise quadratic, so the product is piecewise quartic between the merged
    kinks of h(y) and h(y - t); 3-point Gauss-Legendre per piece is exact.
    """
    t = np.asarray(t, dtype=np.float64)
    bp = footprint_breakpoints(c, s, zeta)
    edges = np.sort(np.concatenate(
        [np.broadcast_to(bp, t.shape + bp.shape), bp + t[..., None]], axis=-1), axis=-1)
    f = lambda y: blurred_footprint(y, c, s, zeta) * blurred_footprint(y - t[..., None], c, s, zeta)
    return gl6_integrate(edges, f) if _multi(zeta) else gl3_integrate(edges, f)


def gl6_integrate(edges, f):
    """As ``gl3_integrate`` with 6-point Gauss-Legendre: exact for degree <= 11."""
    lo = edges[..., :-1]
    w = edges[..., 1:] - lo
    total = 0.0
    for xg, wg in zip(_GL6_X, _GL6_W):
        total = total + np.sum(wg * w * f(lo + xg * w), axis=-1)
    return total


# ----------------------------------------------------------------------------------
# Centred B-splines (used to interpolate the sinogram, Sec. 5)
# ----------------------------------------------------------------------------------

def bspline(x, d):
    """Centred cardinal B-spline beta_d(x) of degree d in {0, 1, 2, 3} (textbook pieces)."""
    x = np.abs(np.asarray(x, dtype=np.float64))
    if d == 0:
        return np.where(x < 0.5, 1.0, np.where(x == 0.5, 0.5, 0.0))
    if d == 1:
        return np.clip(1.0 - x, 0.0, None)
    if d == 2:
        return np.where(x < 0.5, 0.75 - x * x,
                        np.where(x < 1.5, 0.5 * (x - 1.5) ** 2, 0.0))
    if d == 3:
        return np.where(x < 1.0, 2.0 / 3.0 - x * x + 0.5 * x ** 3,
                        np.where(x < 2.0, (2.0 - x) ** 3 / 6.0, 0.0))
    raise ValueError("degree must be 0, 1, 2 or 3")


def directions_gram(c, s, zeta):
    """Direction list of the Gram kernel: [c, c, s, s] (Sec. 4), plus [w, w] per detector box."""
    d = [c, c, s, s]
    for w in blur_widths(zeta):
        d += [w, w]
    return d


def directions_backprojection(c, s, zeta, lam, degree):
    """Directions of the back-projection kernel lambda * M_[c, s, zeta, lambda^(d+1)].

    beta_d((y - y_m)/lambda) = lambda * M_[lambda x (d+1)](y - y_m); convolving it with
    the footprint M_[c, s, zeta] gives the kernel that weighs sample m for a pixel.
    """
    d = [c, s]
    d += list(blur_widths(zeta))
    d += [lam] * (degree + 1)
    return d
