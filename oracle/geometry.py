"""Geometry of the parallel-beam problem (Sec. 2) - oracle side, FP64.

Conventions (the paper fixes none of them; these are the readings used throughout):

* coefficient image ``c[k2, k1]`` row-major, unit pixels (Lambda_x = I, Sec. 4),
  pixel centre x_k = (k1 - (N-1)/2, k2 - (N-1)/2);
* projection direction u_theta = (cos theta, sin theta); a point x projects to the
  detector coordinate y = x . u_theta;
* detector bin centres y_m = (m - (M-1)/2) * lambda_y, m = 0..M-1 (the sampling
  operator S of Sec. 2 samples at lambda_y-spaced points);
* angles are passed as theta / pi ("half turns") so that the axis-aligned angles
  0 and pi/2 give exactly zero sines / cosines.
"""
import numpy as np


def cospi_sinpi(a):
    """cos(pi*a), sin(pi*a) in FP64, exact at multiples of 1/2 (axis-aligned views)."""
    a = np.asarray(a, dtype=np.float64)
    c = np.cos(np.pi * a)
    s = np.sin(np.pi * a)
    two = 2.0 * a
    exact = two == np.round(two)
    if np.any(exact):
        q = np.mod(np.round(two[exact]).astype(np.int64), 4)
        c_tab = np.array([1.0, 0.0, -1.0, 0.0])
        s_tab = np.array([0.0, 1.0, 0.0, -1.0])
        c = np.array(c, copy=True)
        s = np.array(s, copy=True)
        c[exact] = c_tab[q]
        s[exact] = s_tab[q]
    return c, s


def uniform_angles(n_angles):
    """theta_j / pi = j / n_angles, j = 0..n-1 (uniform in [0, pi))."""
    return np.arange(n_angles, dtype=np.float64) / float(n_angles)


def pixel_centres(N):
    """1-D pixel centre coordinates k - (N-1)/2 for unit pixels."""
    return np.arange(N, dtype=np.float64) - (N - 1) / 2.0


def bin_centres(M, lambda_y):
    """Detector sample positions y_m = (m - (M-1)/2) * lambda_y."""
    return (np.arange(M, dtype=np.float64) - (M - 1) / 2.0) * float(lambda_y)


def pixel_projections(N, c, s):
    """t_k = x_k . u for every pixel, as an [N, N] array indexed [k2, k1]."""
    xc = pixel_centres(N)
    return xc[None, :] * c + xc[:, None] * s


def interp_degree(c, s, zeta):
    """B-spline degree used to interpolate one view (Sec. 5).

    The projected pixel is a box spline with directions [|cos|, |sin|] (Eq. 3),
    plus zeta_blur when the detector blurs (Eq. 4).  Its continuity class is
    (number of non-zero directions) - 2, so the interpolating B-spline has degree
    (number of non-zero directions) - 1: degree 1 in general, 0 for axis-aligned
    views without blur, 2 / 1 with blur.
    """
    if np.ndim(zeta) == 0:
        return int(c != 0.0) + int(s != 0.0) + int(zeta > 0.0) - 1
    # several detector boxes: one more direction each
    return int(c != 0.0) + int(s != 0.0) + sum(1 for w in zeta if float(w) > 0.0) - 1
