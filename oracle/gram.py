"""Gram filter of the pixel-basis X-ray transform (Sec. 4) - oracle, FP64.

G = H^T H where H maps pixel coefficients to the (blurred) projections.  The entry
for two pixels depends only on their offset d = k_i - k_j (Toeplitz-block-Toeplitz,
Sec. 4 closing remark), so G is a (2N-1) x (2N-1) filter:

    G[d] = sum_theta A_theta(d . u_theta),   A_theta(t) = int h_theta(y) h_theta(y - t) dy

With the unit-mass readings of the footprint (see ``boxspline``), A_theta is the
box spline with directions [c, c, s, s] (Sec. 4, no blur) or [c, c, s, s, zeta, zeta]
(Sec. 4, with blur).  Filter arrays are indexed [d2 + N - 1, d1 + N - 1].
"""
import numpy as np

from . import boxspline as bs
from .geometry import cospi_sinpi, pixel_projections


def _offsets(N):
    d = np.arange(-(N - 1), N, dtype=np.float64)
    return d[None, :], d[:, None]  # d1 (columns), d2 (rows)


def gram_taps(N, angles_pi, zeta, method="quadrature"):
    """Full (2N-1)^2 filter.

    method="quadrature": A_theta by the autocorrelation integral (definition);
    method="boxspline":  A_theta by the truncated-power box spline of Sec. 4 (FP64).
    Only offsets inside the strip |d.u| < (|c|+|s|+zeta) are evaluated (A vanishes
    outside its support).
    """
    d1, d2 = _offsets(N)
    G = np.zeros((2 * N - 1, 2 * N - 1))
    c_all, s_all = cospi_sinpi(angles_pi)
    for c, s in zip(np.atleast_1d(c_all), np.atleast_1d(s_all)):
        t = d1 * c + d2 * s
        half = abs(c) + abs(s) + sum(bs.blur_widths(zeta))
        mask = np.abs(t) < half
        if not np.any(mask):
            continue
        tv = t[mask]
        if method == "quadrature":
            G[mask] += bs.footprint_autocorrelation(tv, c, s, zeta)
        elif method == "boxspline":
            G[mask] += bs.truncated_power(tv, bs.directions_gram(c, s, zeta))
        else:
            raise ValueError(method)
    return G


def gram_tap_values(offsets, angles_pi, zeta, method="quadrature"):
    """G[d] for a list of integer offsets d = (d1, d2) only (for sampled parity checks)."""
    offsets = np.asarray(offsets, dtype=np.float64).reshape(-1, 2)
    out = np.zeros(len(offsets))
    c_all, s_all = cospi_sinpi(angles_pi)
    for c, s in zip(np.atleast_1d(c_all), np.atleast_1d(s_all)):
        t = offsets[:, 0] * c + offsets[:, 1] * s
        mask = np.abs(t) < abs(c) + abs(s) + sum(bs.blur_widths(zeta))
        if not np.any(mask):
            continue
        if method == "quadrature":
            out[mask] += bs.footprint_autocorrelation(t[mask], c, s, zeta)
        else:
            out[mask] += bs.truncated_power(t[mask], bs.directions_gram(c, s, zeta))
    return out


def explicit_gram_matrix(N, angles_pi, zeta):
    """Explicit N^2 x N^2 matrix H^T H, entry by entry, for tiny grids (Sec. 4).

    Entry (i, j) = sum_theta int h_theta(y - t_i) h_theta(y - t_j) dy, integrated by
    Gauss-Legendre over the union of the kinks of BOTH footprints (not via A_theta),
    so Toeplitz structure is a result here, not an assumption.  Rows / columns are
    pixels in row-major order k = k2 * N + k1.
    """
    c_all, s_all = cospi_sinpi(angles_pi)
    n = N * N
    Gm = np.zeros((n, n))
    for c, s in zip(np.atleast_1d(c_all), np.atleast_1d(s_all)):
        t = pixel_projections(N, c, s).reshape(-1)
        bp = bs.footprint_breakpoints(c, s, zeta)
        for i in range(n):
            ti = t[i]
            edges = np.sort(np.concatenate(
                [np.broadcast_to(bp + ti, (n, bp.size)), bp[None, :] + t[:, None]], axis=1), axis=1)
            f = lambda y: bs.blurred_footprint(y - ti, c, s, zeta) * bs.blurred_footprint(y - t[:, None], c, s, zeta)
            # several detector boxes raise the degree past 3-point Gauss-Legendre
            Gm[i, :] += bs.gl6_integrate(edges, f) if len(bs.blur_widths(zeta)) >= 2 else bs.gl3_integrate(edges, f)
    return Gm


def embed_circulant(G):
    """Place the (2N-1)^2 taps into a 2N x 2N circulant kernel (tap d at index d mod 2N).

    The slot d = +-N stays zero.  A 2N-periodic circular convolution with this kernel
    equals the linear convolution on an N x N support (the zero-padding of the FFT
    method), which is what makes G x exactly computable by FFT.
    """
    n2 = G.shape[0]
    N = (n2 + 1) // 2
    L = 2 * N
    K = np.zeros((L, L))
    idx = np.arange(-(N - 1), N) % L
    K[np.ix_(idx, idx)] = G
    return K


def gram_spectrum(G):
    """Real 2N x 2N spectrum of the circulant embedding (G[d] = G[-d] makes it real)."""
    S = np.fft.fft2(embed_circulant(G))
    return S.real, S.imag


def gram_apply_direct(G, x):
    """y[i] = sum_j G[i - j] x[j] - the definition of the Gram product, as shifted sums.

    Plain loop over every filter offset; intended for N <= 128.
    """
    N = x.shape[0]
    y = np.zeros((N, N))
    for a2 in range(-(N - 1), N):
        for a1 in range(-(N - 1), N):
            g = G[a2 + N - 1, a1 + N - 1]
            if g == 0.0:
                continue
            # y[i2, i1] += g * x[i2 - a2, i1 - a1]
            i2lo, i2hi = max(0, a2), min(N, N + a2)
            i1lo, i1hi = max(0, a1), min(N, N + a1)
            y[i2lo:i2hi, i1lo:i1hi] += g * x[i2lo - a2:i2hi - a2, i1lo - a1:i1hi - a1]
    return y


def gram_apply_fft(G, x):
    """Same product by zero-padded 2N x 2N FFT convolution (numpy FFT, FP64)."""
    N = x.shape[0]
    L = 2 * N
    K = embed_circulant(G)
    xp = np.zeros((L, L))
    xp[:N, :N] = x
    y = np.fft.ifft2(np.fft.fft2(K) * np.fft.fft2(xp))
    return y.real[:N, :N]


def gram_apply_sampled(G, x, points):
    """y at selected output pixels (i2, i1) only, by the definition (for large-N parity)."""
    N = x.shape[0]
    out = []
    for i2, i1 in points:
        # G[i - j] for all j: offsets i - j range over the sub-block of G
        sub = G[i2:i2 + N, i1:i1 + N][::-1, ::-1]
        out.append(float(np.sum(sub * x)))
    return np.array(out)


def circulant_precond_symbol(G, eps):
    """Fourier symbol of the circulant preconditioner: 1 / max(G^, eps G^(0)) on the 2N x 2N grid.

    G is Toeplitz-block-Toeplitz (Sec. 4), so it is the N x N section of the 2N-periodic
    circulant C whose eigenvalues are the spectrum G^ of the embedded filter.  The
    preconditioner is the same section of C^-1.  G^ may dip slightly below zero for
    sparse angle sets (the truncated filter is not a positive symbol), so the symbol is
    floored at eps times its largest value G^(0) = sum of the taps (all taps are >= 0);
    that keeps the preconditioner symmetric positive definite for any eps in (0, 1].
    """
    if not 0.0 < eps <= 1.0:
        raise ValueError("eps must lie in (0, 1]")
    Ghat, _ = gram_spectrum(G)
    g0 = Ghat[0, 0]
    return 1.0 / np.maximum(Ghat, eps * g0)


def circulant_inverse_full(G, x, eps):
    """F^-1 diag(symbol) F applied to x zero-padded to 2N x 2N; the whole periodic field."""
    N = x.shape[0]
    L = 2 * N
    xp = np.zeros((L, L))
    xp[:N, :N] = x
    return np.fft.ifft2(np.fft.fft2(xp) * circulant_precond_symbol(G, eps)).real


def circulant_precond_apply(G, x, eps):
    """M^-1 x: the N x N crop of ``circulant_inverse_full`` (the section of C^-1)."""
    N = x.shape[0]
    return circulant_inverse_full(G, x, eps)[:N, :N]
