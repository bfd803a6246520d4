"""Random-ellipse phantoms ("Spots" stand-in) and their analytic sinograms.

The paper's first test image is a set of randomly placed ellipses (Sec. 6); its exact
parameters are not given, so the distributions here are the named workload recipes:
centres U[-0.8, 0.8] * N/2, semi-axes U[2, 20] px, rotation U[0, pi), intensity
U[-0.5, 1], drawn per ellipse in the order (cx, cy, a, b, phi, rho) from
numpy's PCG64 seeded with ``seed + slice_id``.

Line integrals are the textbook chord of an ellipse; with a detector of width zeta
each sample is the cell average over [y_m - zeta/2, y_m + zeta/2] (closed-form
antiderivative).  Everything is FP64 on the host.
"""
import math

import numpy as np


def ellipse_params(N, n_ellipses, seed, slice_id=0):
    """Array [n, 6] of (cx, cy, a, b, phi, rho) in pixel units (image centre at 0)."""
    rng = np.random.default_rng(seed + slice_id)
    out = np.empty((n_ellipses, 6))
    for e in range(n_ellipses):
        cx = rng.uniform(-0.8, 0.8) * N / 2.0
        cy = rng.uniform(-0.8, 0.8) * N / 2.0
        a = rng.uniform(2.0, 20.0)
        b = rng.uniform(2.0, 20.0)
        phi = rng.uniform(0.0, math.pi)
        rho = rng.uniform(-0.5, 1.0)
        out[e] = (cx, cy, a, b, phi, rho)
    return out


def _angles(angles_pi):
    a = np.asarray(angles_pi, dtype=np.float64)
    th = np.pi * a
    c, s = np.cos(th), np.sin(th)
    # exact axis-aligned values (matches the detector geometry used everywhere)
    two = 2 * a
    ex = two == np.round(two)
    q = np.mod(np.round(two[ex]).astype(int), 4)
    c[ex] = np.array([1.0, 0.0, -1.0, 0.0])[q]
    s[ex] = np.array([0.0, 1.0, 0.0, -1.0])[q]
    return c, s


def ellipse_sinogram(params, angles_pi, M, lambda_y, zeta=0.0):
    """Sinogram [n_angles, M] of the ellipse set: point samples (zeta = 0) or cell averages."""
    c, s = _angles(angles_pi)
    ym = (np.arange(M) - (M - 1) / 2.0) * lambda_y
    sino = np.zeros((len(c), M))
    for cx, cy, a, b, phi, rho in params:
        cr = c * math.cos(phi) + s * math.sin(phi)   # cos(theta - phi)
        sr = s * math.cos(phi) - c * math.sin(phi)   # sin(theta - phi)
        r2 = a * a * cr * cr + b * b * sr * sr
        r = np.sqrt(r2)
        t = ym[None, :] - (cx * c + cy * s)[:, None]
        scale = 2.0 * rho * a * b / r2
        if zeta == 0.0:
            sino += np.where(np.abs(t) < r[:, None],
                             scale[:, None] * np.sqrt(np.clip(r2[:, None] - t * t, 0.0, None)), 0.0)
        else:
            def F(u):
                u = np.clip(u, -r[:, None], r[:, None])
                return 0.5 * (u * np.sqrt(np.clip(r2[:, None] - u * u, 0.0, None))
                              + r2[:, None] * np.arcsin(np.clip(u / r[:, None], -1.0, 1.0)))
            sino += scale[:, None] * (F(t + 0.5 * zeta) - F(t - 0.5 * zeta)) / zeta
    return sino


def ellipse_image(params, N, supersample=4):
    """Pixel-average rasterisation of the ellipse set (diagnostics only)."""
    k = (np.arange(N * supersample) + 0.5) / supersample - N / 2.0
    X, Y = np.meshgrid(k, k)
    img = np.zeros((N * supersample, N * supersample))
    for cx, cy, a, b, phi, rho in params:
        xr = (X - cx) * math.cos(phi) + (Y - cy) * math.sin(phi)
        yr = -(X - cx) * math.sin(phi) + (Y - cy) * math.cos(phi)
        img += rho * ((xr / a) ** 2 + (yr / b) ** 2 <= 1.0)
    return img.reshape(N, supersample, N, supersample).mean(axis=(1, 3))


def poisson_log_sinogram(sino, I0, seed):
    """Poisson counting noise on transmitted counts, then -log (Sec. 6.3 analogue).

    Line integrals of unit-density pixels reach tens, so exp(-p) * I0 would
    underflow; the sinogram is scaled by alpha = 4 / max(p) before attenuation and
    the noisy log data are scaled back.  Counts are clamped >= 1.
    """
    rng = np.random.default_rng(seed)
    pmax = float(np.max(np.abs(sino)))
    alpha = 4.0 / pmax if pmax > 0 else 1.0
    counts = rng.poisson(I0 * np.exp(-alpha * sino))
    counts = np.maximum(counts, 1)
    return -np.log(counts / I0) / alpha


def make_problem(cfg, slice_id=0, noise=True):
    """(angles_pi, sinogram, params) for a workload config dict (see configs.py)."""
    N = cfg["N"]
    angles = np.arange(cfg["n_angles"], dtype=np.float64) / cfg["n_angles"]
    params = ellipse_params(N, cfg["n_ellipses"], cfg.get("seed", 0), slice_id)
    sino = ellipse_sinogram(params, angles, cfg["n_bins"], cfg["lambda_y"], cfg["zeta"])
    if noise and cfg.get("I0"):
        sino = poisson_log_sinogram(sino, cfg["I0"], cfg.get("seed", 0) + 1000 + slice_id)
    return angles, sino, params


def ellipse_sinogram_torch(params, angles_pi, M, lambda_y, zeta=0.0, device="cuda", dtype=None):
    """Same analytic sinogram as ``ellipse_sinogram`` evaluated with torch on a device
    (used to synthesise many large batch inputs quickly).  The ellipses' chord terms are
    formed together in blocks (the same FP64 operations, element by element, as one
    ellipse at a time) and added to the sinogram in the parameters' order."""
    import torch

    dtype = dtype or torch.float64
    c_np, s_np = _angles(angles_pi)
    c = torch.tensor(c_np, dtype=torch.float64, device=device)[None, :]
    s = torch.tensor(s_np, dtype=torch.float64, device=device)[None, :]
    ym = (torch.arange(M, dtype=torch.float64, device=device) - (M - 1) / 2.0) * lambda_y
    sino = torch.zeros((len(c_np), M), dtype=torch.float64, device=device)
    params = [tuple(float(v) for v in p) for p in params]
    block = max(1, (1 << 25) // max(1, len(c_np) * M))
    for e0 in range(0, len(params), block):
        P = params[e0:e0 + block]

        def col(v):
            return torch.tensor(v, dtype=torch.float64, device=device)[:, None]

        cx, cy = col([p[0] for p in P]), col([p[1] for p in P])
        a, b, rho = col([p[2] for p in P]), col([p[3] for p in P]), col([p[5] for p in P])
        cphi, sphi = col([math.cos(p[4]) for p in P]), col([math.sin(p[4]) for p in P])
        aa, bb = col([p[2] * p[2] for p in P]), col([p[3] * p[3] for p in P])
        sc2 = col([2.0 * p[5] * p[2] * p[3] for p in P])
        cr = c * cphi + s * sphi
        sr = s * cphi - c * sphi
        r2 = (aa * cr * cr + bb * sr * sr)[:, :, None]
        r = torch.sqrt(r2)
        t = ym[None, None, :] - (cx * c + cy * s)[:, :, None]
        scale = r2.reciprocal() * sc2[:, :, None]  # as torch evaluates number / tensor
        if zeta == 0.0:
            term = torch.where(t.abs() < r, scale * torch.sqrt(torch.clamp(r2 - t * t, min=0.0)),
                               torch.zeros_like(t))
        else:
            def F(u):
                u = torch.maximum(torch.minimum(u, r), -r)
                return 0.5 * (u * torch.sqrt(torch.clamp(r2 - u * u, min=0.0))
                              + r2 * torch.asin(torch.clamp(u / r, -1.0, 1.0)))
            term = scale * (F(t + 0.5 * zeta) - F(t - 0.5 * zeta)) / zeta
        for k in range(len(P)):
            sino += term[k]
    return sino.to(dtype)


def poisson_log_sinogram_torch(sino, I0, generator):
    """Torch version of ``poisson_log_sinogram`` (same scaling reading), for device tensors."""
    import torch

    pmax = float(sino.abs().max())
    alpha = 4.0 / pmax if pmax > 0 else 1.0
    counts = torch.poisson(I0 * torch.exp(-alpha * sino.double()), generator=generator)
    counts = torch.clamp(counts, min=1.0)
    return (-torch.log(counts / I0) / alpha).to(sino.dtype)
