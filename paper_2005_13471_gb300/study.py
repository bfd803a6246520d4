"""Reconstruction accuracy study on synthetic ellipse phantoms (Sec. 6, box-spline curves).

The paper measures unregularised reconstructions by SNR (dB) and SSIM against the ground
truth while the detector sampling step lambda_y (the "downsampling rate", image pixels
being unit) goes from 0.25 to 2 and while Gaussian noise is added to the sinogram; the
reconstruction solves the normal equations G c = H^T g_hat (Sec. 2) by steepest descent.
Here the sinogram is the exact (analytic) blurred X-ray transform of a random-ellipse
phantom, so the data do not come from the pixel model (no inverse crime), and the ground
truth is the phantom's pixel-basis representation: its average over each pixel,
computed from 10 x 10 subsamples (the paper uses a ten times finer grid).

Every step on the GPU goes through the library (back projection, Gram filter, solver);
the metrics are evaluated on the host.
"""
import math

import numpy as np

SSIM_K1, SSIM_K2, SSIM_SIGMA, SSIM_RADIUS = 0.01, 0.03, 1.5, 5


def snr_db(truth, x):
    """10 log10(||truth||^2 / ||truth - x||^2)."""
    t = np.asarray(truth, dtype=np.float64)
    e = t - np.asarray(x, dtype=np.float64)
    den = float(np.sum(e * e))
    return math.inf if den == 0.0 else 10.0 * math.log10(float(np.sum(t * t)) / den)


def _gauss_filter(img):
    # separable normalised Gaussian window, sigma 1.5, radius 5 (11 taps), valid region
    k = np.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=np.float64)
    w = np.exp(-0.5 * (k / SSIM_SIGMA) ** 2)
    w /= w.sum()
    rows = np.apply_along_axis(lambda r: np.convolve(r, w, mode="valid"), 1, img)
    return np.apply_along_axis(lambda c: np.convolve(c, w, mode="valid"), 0, rows)


def ssim(truth, x, data_range=None):
    """Mean structural similarity (Wang, Bovik, Sheikh, Simoncelli 2004): local means,
    variances and covariance under an 11 x 11 Gaussian window (sigma 1.5), constants
    C1 = (0.01 L)^2 and C2 = (0.03 L)^2 with L the truth's dynamic range, averaged over
    the windows that lie inside the image."""
    t = np.asarray(truth, dtype=np.float64)
    y = np.asarray(x, dtype=np.float64)
    L = float(t.max() - t.min()) if data_range is None else float(data_range)
    c1, c2 = (SSIM_K1 * L) ** 2, (SSIM_K2 * L) ** 2
    mt, my = _gauss_filter(t), _gauss_filter(y)
    vt = _gauss_filter(t * t) - mt * mt
    vy = _gauss_filter(y * y) - my * my
    cty = _gauss_filter(t * y) - mt * my
    s = ((2 * mt * my + c1) * (2 * cty + c2)) / ((mt * mt + my * my + c1) * (vt + vy + c2))
    return float(s.mean())


def detector_bins(N, lambda_y, zeta):
    """Samples covering the image's diagonal plus the footprint on both sides."""
    return int(math.ceil((N * math.sqrt(2.0) + 2.0 + zeta) / lambda_y)) + 2


def reconstruct(bsct, N, n_views, lambda_y, zeta, sino, solver="sd", iters=100, rel_tol=0.0):
    """b = H^T g_hat, then `iters` solver steps on G c = b (F32 path)."""
    import torch

    angles = np.arange(n_views, dtype=np.float64) / n_views
    geom = bsct.Geometry(N, angles, sino.shape[1], lambda_y, zeta)
    s = torch.tensor(sino, dtype=torch.float32, device="cuda")
    b = bsct.backproject(geom, s, bsct.F32)
    g = bsct.gram_build(geom, bsct.F32)
    try:
        if solver == "sd":
            x, rep = g.sd_solve(b, max_iter=iters, rel_tol=rel_tol)
        elif solver == "pcg":
            x, rep = g.pcg_solve(b, max_iter=iters, rel_tol=rel_tol)
        else:
            x, rep = g.cg_solve(b, max_iter=iters, rel_tol=rel_tol)
        torch.cuda.synchronize()
        return x.cpu().double().numpy(), rep
    finally:
        g.close()


def accuracy_sweep(bsct, N=256, n_views=180, zeta=1.0, lambdas=(0.25, 0.5, 1.0, 1.5, 2.0),
                   noise=(0.0, 0.01, 0.05), solver="sd", iters=100, n_ellipses=30, seed=0):
    """SNR / SSIM of reconstructions over detector steps and Gaussian noise levels.

    noise: standard deviation of the added Gaussian noise relative to the largest
    noise-free sample.  Returns a list of dicts, one per (lambda_y, noise) pair.
    """
    from workloads import ellipse_image, ellipse_params, ellipse_sinogram

    params = ellipse_params(N, n_ellipses, seed)
    truth = ellipse_image(params, N, supersample=10)
    angles = np.arange(n_views, dtype=np.float64) / n_views
    rng = np.random.default_rng(seed + 1)
    out = []
    for lam in lambdas:
        M = detector_bins(N, lam, zeta)
        clean = ellipse_sinogram(params, angles, M, lam, zeta)
        peak = float(np.abs(clean).max())
        for sigma in noise:
            sino = clean + sigma * peak * rng.standard_normal(clean.shape) if sigma > 0 else clean
            x, rep = reconstruct(bsct, N, n_views, lam, zeta, sino, solver, iters)
            out.append({"lambda_y": lam, "noise": sigma, "bins": M, "snr_db": snr_db(truth, x),
                        "ssim": ssim(truth, x), "iterations": rep["iterations"]})
    return out
