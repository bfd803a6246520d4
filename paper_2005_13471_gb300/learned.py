"""Learned CG warm start: training data from the method itself, training, evaluation.

Pairs (back projection b, converged reconstruction x) are produced by the library on
seeded random-ellipse phantoms with Poisson noise: b by bsct_backproject, x by the
batched graph solver (bsct_batch_solve) running `cg_iters` CG iterations.  The network
input is b / n_views (b grows with the number of views), the target is x.  Training
uses the library's forward / backward / Adam kernels; this module only orchestrates
(selects minibatches, calls the entry points, records losses).
"""
import math
import time

import numpy as np

import paper_2005_13471_gb300 as bsct


def _phantom_sinograms(n, N, angles, n_bins, zeta, I0, seed, device, n_ellipses=40):
    import torch

    from workloads.phantom import ellipse_params, ellipse_sinogram_torch, poisson_log_sinogram_torch

    gen = torch.Generator(device=device).manual_seed(seed)
    out = []
    for i in range(n):
        p = ellipse_params(N, n_ellipses, seed, slice_id=i)
        s = ellipse_sinogram_torch(p, angles, n_bins, 1.0, zeta, device=device, dtype=torch.float64)
        if I0:
            s = poisson_log_sinogram_torch(s, I0, gen)
        out.append(s.float())
    return out


def generate_pairs(n_pairs, N=256, n_angles=360, n_bins=364, zeta=1.0, I0=1e5, cg_iters=200, chunk=128, seed=0,
                   device="cuda"):
    """Inputs b / n_views and targets x (CG after cg_iters iterations), each [n_pairs, N, N] on the device."""
    import torch

    angles = np.arange(n_angles) / n_angles
    geom = bsct.Geometry(N, angles, n_bins, 1.0, zeta)
    chunk = min(chunk, n_pairs)
    batch = bsct.Batch([geom] * chunk)
    sino_buf = [torch.empty((n_angles, n_bins), dtype=torch.float32, device=device) for _ in range(chunk)]
    x_buf = [torch.empty((N, N), dtype=torch.float32, device=device) for _ in range(chunk)]
    X = torch.empty((n_pairs, N, N), dtype=torch.float32, device=device)
    Y = torch.empty((n_pairs, N, N), dtype=torch.float32, device=device)
    work = torch.empty(bsct.backproject_workspace(geom, bsct.F32), dtype=torch.uint8, device=device)
    for c0 in range(0, n_pairs, chunk):
        m = min(chunk, n_pairs - c0)
        sinos = _phantom_sinograms(m, N, angles, n_bins, zeta, I0, seed * 1_000_003 + c0, device)
        for i in range(chunk):
            sino_buf[i].copy_(sinos[i] if i < m else sinos[0])
        batch.solve(sino_buf, xs=x_buf, cg_iters=cg_iters)
        for i in range(m):
            bsct.backproject(geom, sino_buf[i], bsct.F32, out=X[c0 + i], work=work)
            Y[c0 + i].copy_(x_buf[i])
        X[c0:c0 + m] *= 1.0 / n_angles
    torch.cuda.synchronize()
    batch.close()
    return X, Y


def gnorm_weights(gram, Y, chunk=64):
    """Per-target weights 1 / <y, G y> (FP64, device) that make the G-norm loss relative."""
    import torch

    n = Y.shape[0]
    w = torch.empty(n, dtype=torch.float64, device=Y.device)
    zero = torch.zeros((min(chunk, n),) + tuple(Y.shape[1:]), dtype=torch.float32, device=Y.device)
    grad = torch.empty_like(zero)
    acc = torch.zeros(1, dtype=torch.float64, device=Y.device)
    for i in range(n):
        acc.zero_()
        bsct.gnorm_loss_grad(gram, Y[i:i + 1], zero[:1], grad[:1], acc)
        w[i] = 1.0 / acc[0].clamp_min(1e-300)
    return w


def train(net, X, Y, epochs=1, batch_size=8, lr=1e-3, lr_final=1e-4, seed=0, log_every=0, loss="mse", gram=None,
          weights=None):
    """Adam on the mean-squared error (loss="mse") or on the relative G-norm error
    <e, G e> / <y, G y> (loss="gnorm": the norm CG minimises; gram = the Gram filter of the
    training geometry, weights = gnorm_weights(gram, Y)); returns the per-step losses."""
    import torch

    if loss not in ("mse", "gnorm") or (loss == "gnorm" and (gram is None or weights is None)):
        raise ValueError("loss must be 'mse', or 'gnorm' with gram and weights")
    n = X.shape[0]
    gen = torch.Generator(device="cpu").manual_seed(seed)
    steps_per_epoch = n // batch_size
    total = max(1, epochs * steps_per_epoch)
    grad = torch.empty((batch_size,) + tuple(X.shape[1:]), dtype=torch.float32, device=X.device)
    loss_acc = torch.zeros(1, dtype=torch.float64, device=X.device)
    losses = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen).to(X.device)
        for s in range(steps_per_epoch):
            idx = perm[s * batch_size:(s + 1) * batch_size]
            xb = X.index_select(0, idx)
            yb = Y.index_select(0, idx)
            pred = net.forward(xb)
            loss_acc.zero_()
            if loss == "mse":
                bsct.mse_loss_grad(pred, yb, grad, loss_acc)
            else:
                bsct.gnorm_loss_grad(gram, pred.contiguous(), yb, grad, loss_acc, weights.index_select(0, idx))
            net.backward(grad)
            step += 1
            # cosine decay from lr to lr_final
            cur = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * step / total))
            net.adam_step(cur, step)
            if log_every and step % log_every == 0:
                losses.append(float(loss_acc.item()))
    torch.cuda.synchronize()
    return losses


def compare_solvers(net, gram, b, n_views, rel_tol=1e-4, max_iter=2000, check_every=5):
    """Wall time and iterations to rel_tol for plain CG and for the learned warm start."""
    import torch

    gram.cg_solve(b, max_iter=5)  # warm the kernels
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xp, rp = gram.cg_solve(b, max_iter=max_iter, rel_tol=rel_tol, check_every=check_every)
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    gram.cg_solve_learned(net, b, 1.0 / n_views, max_iter=5, rel_tol=0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xl, rl = gram.cg_solve_learned(net, b, 1.0 / n_views, max_iter=max_iter, rel_tol=rel_tol, check_every=check_every)
    torch.cuda.synchronize()
    tl = time.perf_counter() - t0
    return dict(plain_ms=1e3 * tp, plain_iters=rp["iterations"], plain_true=rp["true_rel_residual"],
                learned_ms=1e3 * tl, learned_iters=rl["iterations"], learned_true=rl["true_rel_residual"],
                alpha=rl["alpha"]), xp, xl
