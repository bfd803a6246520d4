"""Learned warm start: the library's CNN forward / backward kernels against the FP64
CPU oracle (same BF16 rounding points), the Adam update, and the gain of the trained
network over plain CG (judged by plain CG's own residual)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet as ounet  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def bsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_13471_gb300 as m

    m.lib()
    return m


def rel(a, b):
    return float((a - b).norm() / b.norm())


def test_unet_forward_backward_vs_oracle(bsct):
    # Tolerances: both sides round the same values to BF16, but a value computed with
    # FP32 accumulation can round to the neighbouring BF16 number (2^-8 apart) where
    # the FP64 value does not; such flips compound over the 17 layers (measured forward
    # agreement 2.3e-3).  The backward pass adds discrete decisions taken on those
    # slightly different forward values (ReLU masks near zero, max-pool argmax between
    # near-equal inputs), measured 4.7e-2 over all parameters.  An indexing error in any
    # kernel gives O(1) differences; the GEMM itself is checked at 1e-5 elsewhere.
    base, nb, H = 8, 2, 64
    net = bsct.UNet(base_channels=base, seed=3)
    _, _, n = ounet.layout(base)
    assert net.n_params == n
    g = torch.Generator().manual_seed(0)
    x = torch.randn((nb, H, H), generator=g)
    gout = torch.randn((nb, H, H), generator=g) * 1e-2
    out = net.forward(x.to(DEV)).cpu()
    net.backward(gout.to(DEV))
    grads = net.get_grads().cpu().double()
    params = net.get_params().cpu()
    tensors, head = ounet.unpack(params, base)
    ref = ounet.forward(x.double(), tensors, head)
    err_f = rel(out.double(), ref.detach())
    ref.backward(gout.double())
    gref = ounet.pack_grads(tensors, head, base)
    err_g = rel(grads, gref)
    print(f"U-Net vs FP64 oracle: forward {err_f:.2e}, parameter gradients {err_g:.2e}")
    assert err_f < 5e-3
    assert err_g < 1e-1
    # per-layer groups: every layer's gradient agrees on its own
    layers, hd, _ = ounet.layout(base)
    for L in layers:
        sl = slice(L["w"], L["b"] + L["cout"])
        assert rel(grads[sl], gref[sl]) < 2.5e-1, L
    net.close()


def test_adam_step(bsct):
    net = bsct.UNet(base_channels=8, seed=1)
    x = torch.randn((1, 64, 64), device=DEV)
    net.forward(x)
    net.backward(torch.randn((1, 64, 64), device=DEV) * 1e-2)
    w0 = net.get_params().double()
    g0 = net.get_grads().double()
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    net.adam_step(lr, 1, b1, b2, eps)
    w1 = net.get_params().double()
    m = (1 - b1) * g0
    v = (1 - b2) * g0 * g0
    ref = w0 - lr * (m / (1 - b1)) / (torch.sqrt(v / (1 - b2)) + eps)
    assert float((w1 - ref).abs().max()) < 1e-6
    assert float(net.get_grads().abs().max()) == 0.0
    net.close()


def test_learned_warm_start_gain(bsct):
    # Trains a small network on pairs the method generates, then measures what its warm
    # start buys: the starting residual (vs 1 for x0 = 0) and the iterations / time to a
    # 1e-4 relative residual, with plain CG as the reference (both must reach the tolerance
    # by the FP32 true residual).  An untrained network falls back to plain CG.
    from paper_2005_13471_gb300 import learned

    N, na, M = 64, 90, 92
    X, Y = learned.generate_pairs(384, N=N, n_angles=na, n_bins=M, zeta=1.0, I0=1e5, cg_iters=200, chunk=128, seed=0)
    net = bsct.UNet(base_channels=32, seed=0)
    losses = learned.train(net, X, Y, epochs=6, batch_size=8, lr=2e-3, lr_final=1e-4, log_every=24)
    assert losses[-1] < 0.5 * losses[0]
    geom = bsct.Geometry(N, np.arange(na) / na, M, 1.0, 1.0)
    g = bsct.gram_build(geom, bsct.F32)
    Xe, _ = learned.generate_pairs(6, N=N, n_angles=na, n_bins=M, zeta=1.0, I0=1e5, cg_iters=1, chunk=6, seed=99)
    rows = []
    for i in range(Xe.shape[0]):
        b = (Xe[i] * na).contiguous()
        r, _, _ = learned.compare_solvers(net, g, b, na)
        assert r["learned_true"] <= 1.2e-4 and r["plain_true"] <= 1.2e-4
        x0 = r["alpha"] * net.forward((b / na).unsqueeze(0))[0]
        r0 = float((b - g.apply(x0)).norm() / b.norm())
        rows.append((r0, r["plain_iters"], r["learned_iters"], r["plain_ms"], r["learned_ms"]))
    print("warm-start residual, iterations plain/learned, ms plain/learned:", rows)
    assert np.mean([row[0] for row in rows]) < 0.5  # the warm start beats x0 = 0 by this measure
    # the same network as flexible-CG preconditioner: reaches the tolerance (by the FP32
    # true residual) with the network applied every iteration and every 4th
    b = (Xe[1] * na).contiguous()
    _, rp = g.cg_solve(b, max_iter=2000, rel_tol=1e-4, check_every=1)
    fc = []
    for every in (1, 4):
        _, rf = g.fcg_solve_learned(net, b, 1.0 / na, max_iter=2000, rel_tol=1e-4, precond_every=every)
        assert rf["converged"] and rf["true_rel_residual"] <= 1.2e-4
        assert rf["n_precond"] == (rf["iterations"] - 1) // every + 1
        fc.append((every, rf["iterations"], rf["n_precond"], rf["n_fallback"]))
    print("flexible CG (every, iterations, network applications, fallbacks) vs plain", rp["iterations"], fc)
    # fallback: a network whose output is useless (alpha <= 0) leaves plain CG unchanged
    bad = bsct.UNet(base_channels=8, seed=5)
    bad.set_params(torch.zeros(bad.n_params, device=DEV))
    b = (Xe[0] * na).contiguous()
    _, rp = g.cg_solve(b, max_iter=2000, rel_tol=1e-4, check_every=5)
    _, rl = g.cg_solve_learned(bad, b, 1.0 / na, max_iter=2000, rel_tol=1e-4, check_every=5)
    assert rl["alpha"] == 0.0 and rl["iterations"] == rp["iterations"]
    # ... and as a preconditioner (<r, z> = 0) falls back to the identity every time, which
    # makes flexible CG the same method as CG in exact arithmetic.  In FP32 the two take
    # their scalars from different products (flexible: alpha = <p, r> / <p, Gp>, beta =
    # -<z, Gp> / <p, Gp>; CG: <r, r>-ratios), which lose orthogonality differently on this
    # ill-conditioned G, so the iterations to 1e-4 differ by a few (32 against 35 seen after
    # a rounding-level change of b): within 15 %
    _, rp1 = g.cg_solve(b, max_iter=2000, rel_tol=1e-4, check_every=1)
    _, rf = g.fcg_solve_learned(bad, b, 1.0 / na, max_iter=2000, rel_tol=1e-4, precond_every=1)
    assert rf["converged"] and rf["n_fallback"] == rf["n_precond"] == rf["iterations"]
    assert abs(rf["iterations"] - rp1["iterations"]) <= max(2, 0.15 * rp1["iterations"])
    # warm start followed by circulant-preconditioned CG: reaches the tolerance; with the
    # useless network it is PCG from x0 = 0 exactly
    b = (Xe[2] * na).contiguous()
    _, rz = g.pcg_solve(b, max_iter=500, rel_tol=1e-4, check_every=1)
    _, rw = g.pcg_solve_learned(net, b, 1.0 / na, max_iter=500, rel_tol=1e-4, check_every=1)
    assert rw["converged"] and rw["true_rel_residual"] <= 1.2e-4
    print("PCG iterations from 0 / from the warm start:", rz["iterations"], rw["iterations"])
    _, rb = g.pcg_solve_learned(bad, b, 1.0 / na, max_iter=500, rel_tol=1e-4, check_every=1)
    assert rb["alpha"] == 0.0 and rb["iterations"] == rz["iterations"]
    g.close()
    net.close()
    bad.close()


def test_gnorm_loss_against_oracle(bsct):
    # the G-norm training loss: loss = (1/n) sum_i w_i <e_i, G e_i>, grad_i = (2 w_i / n) G e_i,
    # e = pred - target, against the FP64 oracle's Gram apply on the same FP32 inputs
    from oracle import gram as ogram

    N, na, n = 64, 30, 3
    angles = np.arange(na) / na
    g = bsct.gram_build(bsct.Geometry(N, angles, 92, 1.0, 1.0), bsct.F32)
    G = ogram.gram_taps(N, angles, 1.0)
    gen = torch.Generator().manual_seed(11)
    pred = torch.randn((n, N, N), generator=gen)
    target = torch.randn((n, N, N), generator=gen)
    w = torch.tensor([0.5, 1.0, 2.0], dtype=torch.float64)
    grad = torch.empty((n, N, N), device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    bsct.gnorm_loss_grad(g, pred.to(DEV), target.to(DEV), grad, loss, w.to(DEV))
    e = (pred - target).double().numpy()
    ge = np.stack([ogram.gram_apply_fft(G, e[i]) for i in range(n)])
    ref_loss = sum(float(w[i]) * float((e[i] * ge[i]).sum()) for i in range(n)) / n
    ref_grad = np.stack([2.0 * float(w[i]) / n * ge[i] for i in range(n)])
    assert abs(float(loss.item()) - ref_loss) < 1e-5 * abs(ref_loss)
    err = np.linalg.norm(grad.cpu().double().numpy() - ref_grad) / np.linalg.norm(ref_grad)
    assert err < 1e-5
    # accumulates, and runs in a fixed order: a second call adds the same value exactly
    first = float(loss.item())
    bsct.gnorm_loss_grad(g, pred.to(DEV), target.to(DEV), grad, loss, w.to(DEV))
    assert float(loss.item()) == 2 * first
    g.close()


def test_training_and_solvers_are_bit_reproducible(bsct):
    # every reduction of the CNN and of the learned solvers sums in a fixed order (per-block
    # partials added in block order), so the same inputs give the same bits on every run:
    # two networks from the same seed after a forward / backward / Adam step, the MSE loss,
    # the warm start and flexible CG
    def step():
        net = bsct.UNet(base_channels=8, seed=11)
        g = torch.Generator().manual_seed(4)
        x = torch.randn((4, 64, 64), generator=g).to(DEV)
        target = torch.randn((4, 64, 64), generator=g).to(DEV)
        pred = net.forward(x)
        grad = torch.empty_like(pred)
        loss = torch.zeros(1, dtype=torch.float64, device=DEV)
        bsct.mse_loss_grad(pred, target, grad, loss)
        net.backward(grad)
        grads = net.get_grads().clone()
        net.adam_step(1e-3, 1)
        params = net.get_params().clone()
        return net, grads, params, loss.clone()

    net1, g1, p1, l1 = step()
    net2, g2, p2, l2 = step()
    assert torch.equal(g1, g2) and torch.equal(p1, p2) and torch.equal(l1, l2)
    N, na = 64, 90
    geom = bsct.Geometry(N, np.arange(na) / na, 92, 1.0, 1.0)
    gm = bsct.gram_build(geom, bsct.F32)
    b = gm.apply(torch.randn((N, N), generator=torch.Generator().manual_seed(7)).to(DEV))
    xa, ra = gm.cg_solve_learned(net1, b, 1.0 / na, max_iter=60, rel_tol=0.0, check_every=5)
    xb, rb = gm.cg_solve_learned(net2, b, 1.0 / na, max_iter=60, rel_tol=0.0, check_every=5)
    assert ra["alpha"] == rb["alpha"] and torch.equal(xa, xb)
    fa, _ = gm.fcg_solve_learned(net1, b, 1.0 / na, max_iter=40, rel_tol=0.0, precond_every=2)
    fb, _ = gm.fcg_solve_learned(net2, b, 1.0 / na, max_iter=40, rel_tol=0.0, precond_every=2)
    assert torch.equal(fa, fb)
    gm.close()
    net1.close()
    net2.close()
