"""GPU parity of the circulant preconditioner and preconditioned CG (through the C ABI).

The preconditioner M^-1 = crop F^-1 diag(1 / max(G^, eps G^(0))) F pad is the N x N
section of the inverse of G's 2N-periodic circulant embedding (G is Toeplitz-block-
Toeplitz, Sec. 4).  Small sizes are compared element by element with the oracle; at the
bench size N = 2048 properties that hold at any size are checked: eps = 1 gives the
scaled identity, M^-1 is symmetric and positive, and PCG reaches its tolerance with a
true residual to match.

Tolerances (relative L2).  FP32 apply: 1e-5 (a CPU emulation with complex64 FFTs differs
from FP64 by ~1e-7 on these inputs).  FP64 apply: the FP64 spectrum carries absolute
rounding of ~u log2(4N^2) G^(0), which the floored reciprocal turns into relative error
up to that / eps in M^-1's symbol, so the gate is 10 u log2(4N^2) / eps, at least 1e-12
and at most 1e-11.  FP32 PCG iterates: the oracle's own FP64 PCG moves iterates 1 and 3
of the N = 128 problem by 2.7e-6 and 1.1e-5 when b is perturbed at the FP32 rounding
level (6e-8 relative; the circulant preconditioner amplifies it), so they are gated at
about four times that: 1e-5 and 4e-5.
"""
import math
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import backproject as obp  # noqa: E402
from oracle import cg as ocg  # noqa: E402
from oracle import gram as ogram  # noqa: E402
from workloads import ellipse_params, ellipse_sinogram, get_config, make_problem  # noqa: E402

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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("N,na,zeta,eps", [
    (16, 18, 1.0, 1e-3), (64, 90, 0.0, 1e-4), (64, 90, 1.0, 1e-2), (128, 180, 1.0, 1e-4), (128, 37, 0.5, 1.0),
])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_precond_apply_matches_oracle(bsct, N, na, zeta, eps, prec):
    angles = np.arange(na) / na
    f64 = prec == "f64"
    g = bsct.gram_build(bsct.Geometry(N, angles, 2 * N, 1.0, zeta), bsct.F64 if f64 else bsct.F32)
    G = ogram.gram_taps(N, angles, zeta)
    rng = np.random.default_rng(N + na)
    x = rng.standard_normal((N, N))
    if not f64:
        x = x.astype(np.float32).astype(np.float64)
    xd = torch.tensor(x, dtype=torch.float64 if f64 else torch.float32, device=DEV)
    y = g.precond_apply(xd, eps=eps).cpu().double().numpy()
    ref = ogram.circulant_precond_apply(G, x, eps)
    u64 = 2.0 ** -53
    tol64 = min(1e-11, max(1e-12, 10.0 * u64 * math.log2(4.0 * N * N) / eps))
    err = rel(y, ref)
    print(f"precond apply N={N} eps={eps} {prec}: {err:.2e}")
    assert err < (tol64 if f64 else 1e-5)
    # the spectrum is rebuilt when eps changes
    y2 = g.precond_apply(xd, eps=1.0).cpu().double().numpy()
    assert rel(y2, x / G.sum()) < (1e-12 if f64 else 2e-6)
    g.close()


def test_pcg_fp64_follows_oracle_iterates(bsct):
    cfg = get_config("fp64_n64")
    angles, sino, _ = make_problem(cfg)
    N, eps = cfg["N"], 1e-4
    g = bsct.gram_build(bsct.Geometry(N, angles, cfg["n_bins"], cfg["lambda_y"], cfg["zeta"]), bsct.F64)
    b_ref = obp.backproject(sino, N, angles, cfg["lambda_y"], cfg["zeta"])
    b = torch.tensor(b_ref, device=DEV)
    G = ogram.gram_taps(N, angles, cfg["zeta"])
    apply = lambda v: ogram.gram_apply_fft(G, v)
    minv = lambda v: ogram.circulant_precond_apply(G, v, eps)
    _, hist, iters = ocg.pcg(apply, minv, b_ref, iters=8)
    for k in (1, 2, 5):
        xk, rk = g.pcg_solve(b, max_iter=k, eps=eps)
        assert rk["iterations"] == k
        assert rel(xk.cpu().numpy(), iters[k - 1]) < 1e-9
        assert abs(rk["rel_residual"] - hist[k]) < 1e-8 * hist[k]
    x, rep = g.pcg_solve(b, max_iter=500, rel_tol=1e-8, check_every=1, eps=eps)
    assert rep["converged"] and rep["rel_residual"] <= 1e-8
    assert ocg.true_relative_residual(apply, b_ref, x.cpu().numpy()) < 2e-8
    _, crep = g.cg_solve(b, max_iter=2000, rel_tol=1e-8, check_every=1)
    assert crep["converged"] and 3 * rep["iterations"] < 2 * crep["iterations"]  # 44 against 95 in the oracle
    g.close()


def test_pcg_fp32_converges(bsct):
    N, na = 128, 180
    angles = np.arange(na) / na
    sino = ellipse_sinogram(ellipse_params(N, 20, seed=2), angles, 184, 1.0, 1.0)
    g = bsct.gram_build(bsct.Geometry(N, angles, 184, 1.0, 1.0), bsct.F32)
    bd = obp.backproject(sino, N, angles, 1.0, 1.0).astype(np.float32).astype(np.float64)
    b = torch.tensor(bd, dtype=torch.float32, device=DEV)
    G = ogram.gram_taps(N, angles, 1.0)
    apply = lambda v: ogram.gram_apply_fft(G, v)
    _, _, iters = ocg.pcg(apply, lambda v: ogram.circulant_precond_apply(G, v, 1e-4), bd, iters=3)
    for k, tol in ((1, 1e-5), (3, 4e-5)):
        xk, _ = g.pcg_solve(b, max_iter=k)
        err = rel(xk.cpu().numpy(), iters[k - 1])
        print(f"FP32 PCG iterate {k}: {err:.2e}")
        assert err < tol
    x, rep = g.pcg_solve(b, max_iter=500, rel_tol=1e-4, check_every=1)
    assert rep["converged"] and rep["rel_residual"] <= 1e-4
    r_final = ocg.true_relative_residual(apply, bd, x.cpu().double().numpy())
    assert r_final < 2e-4 and abs(rep["true_rel_residual"] - r_final) < 0.05 * r_final
    _, crep = g.cg_solve(b, max_iter=500, rel_tol=1e-4, check_every=1)
    assert rep["iterations"] * 2 < crep["iterations"]
    g.close()


def test_precond_and_pcg_at_bench_size(bsct):
    # N = 2048, 1800 views, zeta = 1 (the Gram-apply workload): properties at full size
    cfg = get_config("fp32_n2048")
    N, na = cfg["N"], cfg["n_angles"]
    g = bsct.gram_build(bsct.Geometry(N, np.arange(na) / na, cfg["n_bins"], cfg["lambda_y"], cfg["zeta"]), bsct.F32)
    gen = torch.Generator(device=DEV).manual_seed(7)
    a = torch.randn((N, N), device=DEV, generator=gen)
    c = torch.randn((N, N), device=DEV, generator=gen)
    g0 = float(g.spectrum()[0, 0])
    # eps = 1: every frequency floored at G^(0), M^-1 = I / G^(0)
    y1 = g.precond_apply(a, eps=1.0)
    assert rel(y1.cpu().numpy(), a.cpu().numpy() / g0) < 2e-6
    ma, mc = g.precond_apply(a), g.precond_apply(c)
    lhs, rhs = float((a.double() * mc.double()).sum()), float((ma.double() * c.double()).sum())
    assert abs(lhs - rhs) < 1e-5 * float((a.double() * ma.double()).sum())
    assert float((a.double() * ma.double()).sum()) > 0
    # PCG on b = G a reaches 1e-4; its true residual agrees
    b = g.apply(a)
    x, rep = g.pcg_solve(b, max_iter=400, rel_tol=1e-4, check_every=5)
    assert rep["converged"] and rep["true_rel_residual"] < 2e-4
    _, crep = g.cg_solve(b, max_iter=2000, rel_tol=1e-4, check_every=5)
    assert rep["iterations"] * 2 < crep["iterations"]
    g.close()


def test_pcg_degenerate_and_errors(bsct):
    N = 32
    g = bsct.gram_build(bsct.Geometry.uniform(N, 30, 48, 1.0, 1.0), bsct.F32)
    zero = torch.zeros((N, N), device=DEV)
    x, rep = g.pcg_solve(zero, max_iter=10, rel_tol=1e-4)
    assert rep["converged"] and rep["iterations"] == 0 and float(x.abs().max()) == 0.0
    x, rep = g.pcg_solve(zero, max_iter=3)  # no tolerance: three steps on a zero residual stay finite
    assert rep["iterations"] == 3 and float(x.abs().max()) == 0.0
    for bad in (0.0, -1e-3, 1.5):
        with pytest.raises(RuntimeError, match="invalid argument"):
            g.precond_apply(zero, eps=bad)
    g.close()


def test_steepest_descent_follows_oracle(bsct):
    cfg = get_config("fp64_n64")
    angles, sino, _ = make_problem(cfg)
    N = cfg["N"]
    g = bsct.gram_build(bsct.Geometry(N, angles, cfg["n_bins"], cfg["lambda_y"], cfg["zeta"]), bsct.F64)
    b_ref = obp.backproject(sino, N, angles, cfg["lambda_y"], cfg["zeta"])
    b = torch.tensor(b_ref, device=DEV)
    G = ogram.gram_taps(N, angles, cfg["zeta"])
    apply = lambda v: ogram.gram_apply_fft(G, v)
    _, hist, iters = ocg.steepest_descent(apply, b_ref, iters=20)
    for k in (1, 2, 5, 20):
        xk, rk = g.sd_solve(b, max_iter=k)
        assert rk["iterations"] == k
        assert rel(xk.cpu().numpy(), iters[k - 1]) < 1e-10
        assert abs(rk["rel_residual"] - hist[k]) < 1e-9 * hist[k]
    g.close()


def test_steepest_descent_fp32_converges(bsct):
    N, na = 128, 180
    angles = np.arange(na) / na
    sino = ellipse_sinogram(ellipse_params(N, 20, seed=2), angles, 184, 1.0, 1.0)
    g = bsct.gram_build(bsct.Geometry(N, angles, 184, 1.0, 1.0), bsct.F32)
    bd = obp.backproject(sino, N, angles, 1.0, 1.0).astype(np.float32).astype(np.float64)
    b = torch.tensor(bd, dtype=torch.float32, device=DEV)
    G = ogram.gram_taps(N, angles, 1.0)
    apply = lambda v: ogram.gram_apply_fft(G, v)
    _, hist, iters = ocg.steepest_descent(apply, bd, iters=5)
    for k in (1, 5):
        xk, _ = g.sd_solve(b, max_iter=k)
        assert rel(xk.cpu().numpy(), iters[k - 1]) < 1e-5
    x, rep = g.sd_solve(b, max_iter=3000, rel_tol=1e-3, check_every=10)
    assert rep["converged"]
    assert ocg.true_relative_residual(apply, bd, x.cpu().double().numpy()) < 1.2e-3
    g.close()


@pytest.mark.parametrize("method", ["cg", "pcg"])
@pytest.mark.parametrize("N,prec", [(16, 0), (128, 0), (64, 1)])
def test_solve_graph_matches_host_loop(bsct, method, N, prec):
    # the graph-driven solve runs the same iterations as the host-driven one and stops on
    # the device at the same iteration
    dt = torch.float32 if prec == bsct.F32 else torch.float64
    g = bsct.gram_build(bsct.Geometry.uniform(N, 60, int(1.42 * N) + 2, 1.0, 1.0), prec)
    x = torch.randn((N, N), dtype=dt, device=DEV, generator=torch.Generator(device=DEV).manual_seed(N + 1))
    b = g.apply(x)
    tol = 1e-4 if prec == bsct.F32 else 1e-9
    if method == "cg":
        xr, rr = g.cg_solve(b, max_iter=3000, rel_tol=tol, check_every=1)
    else:
        xr, rr = g.pcg_solve(b, max_iter=3000, rel_tol=tol, check_every=1)
    for _ in range(2):  # the second call replays the cached graph
        xg, rg = g.solve_graph(b, method=method, max_iter=3000, rel_tol=tol)
        assert rg["converged"] and rg["iterations"] == rr["iterations"]
        assert float((xg - xr).norm() / xr.norm()) < (1e-6 if prec == bsct.F32 else 1e-12)
        assert abs(rg["true_rel_residual"] - rr["true_rel_residual"]) < 0.05 * rr["true_rel_residual"]
    # a fixed number of iterations (no tolerance) and max_iter = 0
    xk, rk = g.solve_graph(b, method=method, max_iter=5, rel_tol=0.0)
    assert rk["iterations"] == 5
    _, r0 = g.solve_graph(b, method=method, max_iter=0, rel_tol=0.0)
    assert r0["iterations"] == 0
    g.close()
