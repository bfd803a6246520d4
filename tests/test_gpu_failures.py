"""Failure paths of the C ABI on the GPU, made on the host: non-finite inputs and a solve
that cannot converge within its iteration budget.

A NaN or infinity in the right-hand side or initial guess of a synchronous solver is
reported as BSCT_ERR_NONFINITE before the first iteration; the asynchronous calls (Gram
apply, back projection, forward projection) flag non-finite inputs in the library's input
status, read and cleared by bsct_input_status.  max_iter too small for rel_tol > 0 returns
BSCT_WARN_NOT_CONVERGED with the iterate and an honest report.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def bsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_13471_gb300 as m

    m.lib()
    assert m.input_status() == m.OK  # clear what earlier tests left
    return m


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_async_calls_flag_nonfinite_inputs(bsct, bad, prec):
    f32 = prec == "f32"
    P = bsct.F32 if f32 else bsct.F64
    dt = torch.float32 if f32 else torch.float64
    N, na, M = 64, 30, 92
    geom = bsct.Geometry.uniform(N, na, M, 1.0, 1.0)
    g = bsct.gram_build(geom, P)
    x = torch.randn((N, N), dtype=dt, device=DEV)
    g.apply(x)
    assert bsct.input_status() == bsct.OK
    x[17, 5] = bad
    g.apply(x)
    assert bsct.input_status() == bsct.ERR_NONFINITE
    assert bsct.input_status() == bsct.OK  # reading clears it
    sino = torch.randn((na, M), dtype=dt, device=DEV)
    bsct.backproject(geom, sino, P)
    assert bsct.input_status() == bsct.OK
    sino[na - 1, M - 1] = bad
    bsct.backproject(geom, sino, P)
    assert bsct.input_status() == bsct.ERR_NONFINITE
    c = torch.randn((N, N), dtype=dt, device=DEV)
    bsct.forward_project(geom, c, P)
    assert bsct.input_status() == bsct.OK
    c[0, 0] = bad
    bsct.forward_project(geom, c, P)
    assert bsct.input_status() == bsct.ERR_NONFINITE
    assert bsct.check_finite(x) is False and bsct.check_finite(torch.ones(5, dtype=dt, device=DEV)) is True
    g.close()


def test_dftgemm_apply_flags_nonfinite_input(bsct):
    N = 64
    g = bsct.gram_build(bsct.Geometry.uniform(N, 30, 92, 1.0, 1.0), bsct.F32)
    x = torch.randn((N, N), device=DEV)
    x[3, 3] = float("nan")
    g.apply(x, mode=bsct.APPLY_DFTGEMM_BF16)
    assert bsct.input_status() == bsct.ERR_NONFINITE
    g.close()


@pytest.mark.parametrize("where", ["b", "x0"])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_solvers_reject_nonfinite_start(bsct, where, prec):
    f32 = prec == "f32"
    dt = torch.float32 if f32 else torch.float64
    N = 64
    g = bsct.gram_build(bsct.Geometry.uniform(N, 30, 92, 1.0, 1.0), bsct.F32 if f32 else bsct.F64)
    b = torch.randn((N, N), dtype=dt, device=DEV)
    x0 = torch.zeros((N, N), dtype=dt, device=DEV)
    if where == "b":
        b[10, 20] = float("nan")
    else:
        x0[1, 2] = float("inf")
    for tol in (0.0, 1e-4):  # with and without a stopping test
        with pytest.raises(RuntimeError, match="non-finite"):
            g.cg_solve(b, x0=x0, max_iter=5, rel_tol=tol)
        with pytest.raises(RuntimeError, match="non-finite"):
            g.pcg_solve(b, x0=x0, max_iter=5, rel_tol=tol)
        with pytest.raises(RuntimeError, match="non-finite"):
            g.sd_solve(b, x0=x0, max_iter=5, rel_tol=tol)
    if where == "b":
        with pytest.raises(RuntimeError, match="non-finite"):
            g.solve_graph(b, method="cg", max_iter=5)
        with pytest.raises(RuntimeError, match="non-finite"):
            g.solve_graph(b, method="pcg", max_iter=5)
        if f32:
            with pytest.raises(RuntimeError, match="non-finite"):
                g.cg_solve_mixed(b, n_low=3, n_refine=2)
    # the handle stays usable after the refusal: the same iterates as a fresh handle
    b2 = g.apply(torch.randn((N, N), dtype=dt, device=DEV))
    x_used, rep = g.cg_solve(b2, max_iter=10, rel_tol=1e-12, check_every=1)
    assert rep["status"] in (bsct.OK, bsct.WARN_NOT_CONVERGED) and torch.isfinite(x_used).all()
    fresh = bsct.gram_build(bsct.Geometry.uniform(N, 30, 92, 1.0, 1.0), bsct.F32 if f32 else bsct.F64)
    x_fresh, rep_fresh = fresh.cg_solve(b2, max_iter=10, rel_tol=1e-12, check_every=1)
    assert torch.equal(x_used, x_fresh) and rep["iterations"] == rep_fresh["iterations"]
    fresh.close()
    g.close()


def test_forced_nonconvergence_reports_warning(bsct):
    # a host-made failure: the iteration budget is too small for the tolerance
    N = 128
    g = bsct.gram_build(bsct.Geometry.uniform(N, 90, 182, 1.0, 1.0), bsct.F32)
    b = torch.randn((N, N), device=DEV, generator=torch.Generator(device=DEV).manual_seed(3))
    for solve in (g.cg_solve, g.pcg_solve, g.sd_solve):
        x, rep = solve(b, max_iter=2, rel_tol=1e-10, check_every=1)
        assert rep["status"] == bsct.WARN_NOT_CONVERGED
        assert not rep["converged"] and rep["iterations"] == 2
        # the report is honest: the recomputed residual matches the recursive one (steepest
        # descent minimises the G-norm error, so either may exceed 1 after two steps)
        assert rep["true_rel_residual"] > 1e-10
        assert abs(rep["true_rel_residual"] - rep["rel_residual"]) < 1e-3 * rep["rel_residual"]
        assert torch.isfinite(x).all()
    x, rep = g.solve_graph(b, method="pcg", max_iter=2, rel_tol=1e-10)
    assert rep["status"] == bsct.WARN_NOT_CONVERGED and rep["iterations"] == 2
    g.close()
