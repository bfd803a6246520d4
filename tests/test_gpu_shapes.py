"""FFT launch shapes and the autotuner (through the C ABI).

Every valid shape (rows per CTA of the two row passes, CTAs per SM of the column pass)
must give a bit-identical Gram apply: the rows and columns are transformed by the same
code, only their grouping into CTAs changes.  CG and preconditioned CG sum their inner
products per CTA, so a different grouping changes the FP64 summation order: their
iterates agree to rounding.  The autotuner must leave a valid shape that computes the
same apply.  Every test restores the built-in shape.
"""
import itertools

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
    return m


def shapes(bsct, N, prec):
    f, v = bsct.fft_shape_candidates(N, prec)
    assert f[1] and v[1]  # the built-in default is always valid
    return [(a, b, c) for a, b, c in itertools.product([x for x in f if x], [x for x in v if x], (0, 1))]


def restore(bsct, N, prec):
    f, v = bsct.fft_shape_candidates(N, prec)
    bsct.set_fft_shape(N, f[1], v[1], 0, prec)


@pytest.mark.parametrize("N,prec", [(16, 0), (64, 0), (384, 0), (2048, 0), (64, 1), (256, 1)])
def test_every_shape_same_apply(bsct, N, prec):
    dt = torch.float32 if prec == bsct.F32 else torch.float64
    g = bsct.gram_build(bsct.Geometry.uniform(N, 30, int(1.42 * N) + 2, 1.0, 1.0), prec)
    x = torch.randn((N, N), dtype=dt, device=DEV, generator=torch.Generator(device=DEV).manual_seed(N))
    restore(bsct, N, prec)
    ref = g.apply(x).clone()
    b = ref.clone()
    x_cg, _ = g.cg_solve(b, max_iter=5)
    x_pc, _ = g.pcg_solve(b, max_iter=3)
    tol = 1e-5 if prec == bsct.F32 else 1e-12
    try:
        for shp in shapes(bsct, N, prec):
            bsct.set_fft_shape(N, *shp, precision=prec)
            assert bsct.fft_shape(N, prec) == shp
            y = g.apply(x)
            assert torch.equal(y, ref), shp
            xc, _ = g.cg_solve(b, max_iter=5)
            xp, _ = g.pcg_solve(b, max_iter=3)
            assert float((xc - x_cg).norm() / x_cg.norm()) < tol, shp
            assert float((xp - x_pc).norm() / x_pc.norm()) < tol, shp
    finally:
        restore(bsct, N, prec)
        g.close()


@pytest.mark.parametrize("flush", [0, 256 << 20])
def test_autotune_keeps_a_valid_shape(bsct, flush):
    N = 512
    g = bsct.gram_build(bsct.Geometry.uniform(N, 60, 730, 1.0, 1.0), bsct.F32)
    x = torch.randn((N, N), device=DEV, generator=torch.Generator(device=DEV).manual_seed(3))
    restore(bsct, N, bsct.F32)
    ref = g.apply(x).clone()
    try:
        best, us, all_us = bsct.fft_autotune(N, bsct.F32, reps=5, flush_bytes=flush)
        assert best in shapes(bsct, N, bsct.F32) and bsct.fft_shape(N, bsct.F32) == best
        timed = [t for t in all_us if t >= 0]
        assert len(timed) == len(shapes(bsct, N, bsct.F32)) and us == pytest.approx(min(timed))
        assert torch.equal(g.apply(x), ref)
    finally:
        restore(bsct, N, bsct.F32)
        g.close()


def test_shape_errors(bsct):
    f, v = bsct.fft_shape_candidates(64, bsct.F32)
    with pytest.raises(RuntimeError, match="invalid argument"):
        bsct.set_fft_shape(64, 3, v[1])
    with pytest.raises(RuntimeError, match="unsupported size"):
        bsct.fft_shape(100)
    assert bsct.fft_shape(64) == (f[1], v[1], 0)
