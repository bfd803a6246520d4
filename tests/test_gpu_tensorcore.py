"""Tensor-core paths: the BF16 GEMM building block and the split-BF16 DFT-GEMM Gram apply.

GEMM: against an FP64 CPU product of the same BF16-rounded operands (FP32-accumulate
tolerance 1e-5).  DFT-GEMM apply: error against the FP64 oracle, gated at 2e-5
relative L2: the hi/lo split keeps ~16 significant bits per operand (the dropped lo x lo
product and the lo parts' own rounding are ~2^-16 relative per GEMM), and measured
errors are 5-7e-6 over four GEMM stages; refinement by FP32 residual CG steps must reach
the FP32 path's residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cg as ocg  # noqa: E402
from oracle import gram as ogram  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def bsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_13471_gb300 as m

    m.lib()
    return m


GEMM_SHAPES = [(128, 128, 64, 1),  # one CTA, one K tile: the smallest case of the tcgen05 kernel
               (200, 136, 72, 2), (128, 256, 384, 1), (16, 8, 24, 3), (264, 520, 40, 1),
               (32, 1024, 288, 1),  # U-Net level 0 (M < 128: the roles of A and B are exchanged)
               (128, 2048, 384, 1),  # a DFT-GEMM stage (M = 2P, K = 6P)
               (520, 392, 1032, 2),  # ragged tiles in M, N and K, several K tiles, batches
               (256, 48, 200, 2), (136, 24, 64, 1)]  # narrow N: 64- and 32-column tiles for K-major B


@pytest.mark.parametrize("path", [0, 1])  # 0: tcgen05 tensor cores, 1: warp-level mma.sync
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K,batch", GEMM_SHAPES)
def test_gemm_bf16(bsct, path, ta, tb, M, N, K, batch):
    g = torch.Generator().manual_seed(M * N + K)
    a = torch.randn((batch, K, M) if ta else (batch, M, K), generator=g).to(torch.bfloat16)
    b = torch.randn((batch, N, K) if tb else (batch, K, N), generator=g).to(torch.bfloat16)
    c0 = torch.randn((batch, M, N), generator=g)
    bsct.set_gemm_path(path)
    bsct.input_status()  # clear what earlier work on the device left in the (sticky) status
    try:
        c = bsct.gemm_bf16(a.to(DEV), b.to(DEV), c0.clone().to(DEV), trans_a=ta, trans_b=tb, alpha=0.5, beta=2.0)
        torch.cuda.synchronize()
    finally:
        bsct.set_gemm_path(0)
    A = a.double().transpose(1, 2) if ta else a.double()
    B = b.double().transpose(1, 2) if tb else b.double()
    ref = 0.5 * torch.bmm(A, B) + 2.0 * c0.double()
    err = float((c.cpu().double() - ref).norm() / ref.norm())
    assert err < 1e-5
    assert bsct.input_status() == bsct.OK  # no bounded wait gave up


def test_gemm_rejects_misaligned(bsct):
    a = torch.zeros((16, 12), dtype=torch.bfloat16, device=DEV)
    b = torch.zeros((12, 8), dtype=torch.bfloat16, device=DEV)
    with pytest.raises(RuntimeError, match="multiples of 8"):
        bsct.gemm_bf16(a, b)


@pytest.mark.parametrize("N", [16, 64, 256, 384])
def test_dftgemm_apply_error_vs_oracle(bsct, N):
    angles = np.arange(30) / 30
    geom = bsct.Geometry(N, angles, 2 * N, 1.0, 1.0)
    g = bsct.gram_build(geom, bsct.F32)
    G = ogram.gram_taps(N, angles, 1.0)
    x = np.random.default_rng(N).standard_normal((N, N)).astype(np.float32)
    xd = torch.tensor(x, device=DEV)
    y = g.apply(xd, mode=bsct.APPLY_DFTGEMM_BF16).cpu().numpy()
    ref = ogram.gram_apply_fft(G, x.astype(np.float64))
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    print(f"N={N} split-BF16 DFT-GEMM apply rel-L2 error vs FP64 oracle: {err:.3e}")
    assert err < 2e-5
    y32 = g.apply(xd).cpu().numpy()
    assert np.linalg.norm(y32 - ref) / np.linalg.norm(ref) < err  # FP32 FFT is the more accurate path
    g.close()


def test_dftgemm_full_size_sampled(bsct):
    N = 2048
    angles = np.arange(12) / 12
    g = bsct.gram_build(bsct.Geometry(N, angles, 2900, 1.0, 1.0), bsct.F32)
    G = ogram.gram_taps(N, angles, 1.0)
    x = np.random.default_rng(3).standard_normal((N, N)).astype(np.float32)
    y = g.apply(torch.tensor(x, device=DEV), mode=bsct.APPLY_DFTGEMM_BF16).cpu().numpy()
    pts = [tuple(p) for p in np.random.default_rng(2).integers(0, N, size=(10, 2))]
    ref = ogram.gram_apply_sampled(G, x.astype(np.float64), pts)
    got = np.array([y[p] for p in pts])
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-5
    g.close()


def test_mixed_cg_refinement(bsct):
    # BF16 DFT-GEMM CG stalls at the operator's precision; FP32 residual CG steps recover
    N, na = 128, 90
    angles = np.arange(na) / na
    geom = bsct.Geometry(N, angles, 182, 1.0, 1.0)
    g = bsct.gram_build(geom, bsct.F32)
    G = ogram.gram_taps(N, angles, 1.0)
    rng = np.random.default_rng(0)
    xt = rng.standard_normal((N, N))
    b = ogram.gram_apply_fft(G, xt).astype(np.float32)
    bd = torch.tensor(b, device=DEV)
    apply = lambda v: ogram.gram_apply_fft(G, v)
    x_low, rep_low = g.cg_solve_mixed(bd, n_low=60, n_refine=0)
    x_mix, rep_mix = g.cg_solve_mixed(bd, n_low=60, n_refine=20)
    x_32, _ = g.cg_solve(bd, max_iter=80)
    r_low = ocg.true_relative_residual(apply, b.astype(np.float64), x_low.cpu().double().numpy())
    r_mix = ocg.true_relative_residual(apply, b.astype(np.float64), x_mix.cpu().double().numpy())
    r_32 = ocg.true_relative_residual(apply, b.astype(np.float64), x_32.cpu().double().numpy())
    print(f"true residual: bf16-only {r_low:.2e}, refined {r_mix:.2e}, fp32 {r_32:.2e}")
    assert r_mix < r_low
    assert r_mix < 3 * r_32
    g.close()
