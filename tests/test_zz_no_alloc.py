"""The no-allocation Gram apply (bsct_gram_apply_noalloc) against bsct_gram_apply.

bsct_gram_apply_noalloc serves callers that cannot allocate device memory (a plug-in
whose host application owns the device memory pool, or a latency-critical path where
cudaMalloc / cudaFree would synchronise the device): its scratch lives in fixed-size
arrays inside the library.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes alone in a fresh
process (it builds its own Gram filter).
"""
import ctypes

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

    L = m.lib()
    L.bsct_gram_apply_noalloc.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]
    L.bsct_gram_apply_noalloc.restype = ctypes.c_int
    return m


def _noalloc(m, N, spec, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return m.lib().bsct_gram_apply_noalloc(N, ctypes.c_void_p(spec.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(y.data_ptr()), stream)


def rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


@pytest.mark.parametrize("N,zeta", [(64, 0.0), (512, 1.0)])
def test_noalloc_matches_gram_apply_twice(bsct, N, zeta):
    geom = bsct.Geometry.uniform(N, 90, int(1.42 * N), 1.0, zeta)
    g = bsct.gram_build(geom, bsct.F32)
    spec = g.spectrum()  # [2N][N+1] FP64, caller-owned
    gen = torch.Generator(device=DEV).manual_seed(N)
    for call in range(2):  # two calls in a row share the library's scratch
        x = torch.randn((N, N), device=DEV, generator=gen)
        y_ref = g.apply(x)
        y = torch.full((N, N), float("nan"), device=DEV)
        assert _noalloc(bsct, N, spec, x, y) == 0
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        assert rel(y, y_ref) < 1e-5, f"call {call}"
    g.close()


def test_noalloc_sizes_in_any_order_and_against_the_oracle(bsct):
    """Calls with N = 64, then 512, then 64 again: each call writes the twiddle tables of
    its own N, so returning to an earlier size reads no stale tables.  The N = 64 results
    are also compared with the FP64 oracle's FFT convolution of the same taps."""
    from oracle import gram as ogram

    handles = {}
    for N in (64, 512):
        geom = bsct.Geometry.uniform(N, 90, int(1.42 * N), 1.0, 1.0)
        g = bsct.gram_build(geom, bsct.F32)
        handles[N] = (g, g.spectrum())
    gen = torch.Generator(device=DEV).manual_seed(7)
    for N in (64, 512, 64):
        g, spec = handles[N]
        x = torch.randn((N, N), device=DEV, generator=gen)
        y = torch.full((N, N), float("nan"), device=DEV)
        assert _noalloc(bsct, N, spec, x, y) == 0
        torch.cuda.synchronize()
        assert rel(y, g.apply(x)) < 1e-5, f"N = {N}"
        if N == 64:
            taps = g.taps().cpu().numpy()
            y_ref = ogram.gram_apply_fft(taps, x.cpu().double().numpy())
            err = np.linalg.norm(y.cpu().double().numpy() - y_ref) / np.linalg.norm(y_ref)
            assert err < 1e-5, f"oracle, N = {N}: {err:.2e}"
    for g, _ in handles.values():
        g.close()


def test_noalloc_rejects_sizes_beyond_its_limit(bsct):
    N = 1024  # supported by bsct_gram_apply, above BSCT_NOALLOC_MAX_N = 512
    spec = torch.zeros((2 * N, N + 1), dtype=torch.float64, device=DEV)
    x = torch.zeros((N, N), device=DEV)
    y = torch.zeros((N, N), device=DEV)
    assert _noalloc(bsct, N, spec, x, y) == -2
    assert b"512" in bsct.lib().bsct_last_error_string()
    assert _noalloc(bsct, 100, spec, x, y) == -2
