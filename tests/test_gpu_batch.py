"""Batched multi-slice solve (one CUDA-graph launch) against the single-slice path and the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import backproject as obp  # noqa: E402
from oracle import cg as ocg  # noqa: E402
from oracle import gram as ogram  # noqa: E402
from workloads import ellipse_params, ellipse_sinogram  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def bsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_13471_gb300 as m

    m.lib()
    return m


def slice_set(bsct):
    spec = [(32, 20, 46, 0.0), (64, 45, 91, 1.0), (32, 20, 46, 0.0), (128, 33, 182, 1.0), (16, 9, 23, 0.0),
            (384, 24, 546, 1.0), (64, 45, 91, 1.0)]
    geoms, sinos = [], []
    for i, (N, na, M, zeta) in enumerate(spec):
        ang = np.arange(na) / na
        geoms.append(bsct.Geometry(N, ang, M, 1.0, zeta))
        sino = ellipse_sinogram(ellipse_params(N, 5, seed=i), ang, M, 1.0, zeta)
        sinos.append(torch.tensor(sino, dtype=torch.float32, device=DEV))
    return geoms, sinos


def test_batch_equals_single_slice_path(bsct):
    geoms, sinos = slice_set(bsct)
    batch = bsct.Batch(geoms)
    info = batch.info()
    assert info["geometries"] == 5  # two pairs of slices share a geometry
    xs = batch.solve(sinos, cg_iters=12)
    torch.cuda.synchronize()
    assert batch.info()["graph_nodes"] > 0
    for g, s, x in zip(geoms, sinos, xs):
        f = bsct.gram_build(g, bsct.F32)
        b = bsct.backproject(g, s, bsct.F32)
        x1, _ = f.cg_solve(b, max_iter=12)
        assert torch.equal(x, x1), "batched result differs from the single-slice path"
        f.close()
    # replay (same pointers: no re-recording) and re-record (new outputs)
    xs2 = batch.solve(sinos, xs=[torch.empty_like(x) for x in xs], cg_iters=12)
    xs3 = batch.solve(sinos, xs=xs2, cg_iters=12)
    torch.cuda.synchronize()
    for a, b_ in zip(xs, xs3):
        assert torch.equal(a, b_)
    batch.close()


def test_batch_against_oracle(bsct):
    N, na, M, zeta = 64, 45, 91, 1.0
    ang = np.arange(na) / na
    sino = ellipse_sinogram(ellipse_params(N, 5, seed=1), ang, M, 1.0, zeta)
    batch = bsct.Batch([bsct.Geometry(N, ang, M, 1.0, zeta)])
    (x,) = batch.solve([torch.tensor(sino, dtype=torch.float32, device=DEV)], cg_iters=3)
    torch.cuda.synchronize()
    b = obp.backproject(sino.astype(np.float32).astype(np.float64), N, ang, 1.0, zeta)
    G = ogram.gram_taps(N, ang, zeta)
    _, _, iters = ocg.cg(lambda v: ogram.gram_apply_fft(G, v), b, iters=3)
    xr = iters[-1]
    assert np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr) < 1e-5
    batch.close()


def test_batch_rejects_unsupported(bsct):
    with pytest.raises(RuntimeError, match="unsupported"):
        bsct.Batch([bsct.Geometry.uniform(100, 10, 150)])
