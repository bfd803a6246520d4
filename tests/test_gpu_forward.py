"""GPU parity of the forward projection g_s = S H c (Sec. 2, Eq. 3-4) through the C ABI.

Small images are compared sample by sample with the oracle's ``forward_sample``; at the
bench size (N = 2048, 1800 views, 2900 bins, zeta = 1) sampled detector values are
compared with the oracle's one-sample sum, and two properties that hold at any size are
checked: with zeta = lambda_y = 1 every view sums to the sum of the coefficients, and for
the axis-aligned views {0, pi/2} with lambda_y = 1 and N = M even the back projection of
the projection is exactly G c (Sec. 5).

Tolerances (relative to the largest sample): FP64 1e-11; FP32 1e-5, except unblurred
views within a fraction of a degree of an axis, whose footprint ramps have slope
1 / (|cos| |sin|) (~320 per pixel at 0.18 degrees): an FP32 sample coordinate accurate to
~1.2e-7 pixel moves each of the (up to four) ramp pixels of a sample by ~4e-5 of its
coefficient, so such samples are gated at 2e-4 of the largest sample.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import backproject as obp  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def bsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_13471_gb300 as m

    m.lib()
    return m


CASES = [
    # N, M, lambda_y, zeta, angles (half turns), FP32 tolerance
    (8, 13, 1.0, 1.0, [0.0, 0.07, 0.25, 0.31, 0.5, 0.83, 1.0, 1.37], 1e-5),
    (9, 17, 0.8, 0.5, [0.13, 0.5, 0.77, 1.5, 1.91], 1e-5),
    (12, 20, 1.0, 0.0, [0.0, 0.5, 0.25, 0.1, 0.6], 1e-5),
    (10, 16, 1.7, 2.5, [0.0, 0.3, 0.75], 1e-5),
    (7, 30, 0.6, 0.0, [0.001, 0.4999, 0.2], 2e-4),
    (16, 24, 1.0, 4.0, [0.25, 0.1], 1e-5),
    (64, 92, 1.0, 1.0, list(np.arange(90) / 90), 1e-5),
    (100, 150, 0.9, 0.0, list(np.random.default_rng(3).uniform(-1.0, 3.0, 37)), 1e-5),
]


@pytest.mark.parametrize("N,M,lam,zeta,angles,tol32", CASES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_forward_matches_oracle(bsct, N, M, lam, zeta, angles, tol32, prec):
    angles = np.asarray(angles, dtype=np.float64)
    f64 = prec == "f64"
    c = np.random.default_rng(N * M).standard_normal((N, N))
    if not f64:
        c = c.astype(np.float32).astype(np.float64)
    geom = bsct.Geometry(N, angles, M, lam, zeta)
    cd = torch.tensor(c, dtype=torch.float64 if f64 else torch.float32, device=DEV)
    g = bsct.forward_project(geom, cd, bsct.F64 if f64 else bsct.F32).cpu().double().numpy()
    ref = obp.forward_sample(c, angles, M, lam, zeta)
    # FP64: 1e-12 of the largest sample; the near-axis unblurred case (FP32 gate 2e-4) keeps
    # the ramp-slope allowance of 1e-11 (slope 1 / (|c| |s|) ~ 300 times FP64 coordinates)
    err = np.max(np.abs(g - ref)) / np.max(np.abs(ref))
    print(f"forward N={N} M={M} zeta={zeta} {prec}: {err:.2e}")
    assert err < ((1e-11 if tol32 > 1e-5 else 1e-12) if f64 else tol32)


def test_forward_bench_size_sampled_and_partition_of_unity(bsct):
    N, na, M = 2048, 1800, 2900
    angles = np.arange(na) / na
    geom = bsct.Geometry(N, angles, M, 1.0, 1.0)
    gen = torch.Generator(device=DEV).manual_seed(5)
    cd = torch.rand((N, N), device=DEV, generator=gen)
    g = bsct.forward_project(geom, cd, bsct.F32)
    torch.cuda.synchronize()
    c = cd.cpu().double().numpy()
    rng = np.random.default_rng(6)
    pts = [(int(j), int(m)) for j, m in zip(rng.integers(0, na, 8), rng.integers(300, M - 300, 8))]
    pts += [(0, M // 2), (na // 2, 17), (na // 4, M - 40)]  # axis views, a detector edge, 45 degrees
    ref = obp.forward_sample_points(c, angles, M, 1.0, 1.0, pts)
    gh = g.cpu().double().numpy()
    got = np.array([gh[p] for p in pts])
    assert np.max(np.abs(got - ref)) < 1e-5 * np.max(np.abs(gh))
    # every view's samples add up to the sum of the coefficients
    sums = g.double().sum(dim=1).cpu().numpy()
    assert np.max(np.abs(sums - c.sum())) < 1e-5 * c.sum()


@pytest.mark.parametrize("zeta", [0.0, 1.0])
def test_back_projection_of_projection_is_gram_axis_views(bsct, zeta):
    # views {0, pi/2}, lambda_y = 1, N = M even: every pixel projection falls on a detector
    # sample, so H^T g_hat of the sampled projection equals G c exactly (Sec. 5)
    N = 2048
    geom = bsct.Geometry(N, np.array([0.0, 0.5]), N, 1.0, zeta)
    gen = torch.Generator(device=DEV).manual_seed(8)
    c = torch.randn((N, N), dtype=torch.float64, device=DEV, generator=gen)
    sino = bsct.forward_project(geom, c, bsct.F64)
    b = bsct.backproject(geom, sino, bsct.F64)
    G = bsct.gram_build(geom, bsct.F64)
    gc = G.apply(c)
    err = float((b - gc).norm() / gc.norm())
    G.close()
    assert err < 1e-12


def test_forward_errors(bsct):
    geom = bsct.Geometry(16, np.array([0.1]), 20, 1.0, 4.5)
    with pytest.raises(RuntimeError, match="unsupported size"):
        bsct.forward_project(geom, torch.zeros((16, 16), device=DEV), bsct.F32)
    geom = bsct.Geometry(16, np.array([0.1]), 20, 1.0, 1.0)
    with pytest.raises(ValueError):
        bsct.forward_project(geom, torch.zeros((16, 15), device=DEV), bsct.F32)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_forward_samples_on_box_edges(bsct, prec):
    # axis views without blur, N even and M odd, lambda_y = 1: every sample falls exactly
    # on a pixel edge, where the open box footprint is zero (the oracle agrees)
    N, M = 12, 13
    angles = np.array([0.0, 0.5, 1.0])
    c = np.random.default_rng(1).standard_normal((N, N))
    assert np.all(obp.forward_sample(c, angles, M, 1.0, 0.0) == 0.0)
    dt = torch.float64 if prec == "f64" else torch.float32
    g = bsct.forward_project(bsct.Geometry(N, angles, M, 1.0, 0.0), torch.tensor(c, dtype=dt, device=DEV),
                             bsct.F64 if prec == "f64" else bsct.F32)
    assert float(g.abs().max()) == 0.0
