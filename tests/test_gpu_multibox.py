"""GPU parity for a detector kernel made of two boxes (Sec. 2's series of box convolutions).

With widths w1, w2 the footprint is M_[|c|, |s|, w1, w2], the Gram kernel
M_[c, c, s, s, w1, w1, w2, w2] and the sinogram interpolant has degree 3 on oblique views
(2 on axis views), with the cubic correction filter of Eq. 5.  The Gram taps, the back
projection and the forward projection are compared with the oracle element by element on
seeded inputs, including views on and within a fraction of a degree of the axes (where the
short-direction split carries the accuracy).  Gates (relative to the largest reference
value): FP64 1e-12; FP32 1e-5 (the tables are fitted in FP64 and rounded once; the
detector coordinate is formed in FP64).  Two properties that need no oracle: every view
of the forward projection sums to the sum of the coefficients when lambda_y = 1 (unit
mass of the footprint; with a unit-width box among its directions the unit-spaced
samples form a partition of unity), and on the views
{0, pi/2} with two unit boxes, lambda_y = 1 and even N, M the back projection of the
projection is exactly G c (the footprint is then the quadratic B-spline, Sec. 5).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import backproject as obp  # noqa: E402
from oracle import gram as ogram  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

NEAR_AXIS = [0.0, 1e-3, 0.4998, 0.5, 0.75]


@pytest.fixture(scope="module")
def bsct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_13471_gb300 as m

    m.lib()
    return m


def maxrel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def angles_for(kind, n, seed):
    if kind == "uniform":
        return np.arange(n) / n
    if kind == "near_axis":
        return np.array(NEAR_AXIS + list(np.random.default_rng(seed).uniform(-1.0, 2.0, n)))
    return np.random.default_rng(seed).uniform(-1.0, 2.0, n)


@pytest.mark.parametrize("N,kind,widths", [(16, "uniform", (0.5, 0.8)), (16, "near_axis", (0.7, 1.0)),
                                           (32, "random", (1.0, 1.0)), (16, "near_axis", (2.5, 0.3))])
def test_gram_taps_two_boxes(bsct, N, kind, widths):
    angles = angles_for(kind, 9, N)
    geom = bsct.Geometry(N, angles, 2 * N, 1.0, widths)
    g = bsct.gram_build(geom, bsct.F64)
    taps = g.taps().cpu().numpy()
    g.close()
    assert maxrel(taps, ogram.gram_taps(N, angles, widths)) < 1e-12


BP_CASES = [
    # N, M, lambda_y, widths, angle kind, views
    (9, 17, 1.0, (0.5, 0.8), "uniform", 12),
    (16, 30, 0.9, (0.7, 1.0), "near_axis", 6),
    (12, 24, 0.6, (1.0, 1.0), "random", 8),
    (7, 20, 1.3, (2.5, 0.3), "near_axis", 3),
    (24, 40, 0.8, (0.4, 1.6), "random", 10),
]


@pytest.mark.parametrize("N,M,lam,widths,kind,nv", BP_CASES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_backproject_two_boxes(bsct, N, M, lam, widths, kind, nv, prec):
    angles = angles_for(kind, nv, N + M)
    f64 = prec == "f64"
    sino = np.random.default_rng(N * M).standard_normal((angles.size, M))
    if not f64:
        sino = sino.astype(np.float32).astype(np.float64)
    geom = bsct.Geometry(N, angles, M, lam, widths)
    sd = torch.tensor(sino, dtype=torch.float64 if f64 else torch.float32, device=DEV)
    b = bsct.backproject(geom, sd, bsct.F64 if f64 else bsct.F32).cpu().double().numpy()
    ref = obp.backproject(sino, N, angles, lam, widths)
    assert maxrel(b, ref) < (1e-12 if f64 else 1e-5)


@pytest.mark.parametrize("N,M,lam,widths,kind,nv", BP_CASES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_forward_two_boxes(bsct, N, M, lam, widths, kind, nv, prec):
    angles = angles_for(kind, nv, N * M)
    f64 = prec == "f64"
    c = np.random.default_rng(N + 7 * M).standard_normal((N, N))
    if not f64:
        c = c.astype(np.float32).astype(np.float64)
    geom = bsct.Geometry(N, angles, M, lam, widths)
    cd = torch.tensor(c, dtype=torch.float64 if f64 else torch.float32, device=DEV)
    g = bsct.forward_project(geom, cd, bsct.F64 if f64 else bsct.F32).cpu().double().numpy()
    ref = obp.forward_sample(c, angles, M, lam, widths)
    assert maxrel(g, ref) < (1e-12 if f64 else 1e-5)


def test_forward_two_boxes_unit_mass(bsct):
    # lambda_y = 1, one box of unit width and a detector wide enough for every footprint:
    # the unit box makes the unit-spaced samples of every footprint sum to its unit mass,
    # so each view sums to sum(c)
    N, M = 40, 90
    angles = np.random.default_rng(5).uniform(0.0, 2.0, 23)
    c = np.random.default_rng(6).standard_normal((N, N))
    geom = bsct.Geometry(N, angles, M, 1.0, (1.0, 1.7))
    g = bsct.forward_project(geom, torch.tensor(c, device=DEV), bsct.F64).cpu().numpy()
    assert np.max(np.abs(g.sum(axis=1) - c.sum())) < 1e-11 * np.abs(c).sum()


def test_two_box_exact_recovery_axis_views(bsct):
    N, M = 32, 40
    angles = np.array([0.0, 0.5])
    widths = (1.0, 1.0)
    c = np.random.default_rng(4).standard_normal((N, N))
    geom = bsct.Geometry(N, angles, M, 1.0, widths)
    sino = bsct.forward_project(geom, torch.tensor(c, device=DEV), bsct.F64)
    b = bsct.backproject(geom, sino, bsct.F64).cpu().numpy()
    g = bsct.gram_build(geom, bsct.F64)
    Gc = g.apply(torch.tensor(c, device=DEV)).cpu().numpy()
    g.close()
    assert maxrel(b, Gc) < 1e-12


def test_one_box_list_is_the_scalar_path(bsct):
    N, M = 20, 33
    angles = np.array([0.0, 0.13, 0.5, 0.71])
    sino = torch.tensor(np.random.default_rng(8).standard_normal((4, M)), device=DEV)
    b_list = bsct.backproject(bsct.Geometry(N, angles, M, 0.9, (0.8,)), sino, bsct.F64)
    b_scalar = bsct.backproject(bsct.Geometry(N, angles, M, 0.9, 0.8), sino, bsct.F64)
    assert torch.equal(b_list, b_scalar)
    c = torch.tensor(np.random.default_rng(9).standard_normal((N, N)), device=DEV)
    assert torch.equal(bsct.forward_project(bsct.Geometry(N, angles, M, 0.9, (0.8,)), c, bsct.F64),
                       bsct.forward_project(bsct.Geometry(N, angles, M, 0.9, 0.8), c, bsct.F64))
