"""Pins for the oracle's CG and the end-to-end normal equations (Sec. 2) - CPU only."""
import numpy as np

from oracle import backproject as bp
from oracle import cg as ocg
from oracle import gram
from oracle.geometry import uniform_angles
from workloads import ellipse_params, ellipse_sinogram


def test_cg_matches_dense_solve():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((30, 30))
    A = A @ A.T + 30 * np.eye(30)
    b = rng.standard_normal(30)
    x, hist, _ = ocg.cg(lambda v: A @ v, b, iters=60, tol=1e-14)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)
    assert np.all(np.diff(hist[:5]) != 0)


def test_cg_exact_in_n_steps_on_tiny_system():
    # CG terminates in at most n steps in exact arithmetic (textbook property)
    A = np.diag([1.0, 2.0, 5.0])
    b = np.array([1.0, 1.0, 1.0])
    x, _, _ = ocg.cg(lambda v: A @ v, b, iters=3)
    assert np.max(np.abs(x - b / np.diag(A))) < 1e-14


def test_cg_on_normal_equations_converges():
    # G c = H^T g_hat for a small ellipse phantom: residual <= 1e-10 after enough iterations
    N, M, na = 32, 46, 45
    angles = uniform_angles(na)
    params = ellipse_params(N, 5, seed=0)
    sino = ellipse_sinogram(params, angles, M, 1.0, 0.0)
    b = bp.backproject(sino, N, angles, 1.0, 0.0)
    G = gram.gram_taps(N, angles, 0.0)
    apply = lambda v: gram.gram_apply_fft(G, v)
    x, hist, _ = ocg.cg(apply, b, iters=400, tol=1e-11)
    assert ocg.true_relative_residual(apply, b, x) < 1e-10
    assert hist[-1] < hist[1] < hist[0]
