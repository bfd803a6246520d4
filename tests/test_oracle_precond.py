"""Pins for the oracle's preconditioned CG and circulant preconditioner - CPU only.

The preconditioner is the N x N section of the inverse of the 2N-periodic circulant
that embeds the Toeplitz-block-Toeplitz Gram filter (Sec. 4), with its Fourier symbol
floored at eps * G^(0).  Pins: textbook PCG properties on dense systems, the inverse
checked by a brute-force circular convolution, the closed form when the floor covers
the whole symbol, symmetry and positivity, and fewer iterations than plain CG.
"""
import numpy as np
import pytest

from oracle import cg as ocg
from oracle import gram
from oracle.geometry import uniform_angles


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A @ A.T + n * np.eye(n), rng.standard_normal(n)


def test_pcg_exact_preconditioner_one_step():
    # M^-1 = A^-1: z = x* - x, so the first step lands on the solution
    A, b = _spd(20, 1)
    Ainv = np.linalg.inv(A)
    x, hist, _ = ocg.pcg(lambda v: A @ v, lambda v: Ainv @ v, b, iters=1)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-12 * np.linalg.norm(x)
    assert hist[-1] < 1e-12


def test_pcg_jacobi_matches_dense_solve():
    A, b = _spd(30, 2)
    A = A + np.diag(np.linspace(1.0, 400.0, 30))  # badly scaled diagonal
    d = np.diag(A).copy()
    x, hist, _ = ocg.pcg(lambda v: A @ v, lambda v: v / d, b, iters=60, tol=1e-14)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)


def test_pcg_terminates_in_n_steps():
    # a 3 x 3 SPD system with a non-trivial SPD preconditioner: exact after 3 steps
    A = np.array([[4.0, 1.0, 0.0], [1.0, 3.0, 1.0], [0.0, 1.0, 2.0]])
    P = np.array([[2.0, 0.5, 0.0], [0.5, 1.0, 0.0], [0.0, 0.0, 1.0]])
    b = np.array([1.0, -2.0, 0.5])
    x, _, _ = ocg.pcg(lambda v: A @ v, lambda v: P @ v, b, iters=3)
    assert np.max(np.abs(x - np.linalg.solve(A, b))) < 1e-13


def test_pcg_identity_preconditioner_is_cg():
    A, b = _spd(25, 3)
    x1, h1, _ = ocg.pcg(lambda v: A @ v, lambda v: v, b, iters=12)
    x2, h2, _ = ocg.cg(lambda v: A @ v, b, iters=12)
    assert np.allclose(h1, h2, rtol=1e-10, atol=0) and np.allclose(x1, x2, rtol=1e-10, atol=1e-14)


@pytest.fixture(scope="module")
def dense_filter():
    # 90 views at N = 16 without blur: the embedded symbol is positive (min / max
    # = 2.4e-4; with zeta = 1 it dips to -1 %)
    N = 16
    G = gram.gram_taps(N, uniform_angles(90), 0.0)
    Ghat = gram.gram_spectrum(G)[0]
    assert Ghat.min() > 1e-4 * Ghat[0, 0]
    return N, G


def test_symbol_floor_and_dc(dense_filter):
    N, G = dense_filter
    Ghat, Gim = gram.gram_spectrum(G)
    assert Ghat[0, 0] == pytest.approx(G.sum(), rel=1e-13)  # G^(0) = sum of the taps
    assert np.max(np.abs(Ghat)) == pytest.approx(G.sum(), rel=1e-13)  # taps >= 0
    h = gram.circulant_precond_symbol(G, 1e-5)
    assert np.all(h > 0) and np.allclose(h * Ghat, 1.0, rtol=1e-12)  # floor inactive
    with pytest.raises(ValueError):
        gram.circulant_precond_symbol(G, 0.0)


def test_inverse_by_brute_force_circular_convolution(dense_filter):
    # with the floor inactive, convolving the full periodic field with the embedded
    # kernel (shifted sums, no FFT) gives back the zero-padded input
    N, G = dense_filter
    L = 2 * N
    x = np.random.default_rng(4).standard_normal((N, N))
    w = gram.circulant_inverse_full(G, x, 1e-5)
    K = gram.embed_circulant(G)
    back = np.zeros((L, L))
    for a2 in range(L):
        for a1 in range(L):
            if K[a2, a1] != 0.0:
                back += K[a2, a1] * np.roll(np.roll(w, a2, axis=0), a1, axis=1)
    xp = np.zeros((L, L))
    xp[:N, :N] = x
    assert np.max(np.abs(back - xp)) < 1e-10 * np.max(np.abs(x))


def test_full_floor_is_scaled_identity(dense_filter):
    # eps = 1 floors every frequency at G^(0): M^-1 x = x / sum(taps)
    N, G = dense_filter
    x = np.random.default_rng(5).standard_normal((N, N))
    y = gram.circulant_precond_apply(G, x, 1.0)
    assert np.max(np.abs(y - x / G.sum())) < 1e-14 * np.max(np.abs(x / G.sum()))


def test_sparse_angles_symmetric_positive():
    # 18 views at N = 12: the symbol has negative values; the floored M^-1 is still SPD
    N = 12
    G = gram.gram_taps(N, uniform_angles(18), 1.0)
    assert gram.gram_spectrum(G)[0].min() < 0
    rng = np.random.default_rng(6)
    M = np.zeros((N * N, N * N))
    for k in range(N * N):
        e = np.zeros(N * N)
        e[k] = 1.0
        M[:, k] = gram.circulant_precond_apply(G, e.reshape(N, N), 1e-3).ravel()
    assert np.max(np.abs(M - M.T)) < 1e-13 * np.max(np.abs(M))
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    a = rng.standard_normal((N, N))
    assert np.sum(a * gram.circulant_precond_apply(G, a, 1e-3)) > 0


def test_pcg_needs_fewer_iterations_than_cg():
    N = 48
    G = gram.gram_taps(N, uniform_angles(90), 1.0, method="boxspline")
    apply = lambda v: gram.gram_apply_fft(G, v)
    yy, xx = np.mgrid[0:N, 0:N] / N - 0.5
    xt = ((xx / 0.4) ** 2 + (yy / 0.3) ** 2 < 1).astype(float)
    xt += np.random.default_rng(7).standard_normal((N, N)) * 0.1
    b = apply(xt)
    _, h_cg, _ = ocg.cg(apply, b, iters=500, tol=1e-4)
    x, h_p, _ = ocg.pcg(apply, lambda v: gram.circulant_precond_apply(G, v, 1e-4), b, iters=500, tol=1e-4)
    assert h_p[-1] <= 1e-4 and ocg.true_relative_residual(apply, b, x) < 2e-4
    assert len(h_p) * 2 < len(h_cg)


def test_steepest_descent_scaled_identity_one_step():
    b = np.array([1.0, -2.0, 3.0])
    x, hist, _ = ocg.steepest_descent(lambda v: 4.0 * v, b, iters=1)
    assert np.max(np.abs(x - b / 4.0)) < 1e-15 and hist[-1] < 1e-15


def test_steepest_descent_textbook_rate():
    # A = diag(1, kappa), x0 = 0, b = A (kappa, 1) (error along the worst direction):
    # every step multiplies the A-norm of the error by exactly (kappa - 1) / (kappa + 1)
    kappa = 9.0
    A = np.diag([1.0, kappa])
    xs = np.array([kappa, 1.0])
    b = A @ xs
    _, _, its = ocg.steepest_descent(lambda v: A @ v, b, iters=6)
    en = lambda e: float(np.sqrt(e @ A @ e))
    errs = [en(xs)] + [en(xs - x) for x in its]
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert np.allclose(ratios, (kappa - 1) / (kappa + 1), rtol=1e-12)


def test_steepest_descent_converges_and_energy_decreases():
    A, b = _spd(20, 9)
    xs = np.linalg.solve(A, b)
    x, _, its = ocg.steepest_descent(lambda v: A @ v, b, iters=400, tol=1e-13)
    en = [float((xs - z) @ A @ (xs - z)) for z in its]
    assert np.all(np.diff(en) < 0) and np.linalg.norm(x - xs) < 1e-11 * np.linalg.norm(xs)
