"""Textbook conjugate gradients on the normal equations G c = H^T g_hat - oracle, FP64.

Sec. 2 states the reconstruction as the least-squares problem min ||g_hat - H f||^2
whose normal equations are G c = b with G = H^T H (applied as the Gram filter of
Sec. 4) and b = H^T g_hat (Sec. 5).  The paper solves it by steepest descent; the
hot path uses Hestenes-Stiefel CG, written here in its plain form.
"""
import numpy as np


def cg(apply_G, b, x0=None, iters=20, tol=0.0):
    """Run CG; returns (x, history of ||r_k|| / ||b||, iterates).

    Stops after ``iters`` iterations or when the recursive residual ratio <= tol.
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_G(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    bnorm = float(np.sqrt(np.sum(b * b)))
    hist = [np.sqrt(rr) / bnorm]
    iterates = []
    for _ in range(iters):
        if tol > 0.0 and hist[-1] <= tol:
            break
        q = apply_G(p)
        alpha = rr / float(np.sum(p * q))
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(np.sum(r * r))
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        hist.append(np.sqrt(rr) / bnorm)
        iterates.append(x.copy())
    return x, np.array(hist), iterates


def pcg(apply_G, apply_Minv, b, x0=None, iters=20, tol=0.0):
    """Preconditioned CG with a fixed SPD preconditioner M^-1; returns (x, history of
    ||r_k|| / ||b||, iterates).

    The textbook recurrence: z = M^-1 r, rho = <r, z>, alpha = rho / <p, G p>,
    beta = rho_new / rho, p = z + beta p.  With M^-1 = I it is ``cg``.  Stops after
    ``iters`` iterations or when the residual ratio <= tol.
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_G(x) if x0 is not None else b.copy()
    z = apply_Minv(r)
    p = z.copy()
    rho = float(np.sum(r * z))
    bnorm = float(np.sqrt(np.sum(b * b)))
    hist = [float(np.sqrt(np.sum(r * r))) / bnorm]
    iterates = []
    for _ in range(iters):
        if tol > 0.0 and hist[-1] <= tol:
            break
        q = apply_G(p)
        alpha = rho / float(np.sum(p * q))
        x = x + alpha * p
        r = r - alpha * q
        z = apply_Minv(r)
        rho_new = float(np.sum(r * z))
        p = z + (rho_new / rho) * p
        rho = rho_new
        hist.append(float(np.sqrt(np.sum(r * r))) / bnorm)
        iterates.append(x.copy())
    return x, np.array(hist), iterates


def steepest_descent(apply_G, b, x0=None, iters=20, tol=0.0):
    """Steepest descent on G x = b, the solver of the paper's reconstruction study (Sec. 6).

    Each step moves along the residual r = b - G x by the exact line minimiser of the
    quadratic, alpha = <r, r> / <r, G r>.  Returns (x, history of ||r_k|| / ||b||, iterates).
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_G(x) if x0 is not None else b.copy()
    bnorm = float(np.sqrt(np.sum(b * b)))
    hist = [float(np.sqrt(np.sum(r * r))) / bnorm]
    iterates = []
    for _ in range(iters):
        if tol > 0.0 and hist[-1] <= tol:
            break
        q = apply_G(r)
        alpha = float(np.sum(r * r)) / float(np.sum(r * q))
        x = x + alpha * r
        r = r - alpha * q
        hist.append(float(np.sqrt(np.sum(r * r))) / bnorm)
        iterates.append(x.copy())
    return x, np.array(hist), iterates


def true_relative_residual(apply_G, b, x):
    """||b - G x|| / ||b|| recomputed from scratch (the measure every solver's output is checked by)."""
    r = b - apply_G(x)
    return float(np.sqrt(np.sum(r * r)) / np.sqrt(np.sum(b * b)))
