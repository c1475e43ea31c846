"""Textbook conjugate gradient on Mhat^dag Mhat x = b (oracle; test infrastructure).

The paper's application solves the fermion matrix inside the R algorithm
(Sec. 1, su3_rmd); the solver is the standard CG of Hestenes and Stiefel on the
normal equations, in FP64, stopped on the relative residual ||b - A x|| / ||b||.
"""

import numpy as np


def vdot(a, b):
    """<a, b> = sum conj(a) b."""
    return np.vdot(a.reshape(-1), b.reshape(-1))


def norm2(a):
    return float(np.vdot(a.reshape(-1), a.reshape(-1)).real)


def cg(apply_A, b, tol=1e-8, maxiter=100000, x0=None):
    """Solve A x = b for Hermitian positive definite A.

    Iterates x_{k+1} = x_k + alpha_k p_k, r_{k+1} = r_k - alpha_k A p_k,
    p_{k+1} = r_{k+1} + beta_k p_k with alpha_k = |r_k|^2 / <p_k, A p_k>,
    beta_k = |r_{k+1}|^2 / |r_k|^2, and stops when the recomputed true residual
    |b - A x| <= tol |b|.  Returns (x, iterations, true relative residual).
    """
    x = np.zeros_like(b, dtype=complex) if x0 is None else x0.astype(complex).copy()
    bnorm = np.sqrt(norm2(b))
    if bnorm == 0.0:
        return np.zeros_like(b, dtype=complex), 0, 0.0
    r = b - apply_A(x)
    p = r.copy()
    rr = norm2(r)
    k = 0
    while k < maxiter:
        if np.sqrt(rr) <= tol * bnorm:
            true_res = np.sqrt(norm2(b - apply_A(x))) / bnorm
            if true_res <= tol:
                return x, k, true_res
            r = b - apply_A(x)          # restart from the true residual
            p = r.copy()
            rr = norm2(r)
        Ap = apply_A(p)
        alpha = rr / vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = norm2(r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        k += 1
    true_res = np.sqrt(norm2(b - apply_A(x))) / bnorm
    return x, k, true_res
