"""Oracle for solves and iterative refinement.

TEST INFRASTRUCTURE ONLY.  Definitions written out plainly:

  * triangular solves with the Cholesky factor: L y = r (forward
    substitution), L^T d = y (back substitution);
  * refinement: x_0 = 0, r_0 = B; repeat d = (L L^T)^{-1} r, x += d,
    r = B - A x (FP64), until the backward error is small enough;
  * normwise backward error of column j (Rigal and Gaches):
        eta_j = ||b_j - A x_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf),
    reported as max_j eta_j.
"""
import numpy as np


def forward_sub(L, Rhs):
    """Solve L Y = Rhs, L lower triangular (dense), row by row."""
    n = L.shape[0]
    Y = np.array(Rhs, dtype=np.float64, copy=True)
    for i in range(n):
        Y[i] = (Y[i] - L[i, :i] @ Y[:i]) / L[i, i]
    return Y


def back_sub_t(L, Y):
    """Solve L^T X = Y, L lower triangular (dense), from the last row up."""
    n = L.shape[0]
    X = np.array(Y, dtype=np.float64, copy=True)
    for i in range(n - 1, -1, -1):
        X[i] = (X[i] - L[i + 1:, i] @ X[i + 1:]) / L[i, i]
    return X


def chol_solve(L, Rhs):
    return back_sub_t(L, forward_sub(L, Rhs))


def backward_error(A, X, B):
    """max_j ||b_j - A x_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf) with
    A the full symmetric matrix (FP64)."""
    X = X.reshape(X.shape[0], -1)
    B = B.reshape(B.shape[0], -1)
    Rr = B - A @ X
    anorm = np.max(np.sum(np.abs(A), axis=1))
    num = np.max(np.abs(Rr), axis=0)
    den = anorm * np.max(np.abs(X), axis=0) + np.max(np.abs(B), axis=0)
    return float(np.max(num / den))


def symmetric_from_lower(A):
    Lw = np.tril(A)
    return Lw + np.tril(Lw, -1).T


def refine(A, L, B, tol=1e-12, max_iter=30):
    """Iterative refinement with a (possibly low-accuracy) factor L of A.
    Returns (X, iterations, eta history)."""
    X = np.zeros_like(B, dtype=np.float64)
    Rr = np.array(B, dtype=np.float64)
    hist = []
    for it in range(1, max_iter + 1):
        X = X + chol_solve(L, Rr)
        Rr = B - A @ X
        eta = backward_error(A, X, B)
        hist.append(eta)
        if eta <= tol:
            return X, it, hist
    return X, max_iter, hist
