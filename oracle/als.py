"""ALS and BNGS relaxations (Sections 3 and 5.2), float64.

Readings of points the paper leaves open (each listed in the design notes):
* pseudoinverse solve: Cholesky of Gamma when it succeeds with every pivot above
  R * eps * max(diag); otherwise numpy's Moore-Penrose ``pinv`` with relative
  cutoff R * eps.  Both equal Gamma^+ when Gamma is SPD.
* modes are visited n = 1..N in increasing order.
* Gauss-Seidel inner solve: every row of A^(n) Gamma = B is an independent
  R x R system Gamma x = b; one GS sweep updates x_1..x_R in increasing order
  using the newest values; the sweep count defaults to ten (Section 5.2).
* sort: components in decreasing lambda_r; equal lambdas keep their order.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np

from .tensor import mttkrp, gamma, as64

EPS = np.finfo(np.float64).eps


def pinv_right_solve(M, Gam):
    """Return M Gamma^+ (the ALS update of Section 3)."""
    R = Gam.shape[0]
    d = np.diag(Gam)
    thresh = R * EPS * (d.max() if d.size and d.max() > 0 else 1.0)
    ok = True
    L = np.zeros_like(Gam)
    # Cholesky written out so the pivot test is explicit.
    for j in range(R):
        s = Gam[j, j] - np.dot(L[j, :j], L[j, :j])
        if not (s > thresh):
            ok = False
            break
        L[j, j] = np.sqrt(s)
        for i in range(j + 1, R):
            L[i, j] = (Gam[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    if ok:
        # X Gamma = M  <=>  Gamma X^T = M^T  with Gamma = L L^T
        Y = np.linalg.solve(L, M.T)
        return np.linalg.solve(L.T, Y).T
    return M @ np.linalg.pinv(Gam, rcond=R * EPS)


def normalize(A):
    """Eq. ALSnorm: a_r^(n) <- lambda_r a_r^(n)/||a_r^(n)||, lambda_r = (prod_n ||a_r^(n)||)^(1/N).
    Returns (new factors, lambda).  A column of zero norm is left unchanged (lambda_r = 0)."""
    N = len(A)
    norms = np.array([np.linalg.norm(a, axis=0) for a in A])  # N x R
    lam = np.prod(norms, axis=0) ** (1.0 / N)
    out = []
    for n in range(N):
        scale = np.where(norms[n] > 0, lam / np.where(norms[n] > 0, norms[n], 1.0), 1.0)
        out.append(A[n] * scale[None, :])
    return out, lam


def sort_components(A):
    """Reorder the rank-one terms by decreasing lambda_r = (prod_n ||a_r^(n)||)^(1/N)
    (end of Section 3); ties keep their original order."""
    N = len(A)
    norms = np.array([np.linalg.norm(a, axis=0) for a in A])
    lam = np.prod(norms, axis=0) ** (1.0 / N)
    order = sorted(range(lam.size), key=lambda r: (-lam[r], r))
    return [a[:, order] for a in A]


def als_sweep(Z, A, do_normalize=True):
    """One ALS iteration = one BNGS iteration with the pseudoinverse (Section 3):
    for n = 1..N, A^(n) <- Z_(n) Phi^(n) (Gamma^(n))^+, then Eq. ALSnorm."""
    A = [a.copy() for a in A]
    for n in range(len(A)):
        A[n] = pinv_right_solve(mttkrp(Z, A, n), gamma(A, n))
    if do_normalize:
        A, _ = normalize(A)
    return A


def als(Z, A, iters, sort_at_end=True, tol=None, g_fn=None):
    """``iters`` ALS iterations (normalizing after each), then sort (end of Section 3).
    If ``tol`` is given, stop as soon as ``g_fn(Z, A) < tol`` (checked after each
    iteration).  Returns (A, iterations done)."""
    it = 0
    for it in range(1, iters + 1):
        A = als_sweep(Z, A)
        if tol is not None and g_fn(Z, A) < tol:
            break
    if sort_at_end:
        A = sort_components(A)
    return A, it


def gauss_seidel_rows(X, Gam, B, sweeps=10):
    """Approximately solve X Gamma = B by ``sweeps`` Gauss-Seidel sweeps from X
    (Eq. relaxinnersolve).  Each row x of X satisfies Gamma x^T = b^T."""
    X = X.copy()
    R = Gam.shape[0]
    for _ in range(sweeps):
        for r in range(R):
            s = B[:, r] - X @ Gam[:, r] + X[:, r] * Gam[r, r]
            X[:, r] = s / Gam[r, r]
    return X


def bngs_sweep(Z, A, F, gs_sweeps=10, finest=False):
    """One BNGS iteration on H({A}) = F (Section 5.2): for n = 1..N solve
    A^(n) Gamma^(n) = Z_(n) Phi^(n) + F^(n) by Gauss-Seidel from the current A^(n).
    On the finest level the factors are then normalized (Eq. ALSnorm) and sorted
    by decreasing lambda."""
    A = [a.copy() for a in A]
    for n in range(len(A)):
        B = mttkrp(Z, A, n)
        if F is not None:
            B = B + F[n]
        A[n] = gauss_seidel_rows(A[n], gamma(A, n), B, gs_sweeps)
    if finest:
        A, _ = normalize(A)
        A = sort_components(A)
    return A


__all__ = ["pinv_right_solve", "normalize", "sort_components", "als_sweep", "als",
           "gauss_seidel_rows", "bngs_sweep", "as64"]
