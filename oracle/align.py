"""Alignment of two CP solutions up to the scaling and permutation indeterminacies
(Section 1) for error reporting.

Each component r is written as lambda_r times unit columns; the first N-1 modes'
columns get the sign that makes their largest-magnitude entry positive and the
last mode absorbs the sign product; components are matched by maximizing
prod_n |cos| with the Hungarian method; the error of a mode is
||B_test - B_ref||_F / ||B_ref||_F with B = unit columns times lambda_r^(1/N).

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linear_sum_assignment


def canonical(A):
    """Unit columns with fixed signs, and lambda (product of the column norms)."""
    N = len(A)
    norms = np.array([np.linalg.norm(a, axis=0) for a in A])
    lam = np.prod(norms, axis=0)
    U = [a / np.where(nr > 0, nr, 1.0)[None, :] for a, nr in zip(A, norms)]
    sign_total = np.ones(A[0].shape[1])
    for n in range(N - 1):
        idx = np.argmax(np.abs(U[n]), axis=0)
        s = np.sign(U[n][idx, np.arange(U[n].shape[1])])
        s[s == 0] = 1.0
        U[n] = U[n] * s[None, :]
        sign_total *= s
    U[N - 1] = U[N - 1] * sign_total[None, :]
    return U, lam


def equal_norm(U, lam):
    N = len(U)
    scale = np.abs(lam) ** (1.0 / N)
    return [u * scale[None, :] for u in U]


def factor_error(A_ref, A_test):
    """Max over modes of the relative Frobenius error after alignment."""
    Ur, lr = canonical(A_ref)
    Ut, lt = canonical(A_test)
    R = lr.size
    cost = np.ones((R, R))
    for n in range(len(Ur)):
        cost = cost * np.abs(Ur[n].T @ Ut[n])
    row, col = linear_sum_assignment(-cost)
    perm = col[np.argsort(row)]
    Ut = [u[:, perm] for u in Ut]
    lt = lt[perm]
    # a residual sign difference on the last mode is a genuine difference
    Br = equal_norm(Ur, lr)
    Bt = equal_norm(Ut, lt)
    errs = [np.linalg.norm(bt - br) / np.linalg.norm(br) for br, bt in zip(Br, Bt)]
    return float(max(errs))
