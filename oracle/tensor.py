"""Tensor algebra of Sections 2-3, written out in float64.

Tensors are NumPy arrays indexed Z[i_1, ..., i_N].  Factor matrices are I_n x R.
Modes are 0-based in code (the paper's mode n is ``n-1`` here).

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np


def as64(Z):
    return np.asarray(Z, dtype=np.float64)


def unfold(Z, n):
    """Mode-n matricization Z_(n) (Section 2): the mode-n fibers become the
    columns, and among the remaining indices the earlier modes vary fastest
    (the ordering under which Eq. propMatricized holds)."""
    Z = as64(Z)
    return np.reshape(np.moveaxis(Z, n, 0), (Z.shape[n], -1), order="F")


def fold(Zn, n, shape):
    """Inverse of :func:`unfold` for a target tensor of size ``shape``."""
    shape = tuple(shape)
    rest = shape[:n] + shape[n + 1:]
    T = np.reshape(Zn, (shape[n],) + rest, order="F")
    return np.moveaxis(T, 0, n)


def ttm(Z, M, n):
    """n-mode product Z x_n M, defined by X_(n) = M Z_(n) (Section 2)."""
    Z = as64(Z)
    shape = list(Z.shape)
    shape[n] = M.shape[0]
    return fold(M @ unfold(Z, n), n, shape)


def ttm_modes(Z, mats, modes):
    """Z x_{n in modes} M^(n), applied one mode at a time in increasing n (Section 2 shorthand)."""
    X = as64(Z)
    for n in sorted(modes):
        X = ttm(X, mats[n], n)
    return X


def khatri_rao(mats):
    """A (.) B (.) ... = columnwise Kronecker products, in the order given (Section 2).
    The Kronecker product a (x) b puts b's index fastest."""
    R = mats[0].shape[1]
    out = mats[0]
    for B in mats[1:]:
        out = np.einsum("ir,jr->ijr", out, B).reshape(-1, R)
    return out


def phi(A, n):
    """Phi^(n) = A^(N) (.) ... (.) A^(n+1) (.) A^(n-1) (.) ... (.) A^(1)  (Eq. Phi)."""
    N = len(A)
    return khatri_rao([A[m] for m in range(N - 1, -1, -1) if m != n])


def mttkrp(Z, A, n):
    """Z_(n) Phi^(n), the left-hand side of Eq. fineeq1 (the MTTKRP)."""
    return unfold(Z, n) @ phi(A, n)


def gram(An):
    """Upsilon^(n) = A^(n)^T A^(n) (Eq. Gamma)."""
    return An.T @ An


def gamma(A, n):
    """Gamma^(n) = Hadamard product of Upsilon^(m) over m != n (Eq. Gamma)."""
    R = A[0].shape[1]
    G = np.ones((R, R))
    for m in range(len(A)):
        if m != n:
            G = G * gram(A[m])
    return G


def cp_full(A):
    """[[A^(1), ..., A^(N)]] = sum_r a_r^(1) o ... o a_r^(N) (Eq. tensorCP), formed via
    Eq. propMatricized: its mode-1 unfolding is A^(1) Phi^(1)^T."""
    shape = tuple(a.shape[0] for a in A)
    return fold(A[0] @ phi(A, 0).T, 0, shape)


def f_value(Z, A):
    """f = 1/2 ||Z - [[A]]||^2 (Eq. CPfunctional)."""
    D = as64(Z) - cp_full(A)
    return 0.5 * float(np.sum(D * D))


def gradient(Z, A, n):
    """G^(n) = -Z_(n) Phi^(n) + A^(n) Gamma^(n) (Eq. gradEqn)."""
    return -mttkrp(Z, A, n) + A[n] @ gamma(A, n)


def fas_operator(Z, A, n):
    """H^(n)({A}) = A^(n) Gamma^(n) - Z_(n) Phi^(n) (Eq. FASop); equal to G^(n)."""
    return A[n] @ gamma(A, n) - mttkrp(Z, A, n)


def g_value(Z, A):
    """g = (sum_n ||G^(n)||^2)^(1/2) / ||Z|| (Eq. gradConv)."""
    s = 0.0
    for n in range(len(A)):
        G = gradient(Z, A, n)
        s += float(np.sum(G * G))
    return np.sqrt(s) / float(np.linalg.norm(as64(Z).ravel()))
