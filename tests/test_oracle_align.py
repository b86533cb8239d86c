"""Pins of the alignment used for factor errors (Section 1: a CP decomposition is unique only
up to scaling and permutation of its rank-one terms)."""
import numpy as np

from oracle import align, tensor as T


def factors(dims, R, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((I, R)) for I in dims]


def test_indeterminacies_give_zero_error():
    """Permuted components, rescaled columns whose scales multiply to one per component, and
    sign flips in pairs of modes represent the same tensor: error 0."""
    A = factors((7, 6, 5), 4, 1)
    rng = np.random.default_rng(2)
    perm = rng.permutation(4)
    s0 = rng.uniform(0.5, 2.0, 4) * np.array([1, -1, 1, -1])
    s1 = rng.uniform(0.5, 2.0, 4) * np.array([-1, -1, 1, 1])
    s2 = 1.0 / (s0 * s1)
    B = [A[0][:, perm] * s0[perm], A[1][:, perm] * s1[perm], A[2][:, perm] * s2[perm]]
    assert np.allclose(T.cp_full(A), T.cp_full(B))
    assert align.factor_error(A, B) < 1e-14


def test_known_perturbation_size():
    """Adding eps * e, with e a unit vector orthogonal to the column, to one column of one mode
    of equal-norm sign-canonical factors keeps the column norm to second order, so the error
    is eps / ||B^(n)||_F on that mode and O(eps^2) on the others."""
    A = factors((9, 8, 7), 3, 3)
    U, lam = align.canonical(A)
    B = align.equal_norm(U, lam)
    u = B[1][:, 1] / np.linalg.norm(B[1][:, 1])
    v = np.random.default_rng(6).standard_normal(8)
    v -= (v @ u) * u
    E = np.zeros_like(B[1])
    E[:, 1] = v / np.linalg.norm(v)
    eps = 1e-7
    C = [B[0], B[1] + eps * E, B[2]]
    want = eps / np.linalg.norm(B[1])
    got = align.factor_error(B, C)
    assert abs(got - want) <= 1e-3 * want


def test_different_tensors_are_far():
    A = factors((6, 6, 6), 2, 4)
    B = factors((6, 6, 6), 2, 5)
    assert align.factor_error(A, B) > 0.1
