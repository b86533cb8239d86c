"""Pins for oracle.tensor: brute-force sums, Section 2 identities, finite differences."""
import itertools

import numpy as np
import pytest

from oracle import tensor as T


def rand_tensor(dims, seed):
    return np.random.default_rng(seed).standard_normal(dims)


def rand_factors(dims, R, seed):
    rng = np.random.default_rng(seed + 17)
    return [rng.standard_normal((I, R)) for I in dims]


SHAPES = [(3, 4), (1, 5), (2, 3, 4), (5, 1, 3), (3, 2, 2, 3), (2, 3, 1, 2)]


@pytest.mark.parametrize("dims", SHAPES)
def test_unfold_matches_index_rule(dims):
    """Element (i_1..i_N) sits at row i_n, column sum_{k != n} i_k J_k with
    J_k = prod_{m < k, m != n} I_m (earlier modes fastest)."""
    Z = rand_tensor(dims, 1)
    N = len(dims)
    for n in range(N):
        Zn = T.unfold(Z, n)
        for idx in itertools.product(*[range(I) for I in dims]):
            col, J = 0, 1
            for k in range(N):
                if k == n:
                    continue
                col += idx[k] * J
                J *= dims[k]
            assert Zn[idx[n], col] == Z[idx]
        assert np.array_equal(T.fold(Zn, n, dims), Z)


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("R", [1, 3])
def test_mttkrp_bruteforce(dims, R):
    """Eq. fineeq1 left side against the elementwise sum m_{i r} = sum z prod_{m!=n} a^(m)."""
    Z = rand_tensor(dims, 2)
    A = rand_factors(dims, R, 3)
    N = len(dims)
    for n in range(N):
        M = np.zeros((dims[n], R))
        for idx in itertools.product(*[range(I) for I in dims]):
            for r in range(R):
                p = Z[idx]
                for m in range(N):
                    if m != n:
                        p *= A[m][idx[m], r]
                M[idx[n], r] += p
        got = T.mttkrp(Z, A, n)
        assert np.max(np.abs(got - M)) <= 1e-13 * max(1.0, np.max(np.abs(M)))


@pytest.mark.parametrize("dims", SHAPES)
def test_ttm_bruteforce(dims):
    Z = rand_tensor(dims, 4)
    rng = np.random.default_rng(5)
    for n in range(len(dims)):
        J = 3
        M = rng.standard_normal((J, dims[n]))
        X = T.ttm(Z, M, n)
        shape = list(dims)
        shape[n] = J
        ref = np.zeros(shape)
        for idx in itertools.product(*[range(I) for I in shape]):
            s = 0.0
            for i in range(dims[n]):
                src = list(idx)
                src[n] = i
                s += M[idx[n], i] * Z[tuple(src)]
            ref[idx] = s
        assert np.allclose(X, ref, rtol=1e-13, atol=1e-13)


def test_prop_kkr():
    """Eq. propKKR: (A1 B1) (.) ... (.) (AN BN) = (A1 (x) ... (x) AN)(B1 (.) ... (.) BN)."""
    rng = np.random.default_rng(6)
    K = 3
    As = [rng.standard_normal((2, 3)), rng.standard_normal((3, 2)), rng.standard_normal((2, 4))]
    Bs = [rng.standard_normal((3, K)), rng.standard_normal((2, K)), rng.standard_normal((4, K))]
    lhs = T.khatri_rao([a @ b for a, b in zip(As, Bs)])
    kron = As[0]
    for a in As[1:]:
        kron = np.kron(kron, a)
    rhs = kron @ T.khatri_rao(Bs)
    assert np.allclose(lhs, rhs, rtol=1e-13, atol=1e-13)


def test_khatri_rao_columns_are_kronecker():
    rng = np.random.default_rng(7)
    A, B = rng.standard_normal((3, 2)), rng.standard_normal((4, 2))
    KR = T.khatri_rao([A, B])
    for r in range(2):
        assert np.array_equal(KR[:, r], np.kron(A[:, r], B[:, r]))


@pytest.mark.parametrize("dims", [(2, 3, 4), (3, 2, 2, 3)])
def test_prop_matricized(dims):
    """Eq. propMatricized: X = Z x_1 A1 ... x_N AN  <=>  X_(n) = A_n Z_(n) (A_N (x) ... (x) A_1)^T
    (Kronecker over m != n)."""
    Z = rand_tensor(dims, 8)
    rng = np.random.default_rng(9)
    mats = [rng.standard_normal((I + 1, I)) for I in dims]
    X = T.ttm_modes(Z, mats, range(len(dims)))
    for n in range(len(dims)):
        kron = None
        for m in range(len(dims) - 1, -1, -1):
            if m == n:
                continue
            kron = mats[m] if kron is None else np.kron(kron, mats[m])
        assert np.allclose(T.unfold(X, n), mats[n] @ T.unfold(Z, n) @ kron.T, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims", [(3, 4), (2, 3, 4), (2, 2, 3, 2)])
def test_cp_full_bruteforce(dims):
    A = rand_factors(dims, 3, 10)
    X = T.cp_full(A)
    for idx in itertools.product(*[range(I) for I in dims]):
        s = 0.0
        for r in range(3):
            p = 1.0
            for m, i in enumerate(idx):
                p *= A[m][i, r]
            s += p
        assert abs(X[idx] - s) <= 1e-13 * max(1.0, abs(s))


@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 2, 3)])
def test_gradient_finite_differences(dims):
    """Eq. gradEqn is the derivative of Eq. CPfunctional (central differences)."""
    Z = rand_tensor(dims, 11)
    A = rand_factors(dims, 2, 12)
    h = 1e-6
    for n in range(len(dims)):
        G = T.gradient(Z, A, n)
        for i in range(dims[n]):
            for r in range(2):
                Ap = [a.copy() for a in A]
                Am = [a.copy() for a in A]
                Ap[n][i, r] += h
                Am[n][i, r] -= h
                fd = (T.f_value(Z, Ap) - T.f_value(Z, Am)) / (2 * h)
                assert abs(fd - G[i, r]) <= 1e-6 * max(1.0, abs(G[i, r]))


def test_gamma_is_hadamard_of_grams_and_spsd():
    dims = (4, 5, 3)
    A = rand_factors(dims, 3, 13)
    for n in range(3):
        G = T.gamma(A, n)
        ref = np.ones((3, 3))
        for m in range(3):
            if m != n:
                for r in range(3):
                    for s in range(3):
                        ref[r, s] *= sum(A[m][i, r] * A[m][i, s] for i in range(dims[m]))
        assert np.allclose(G, ref, rtol=1e-13)
        assert np.allclose(G, G.T)
        assert np.linalg.eigvalsh(G).min() > -1e-12


def test_g_zero_at_exact_decomposition_and_f_zero():
    dims = (4, 5, 6)
    A = rand_factors(dims, 2, 14)
    Z = T.cp_full(A)
    assert T.f_value(Z, A) < 1e-25
    assert T.g_value(Z, A) < 1e-13
    # g is the scaled norm of the stacked gradients (Eq. gradConv)
    B = [a * 1.01 for a in A]
    s = sum(np.sum(T.gradient(Z, B, n) ** 2) for n in range(3))
    assert np.isclose(T.g_value(Z, B), np.sqrt(s) / np.linalg.norm(Z))


def test_f_matches_elementwise_definition():
    dims = (3, 4, 2)
    Z = rand_tensor(dims, 15)
    A = rand_factors(dims, 2, 16)
    s = 0.0
    for idx in itertools.product(*[range(I) for I in dims]):
        x = sum(A[0][idx[0], r] * A[1][idx[1], r] * A[2][idx[2], r] for r in range(2))
        s += (Z[idx] - x) ** 2
    assert np.isclose(T.f_value(Z, A), 0.5 * s, rtol=1e-13)


def test_fas_operator_equals_gradient():
    dims = (3, 4, 5)
    Z = rand_tensor(dims, 18)
    A = rand_factors(dims, 2, 19)
    for n in range(3):
        assert np.allclose(T.fas_operator(Z, A, n), T.gradient(Z, A, n))


@pytest.mark.parametrize("dims", [(5, 4, 6), (4, 3, 5, 2)])
def test_mode_products_commute(dims):
    """The restriction's mode products commute (Section 2: x_m and x_n act on different indices):
    applying them in increasing order, or mode 1 first and then the last mode down to mode 2 (the
    order the tensor-core path uses), gives the full contraction with every matrix, written out
    with einsum."""
    Z = rand_tensor(dims, 11)
    rng = np.random.default_rng(12)
    Ms = [rng.standard_normal(((I + 1) // 2, I)) for I in dims]
    N = len(dims)
    inc = Z
    for n in range(N):
        inc = T.ttm(inc, Ms[n], n)
    alt = T.ttm(Z, Ms[0], 0)
    for n in range(N - 1, 0, -1):
        alt = T.ttm(alt, Ms[n], n)
    letters = "abcd"[:N]
    spec = letters + "," + ",".join("%s%s" % (c.upper(), c) for c in letters) + "->" + letters.upper()
    ref = np.einsum(spec, Z, *Ms)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(inc - ref)) <= 1e-12 * scale
    assert np.max(np.abs(alt - ref)) <= 1e-12 * scale
