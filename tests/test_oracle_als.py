"""Pins for oracle.als: exact recovery, monotone f, Eckart-Young, power method, GS fixed point."""
import numpy as np
import pytest

from oracle import tensor as T, als as ALS, align
from paper_1111_6091_gb300 import synth


def test_pinv_solve_equals_pinv_for_spd_and_singular():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((6, 4))
    G = X.T @ X
    M = rng.standard_normal((5, 4))
    assert np.allclose(ALS.pinv_right_solve(M, G), M @ np.linalg.inv(G), rtol=1e-10)
    # rank-deficient Gamma: the Cholesky pivot test must fall through to the pseudoinverse
    Y = rng.standard_normal((6, 2))
    Gs = (Y @ rng.standard_normal((2, 4))).T @ (Y @ rng.standard_normal((2, 4)))
    Gs = 0.5 * (Gs + Gs.T)
    Gs = Gs @ Gs  # SPSD, rank 2
    got = ALS.pinv_right_solve(M, Gs)
    ref = M @ np.linalg.pinv(Gs, rcond=4 * np.finfo(float).eps)
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-8)


def test_normalize_keeps_tensor_and_equalizes_norms():
    rng = np.random.default_rng(1)
    A = [rng.standard_normal((I, 3)) * s for I, s in [(4, 10.0), (5, 0.1), (3, 2.0)]]
    B, lam = ALS.normalize(A)
    assert np.allclose(T.cp_full(A), T.cp_full(B), rtol=1e-13, atol=1e-12)
    for b in B:
        assert np.allclose(np.linalg.norm(b, axis=0), lam, rtol=1e-13)
    ref = np.prod([np.linalg.norm(a, axis=0) for a in A], axis=0) ** (1 / 3)
    assert np.allclose(lam, ref)


def test_sort_decreasing_lambda_ties_stable():
    A = [np.array([[1.0, 3.0, 2.0, 3.0]]), np.array([[1.0, 1.0, 1.0, 1.0]])]
    B = ALS.sort_components(A)
    assert np.array_equal(B[0][0], [3.0, 3.0, 2.0, 1.0])
    # the two lambda = sqrt(3) components keep their original order (index 1 before 3)
    A2 = [np.array([[1.0, 3.0, 2.0, 3.0], [0, 1, 2, 3]]), np.ones((1, 4))]
    B2 = ALS.sort_components([A2[0] / np.array([1, 1, 1, 1.0]), A2[1]])
    lam = np.linalg.norm(B2[0], axis=0)
    assert np.all(np.diff(lam) <= 0)


def test_exact_recovery_20cubed_rank3():
    """An exact rank-3 tensor with N(0,1) factors is recovered: f -> 0, aligned error <= 1e-10."""
    p = synth.make_problem((20, 20, 20), 3, dtype=np.float64, seed=0)
    A, it = ALS.als(p.Z, p.A0, 10000, tol=1e-12, g_fn=T.g_value)
    assert T.g_value(p.Z, A) < 1e-12
    assert T.f_value(p.Z, A) < 1e-16 * np.sum(p.Z ** 2)
    assert align.factor_error(p.truth, A) <= 1e-10


def test_f_monotone_after_every_mode_update():
    """Each mode update is an exact least-squares minimizer, and normalization keeps [[A]]."""
    p = synth.make_problem((12, 10, 8), 4, congruence=0.8, eta_homo=0.05, dtype=np.float64, seed=3)
    A = [a.copy() for a in p.A0]
    f_prev = T.f_value(p.Z, A)
    for _ in range(15):
        for n in range(3):
            A[n] = ALS.pinv_right_solve(T.mttkrp(p.Z, A, n), T.gamma(A, n))
            f = T.f_value(p.Z, A)
            assert f <= f_prev * (1 + 1e-12) + 1e-12
            f_prev = f
        A, _ = ALS.normalize(A)
        assert abs(T.f_value(p.Z, A) - f_prev) <= 1e-10 * max(1.0, f_prev)


@pytest.mark.parametrize("R", [1, 2, 3])
def test_two_way_case_is_eckart_young(R):
    """N = 2: CP is a rank-R matrix approximation; ALS reaches f* = 1/2 sum_{i>R} sigma_i^2."""
    rng = np.random.default_rng(4 + R)
    U, _ = np.linalg.qr(rng.standard_normal((15, 15)))
    V, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    sig = np.array([10.0, 7.0, 5.0, 3.0, 1.0] + [0.5] * 7)
    Z = (U[:, :12] * sig) @ V.T
    A0 = [rng.standard_normal((15, R)), rng.standard_normal((12, R))]
    A, _ = ALS.als(Z, A0, 3000, tol=1e-13, g_fn=T.g_value)
    fstar = 0.5 * np.sum(np.linalg.svd(Z, compute_uv=False)[R:] ** 2)
    assert np.isclose(T.f_value(Z, A), fstar, rtol=1e-10)


def test_rank_one_is_power_method():
    """R = 1 on an exact rank-1 tensor: one sweep recovers it exactly (HOPM step)."""
    rng = np.random.default_rng(9)
    A = [rng.standard_normal((I, 1)) for I in (5, 6, 7)]
    Z = T.cp_full(A)
    B = ALS.als_sweep(Z, [rng.standard_normal((I, 1)) for I in (5, 6, 7)])
    assert T.f_value(Z, B) < 1e-24 * np.sum(Z ** 2) + 1e-26


def test_gauss_seidel_converges_and_keeps_fixed_point():
    rng = np.random.default_rng(10)
    X = rng.standard_normal((8, 4))
    G = X.T @ X + np.eye(4)
    Xs = rng.standard_normal((5, 4))
    B = Xs @ G
    # many sweeps converge to the solution of X Gamma = B
    Y = ALS.gauss_seidel_rows(np.zeros((5, 4)), G, B, sweeps=400)
    assert np.allclose(Y, Xs, rtol=1e-9, atol=1e-9)
    # one sweep by hand on one row
    x0 = rng.standard_normal((1, 4))
    b = B[:1]
    x = x0.copy()
    for r in range(4):
        x[0, r] = (b[0, r] - sum(G[r, s] * x[0, s] for s in range(4) if s != r)) / G[r, r]
    assert np.allclose(ALS.gauss_seidel_rows(x0, G, b, sweeps=1), x)
    # singular Gamma: an exact solution is left unchanged (Section 5.2)
    Ysing = rng.standard_normal((6, 2)) @ rng.standard_normal((2, 4))
    Gs = Ysing.T @ Ysing
    Xf = rng.standard_normal((3, 4))
    assert np.allclose(ALS.gauss_seidel_rows(Xf, Gs, Xf @ Gs, sweeps=10), Xf, atol=1e-10)


def test_bngs_with_zero_rhs_reaches_als_fixed_point():
    """With F = 0 and many GS sweeps, BNGS converges to the same stationary point as ALS."""
    p = synth.make_problem((10, 9, 8), 2, dtype=np.float64, seed=5)
    A = [a.copy() for a in p.A0]
    for _ in range(300):
        A = ALS.bngs_sweep(p.Z, A, None, gs_sweeps=10, finest=True)
    assert T.g_value(p.Z, A) < 1e-10
    assert align.factor_error(p.truth, A) < 1e-9
