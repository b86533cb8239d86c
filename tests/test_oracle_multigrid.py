"""Pins for oracle.multigrid: operator structure, exactness statements of Sections 4-5,
the coarse-gradient identity, and two-level convergence on the 20^3 rank-3 problem."""
import numpy as np
import pytest

from oracle import tensor as T, als as ALS, multigrid as MG, align
from paper_1111_6091_gb300 import synth


@pytest.mark.parametrize("I", [2, 3, 4, 7, 10, 13, 20])
def test_coarsening_structure(I):
    Ic = MG.coarse_size(I)
    assert Ic == (I + 1) // 2
    rng = np.random.default_rng(I)
    U = rng.standard_normal((I, 6))
    P = MG.interpolation(U, np.ones(6), I)
    assert P.shape == (I, Ic)
    for i in range(I):
        nz = np.flatnonzero(P[i])
        if i % 2 == 0:
            assert list(nz) == [i // 2] and P[i, i // 2] == 1.0
        else:
            expect = [(i - 1) // 2] + ([(i + 1) // 2] if i + 1 < I else [])
            assert set(nz) <= set(expect)
    B = P.T @ P
    assert np.allclose(np.triu(B, 2), 0) and np.allclose(np.tril(B, -2), 0)  # tridiagonal


def test_ls_weights_reproduce_interpolable_data():
    """If every fitted vector is exactly P_true u_c, the weighted LS returns P_true."""
    I = 11
    rng = np.random.default_rng(1)
    P_true = MG.interpolation(rng.standard_normal((I, 4)), np.ones(4), I)  # structure
    for i in range(1, I, 2):
        P_true[i, np.flatnonzero(P_true[i])] = rng.uniform(0.2, 0.8, size=np.count_nonzero(P_true[i]))
    Uc = rng.standard_normal((MG.coarse_size(I), 6))
    U = P_true @ Uc
    w = rng.uniform(0.1, 10.0, size=6)
    assert np.allclose(MG.interpolation(U, w, I), P_true, rtol=1e-12, atol=1e-12)


def test_ls_weights_weighted_normal_equations():
    """One fine row by hand: the 2x2 weighted normal equations."""
    I = 5
    rng = np.random.default_rng(2)
    U = rng.standard_normal((I, 4))
    w = np.array([1.0, 2.0, 3.0, 4.0])
    P = MG.interpolation(U, w, I)
    X = np.stack([U[0], U[2]], axis=1)
    W = np.diag(w)
    sol = np.linalg.lstsq(np.sqrt(W) @ X, np.sqrt(W) @ U[1], rcond=None)[0]
    assert np.allclose(P[1, [0, 1]], sol, rtol=1e-10)
    # right endpoint of an even-size mode: one-point fit
    I = 6
    U = rng.standard_normal((I, 4))
    P = MG.interpolation(U, w, I)
    x, y = U[4], U[5]
    assert np.isclose(P[5, 2], np.sum(w * x * y) / np.sum(w * x * x))


def test_singular_normal_equations_fallback():
    I = 5
    U = np.ones((I, 3))  # coarse neighbours identical -> singular 2x2 system
    P = MG.interpolation(U, np.ones(3), I)
    assert np.allclose(P[1, [0, 1]], 0.5) and np.allclose(P[3, [1, 2]], 0.5)


@pytest.mark.parametrize("I", [5, 8, 20, 33])
def test_phat_orthonormal(I):
    """P-hat^T P-hat = L^{-1} P^T P L^{-T} = I."""
    rng = np.random.default_rng(I)
    P = MG.interpolation(rng.standard_normal((I, 6)), rng.uniform(0.5, 2, 6), I)
    Phat, Rhat = MG.transform(P)
    assert np.allclose(Phat.T @ Phat, np.eye(P.shape[1]), atol=1e-13)
    assert np.array_equal(Rhat, Phat.T)
    # L^{-1} P^T with L lower triangular: R-hat is P-hat transposed and lies in range(P^T)
    assert np.allclose(Phat @ (Rhat @ P), P, atol=1e-12)


def _hier_for(dims, R, seed):
    rng = np.random.default_rng(seed)
    Ps, Phats, Rhats = [], [], []
    for I in dims:
        P = MG.interpolation(rng.standard_normal((I, 2 * R)), np.ones(2 * R), I)
        Phat, Rhat = MG.transform(P)
        Ps.append(P), Phats.append(Phat), Rhats.append(Rhat)
    return Ps, Phats, Rhats


def test_cgc_exact_when_factors_in_range():
    """Section 4.1: if A^(n) = P A_c^(n) and the coarse problem is solved exactly, the CGC
    returns A.  The coarse tensor is exactly [[L^T A_c]] and P-hat L^T A_c = A."""
    dims, R = (9, 8, 7), 2
    Ps, Phats, Rhats = _hier_for(dims, R, 3)
    rng = np.random.default_rng(4)
    Ac = [rng.standard_normal((P.shape[1], R)) for P in Ps]
    A = [P @ a for P, a in zip(Ps, Ac)]
    Z = T.cp_full(A)
    Zc = MG.coarse_tensor(Z, Rhats, [True] * 3)
    Ls = [np.linalg.cholesky(P.T @ P) for P in Ps]
    Ahat = [L.T @ a for L, a in zip(Ls, Ac)]
    assert np.allclose(Zc, T.cp_full(Ahat), rtol=1e-12, atol=1e-12)
    assert T.g_value(Zc, Ahat) < 1e-12
    Acgc = [Ph @ a for Ph, a in zip(Phats, Ahat)]
    for a, b in zip(A, Acgc):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_coarse_gradient_is_restricted_fine_gradient():
    """R-hat G^(n)(P-hat A_hat) = G_c^(n)(A_hat), from Eq. propKKR and P-hat^T P-hat = I."""
    dims, R = (9, 6, 7), 3
    _, Phats, Rhats = _hier_for(dims, R, 5)
    rng = np.random.default_rng(6)
    Z = rng.standard_normal(dims)
    Zc = MG.coarse_tensor(Z, Rhats, [True] * 3)
    Ahat = [rng.standard_normal((Ph.shape[1], R)) for Ph in Phats]
    Afine = [Ph @ a for Ph, a in zip(Phats, Ahat)]
    for n in range(3):
        assert np.allclose(Rhats[n] @ T.gradient(Z, Afine, n), T.gradient(Zc, Ahat, n),
                           rtol=1e-11, atol=1e-11)


def test_partial_coarsening_uses_identity():
    """Modes not in I_c are left as they are (Eq. coarseapprox_new)."""
    dims = (9, 4, 7)
    _, Phats, Rhats = _hier_for(dims, 2, 7)
    rng = np.random.default_rng(8)
    Z = rng.standard_normal(dims)
    Ic = [True, False, True]
    Zc = MG.coarse_tensor(Z, Rhats, Ic)
    ref = T.ttm(T.ttm(Z, Rhats[0], 0), Rhats[2], 2)
    assert np.allclose(Zc, ref)
    A = [rng.standard_normal((I, 2)) for I in dims]
    Ac = MG.restrict_factors(A, Rhats, Ic)
    assert np.array_equal(Ac[1], A[1]) and np.allclose(Ac[0], Rhats[0] @ A[0])


def _small_problem():
    p = synth.make_problem((20, 20, 20), 3, dtype=np.float64, seed=0)
    opts = MG.Options(coarsest=(10, 10, 10), tol=1e-10)
    return p, opts


def test_fas_fixed_point():
    """Section 5.2: the exact solution (normalized, sorted) is a fixed point of one CP-FAS
    V-cycle with Gauss-Seidel relaxation, for any hierarchy."""
    p, opts = _small_problem()
    s = MG.mg_setup(p.Z, p.A0, p.tfms, MG.Options(coarsest=(10, 10, 10), max_setup_cycles=1))
    A, _ = ALS.normalize(p.truth)
    A = ALS.sort_components(A)
    B = MG.cp_fas(s.levels, 0, None, A, opts)
    for a, b in zip(A, B):
        assert np.allclose(a, b, rtol=1e-10, atol=1e-10 * np.max(np.abs(a)))


def test_fas_rhs_two_level_identity():
    """If A solves H(A) = F exactly, the restricted A~_c solves the coarse problem exactly:
    F_c = H_c(A~_c) (Eq. FASrhs), and the CGC then leaves A unchanged (Eq. FASCGC)."""
    p, opts = _small_problem()
    s = MG.mg_setup(p.Z, p.A0, p.tfms, MG.Options(coarsest=(10, 10, 10), max_setup_cycles=1))
    rng = np.random.default_rng(3)
    A = [rng.standard_normal((20, 3)) for _ in range(3)]
    F = [T.fas_operator(p.Z, A, n) for n in range(3)]      # A is an exact solution for this F
    At = MG.restrict_factors(A, s.levels[0].Rhat, s.levels[0].Ic)
    Fc = MG.fas_rhs(s.levels, 0, F, A, At)
    for n in range(3):
        hc = T.fas_operator(s.levels[1].Z, At, n)
        assert np.allclose(Fc[n], hc, rtol=1e-12, atol=1e-12 * np.max(np.abs(hc)))
    # and with a residual: F_c - H_c(A~_c) is the restricted residual
    F2 = [f + 1.0 for f in F]
    Fc2 = MG.fas_rhs(s.levels, 0, F2, A, At)
    for n in range(3):
        assert np.allclose(Fc2[n] - Fc[n], s.levels[0].Rhat[n] @ np.ones((20, 3)), rtol=1e-9,
                           atol=1e-9 * np.max(np.abs(Fc[n])))


def test_two_level_mg_converges_20cubed():
    """Two-level multilevel solver: g < 1e-10 and factor error <= 1e-10 against the truth."""
    p, opts = _small_problem()
    r = MG.multilevel(p.Z, p.A0, p.tfms, opts)
    assert r.converged
    assert len(r.levels) == 2
    assert T.g_value(p.Z, r.A) < 1e-10
    assert align.factor_error(p.truth, r.A) <= 1e-10


def test_setup_stagnation_rule(monkeypatch):
    """Eq. stagnation: setup stops at the first cycle k >= 3 with g_k > (1 - eps) g_{k-1}."""
    p, _ = _small_problem()
    seq = iter([1.0, 0.5, 0.46, 0.3, 0.2])
    monkeypatch.setattr(MG, "g_value", lambda Z, A: next(seq))
    s = MG.mg_setup(p.Z, p.A0, p.tfms, MG.Options(coarsest=(10, 10, 10), nu1_setup=1,
                                                    nu2_setup=1, nuc_setup=1, tol=1e-30))
    assert s.setup_cycles == 3          # 0.46 > 0.9 * 0.5
    seq2 = iter([1.0, 0.95, 0.8, 0.5, 0.2])
    monkeypatch.setattr(MG, "g_value", lambda Z, A: next(seq2))
    s = MG.mg_setup(p.Z, p.A0, p.tfms, MG.Options(coarsest=(10, 10, 10), nu1_setup=1,
                                                    nu2_setup=1, nuc_setup=1, tol=1e-30))
    assert s.setup_cycles == 5          # no stagnation from cycle 3 on; cap of five


def test_solve_stagnation_rebuild_once(monkeypatch):
    """Section 6.1: from the sixth solve cycle, g_new >= g_old discards the iterate and rebuilds
    once; later stagnation is ignored (without the fallback)."""
    p, opts = _small_problem()
    s = MG.mg_setup(p.Z, p.A0, p.tfms, MG.Options(coarsest=(10, 10, 10), max_setup_cycles=1))
    gs = iter([1.0] + [0.9, 0.8, 0.7, 0.6, 0.5, 0.55, 0.45, 0.5, 0.4] + [0.3] * 20)
    monkeypatch.setattr(MG, "g_value", lambda Z, A: next(gs))
    calls = []
    real = MG.down_sweep
    monkeypatch.setattr(MG, "down_sweep", lambda *a: (calls.append(1), real(*a))[1])
    o = MG.Options(coarsest=(10, 10, 10), tol=1e-30, max_cycles=10, nuc=1)
    r = MG.mg_fas_solve(p.Z, s.levels, p.A0, s.tfms, o)
    assert r.restarted and len(calls) == 1
    assert r.solve_cycles == 10


def test_last_mode_gradient_is_zero_after_als_so_weights_cap():
    """After one ALS iteration the last mode's gradient vanishes (exact least-squares update,
    then a column rescaling that keeps it zero), so its block weights hit the cap and the
    interpolation of that mode is the unweighted fit, whatever the rounding noise."""
    p = synth.make_problem((12, 10, 8), 3, congruence=0.5, eta_homo=0.1, dtype=np.float64, seed=7)
    blocks = [ALS.als_sweep(p.Z, b) for b in p.tfms]
    for b in blocks:
        G = T.gradient(p.Z, b, 2)
        assert np.linalg.norm(G) <= 1e-12 * np.linalg.norm(b[2] @ T.gamma(b, 2))
        assert MG.block_weight(p.Z, b, 2) == MG.W_CAP
        assert MG.block_weight(p.Z, b, 0) < MG.W_CAP
    U = np.hstack([b[2] for b in blocks])
    w = np.array([MG.block_weight(p.Z, b, 2) for b in blocks]).repeat(3)
    assert np.allclose(MG.interpolation(U, w, 8), MG.interpolation(U, np.ones(6), 8), rtol=1e-12)


def _nested_exact_hierarchy(dims, R, seed):
    """Three levels with hand-built interpolation operators and a tensor whose factors lie in
    the range of the whole chain: A_0 = P-hat_0 A_1, A_1 = P-hat_1 A_2.  Since R-hat P-hat = I,
    every level's tensor is exactly [[A_l]]."""
    rng = np.random.default_rng(seed)
    ops, sizes = [], [tuple(dims)]
    for _ in range(2):
        lv = []
        for I in sizes[-1]:
            P = MG.interpolation(rng.standard_normal((I, 2 * R)), np.ones(2 * R), I)
            lv.append((P,) + MG.transform(P))
        ops.append(lv)
        sizes.append(tuple(MG.coarse_size(I) for I in sizes[-1]))
    A2 = [rng.standard_normal((I, R)) for I in sizes[2]]
    A1 = [o[1] @ a for o, a in zip(ops[1], A2)]
    A0 = [o[1] @ a for o, a in zip(ops[0], A1)]
    Z0 = T.cp_full(A0)
    Z1 = MG.coarse_tensor(Z0, [o[2] for o in ops[0]], [True] * 3)
    Z2 = MG.coarse_tensor(Z1, [o[2] for o in ops[1]], [True] * 3)
    levels = [MG.Level(Z, [True] * 3, [o[0] for o in op], [o[1] for o in op], [o[2] for o in op])
              for Z, op in ((Z0, ops[0]), (Z1, ops[1]))]
    levels.append(MG.Level(Z2, [False] * 3, [None] * 3, [None] * 3, [None] * 3))
    return levels, (A0, A1, A2), rng


def test_fmg_recovers_factors_in_the_range_of_the_interpolation_chain():
    """Algorithm 3 (nested iteration): when the fine factors lie in the range of P-hat_0 P-hat_1,
    every coarse tensor is exactly the restricted decomposition, so the coarsest ALS solve followed
    by prolongation (P-hat, not P) and one CP-FAS cycle per level returns the exact fine
    decomposition."""
    levels, (A0, A1, A2), rng = _nested_exact_hierarchy((13, 11, 9), 2, 21)
    assert np.allclose(levels[1].Z, T.cp_full(A1), atol=1e-12 * np.max(np.abs(levels[1].Z)))
    assert np.allclose(levels[2].Z, T.cp_full(A2), atol=1e-12 * np.max(np.abs(levels[2].Z)))
    opts = MG.Options(tol=1e-10)
    # exact coarsest start, no coarse iterations: the prolongated factors are already exact
    A = MG.fmg_cp_fas(levels, A2, 0, opts)
    assert T.g_value(levels[0].Z, A) < 1e-12
    assert align.factor_error(A0, A) < 1e-10
    # perturbed coarsest start: the coarsest ALS converges, the rest follows
    start = [a + 0.3 * np.std(a) * rng.standard_normal(a.shape) for a in A2]
    A = MG.fmg_cp_fas(levels, start, 300, opts)
    assert T.g_value(levels[0].Z, A) < 1e-9
    assert align.factor_error(A0, A) < 1e-7
    # prolongating with P instead of P-hat (a plausible slip) would not be exact
    bad = [L.P[n] @ a for L in levels[:1] for n, a in enumerate(MG.fmg_cp_fas(levels[1:], A2, 0, opts))]
    assert T.g_value(levels[0].Z, bad) > 1e-3
