"""Pins for the parts of oracle.multigrid that the convergence tests do not fix on their own:
which vectors the interpolation fits on the first and later setup cycles (Algorithm 1,
Section 4.4), the operator rebuild that keeps the boot factors frozen (Section 6.1), the tie
order of the component sort (end of Section 3), and the FAS right-hand side of modes that stop
coarsening before the others (Section 4.5, Eq. FASrhs)."""
import numpy as np
import pytest

from oracle import tensor as T, als as ALS, multigrid as MG, align
from paper_1111_6091_gb300 import synth


def _interp_with_weights(I, a, b, rng):
    """An interpolation matrix whose two-point rows are (a, b) and whose one-point row (the
    right endpoint of an even-size mode) is a + b."""
    P = np.zeros((I, MG.coarse_size(I)))
    for j in range(MG.coarse_size(I)):
        P[2 * j, j] = 1.0
    for i in range(1, I, 2):
        s = MG.stencil(i, I)
        P[i, s] = [a, b] if len(s) == 2 else [a + b]
    return P


def _in_range(P, R, rng):
    return P @ rng.standard_normal((P.shape[1], R))


@pytest.mark.parametrize("dims", [(9, 7, 5), (8, 6, 10)])
def test_build_operators_fits_only_tfms_on_the_first_cycle(dims):
    """Algorithm 1 fits P to the test factor matrices alone on the first cycle and to the TFMs
    together with the boot factors afterwards.  TFMs lying exactly in range(P_true) give P_true
    from the first-cycle fit whatever the boot factors are; adding boot factors that are not in
    that range changes the fit; adding boot factors that are in it does not."""
    rng = np.random.default_rng(5)
    R = 2
    Z = rng.standard_normal(dims)
    Ptrue = [_interp_with_weights(I, 0.3, 0.7, rng) for I in dims]
    tfms = [[_in_range(Ptrue[n], R, rng) for n in range(3)] for _ in range(2)]
    A_out = [rng.standard_normal((I, R)) for I in dims]
    A_in = [_in_range(Ptrue[n], R, rng) for n in range(3)]
    Ic = [True] * 3
    P1, _, _ = MG.build_operators(Z, A_out, tfms, Ic, first_cycle=True)
    P2, _, _ = MG.build_operators(Z, A_out, tfms, Ic, first_cycle=False)
    P3, _, _ = MG.build_operators(Z, A_in, tfms, Ic, first_cycle=False)
    for n in range(3):
        assert np.allclose(P1[n], Ptrue[n], rtol=0, atol=1e-12)
        assert np.max(np.abs(P2[n] - Ptrue[n])) > 1e-3
        assert np.allclose(P3[n], Ptrue[n], rtol=0, atol=1e-12)


def test_down_sweep_freezes_boot_factors_and_relaxes_tfms_nu1_times(monkeypatch):
    """Section 6.1's rebuild: on every level but the coarsest, each TFM block is relaxed by
    nu1 setup ALS iterations and the operators are rebuilt; the boot factors are restricted but
    never relaxed, and nothing is relaxed on the coarsest level."""
    p = synth.make_problem((20, 20, 20), 3, congruence=0.6, eta_homo=0.01, dtype=np.float64, seed=4)
    opts = MG.Options(coarsest=(5, 5, 5), nu1_setup=2)
    A = [a.copy() for a in p.A0]
    calls = []
    real = MG.als

    def spy(Z, X, iters, *a, **k):
        calls.append((Z.shape, [x.copy() for x in X], iters))
        return real(Z, X, iters, *a, **k)

    monkeypatch.setattr(MG, "als", spy)
    levels, tfms = MG.down_sweep(p.Z, A, p.tfms, opts)
    monkeypatch.setattr(MG, "als", real)
    assert [L.dims for L in levels] == [(20, 20, 20), (10, 10, 10), (5, 5, 5)]
    # the caller's boot factors are untouched
    assert all(np.array_equal(a, b) for a, b in zip(A, p.A0))
    # one nu1-iteration call per TFM block on each of the two non-coarsest levels
    assert [(c[0], c[2]) for c in calls] == [((20, 20, 20), 2)] * 2 + [((10, 10, 10), 2)] * 2
    # the returned fine TFMs are the inputs after exactly nu1 iterations
    for got, t in zip(tfms, p.tfms):
        ref = real(p.Z, t, 2)[0]
        assert all(np.array_equal(x, y) for x, y in zip(got, ref))
    # no relaxation ever received the boot factors (fine, or restricted to level 1)
    A1 = MG.restrict_factors(A, levels[0].Rhat, levels[0].Ic)
    for shape, X, _ in calls:
        ref = A if shape == (20, 20, 20) else A1
        assert not all(np.allclose(x, y) for x, y in zip(X, ref))
    # the level-1 TFMs that were relaxed are the restrictions of the relaxed fine TFMs
    lvl1 = [c[1] for c in calls if c[0] == (10, 10, 10)]
    for X, t in zip(lvl1, tfms):
        R1 = MG.restrict_factors(t, levels[0].Rhat, levels[0].Ic)
        assert all(np.allclose(x, y, rtol=1e-13, atol=1e-13) for x, y in zip(X, R1))


def test_sort_ties_keep_the_lower_index_first():
    """Equal lambda_r: the component with the lower index comes first (the stable reading)."""
    A = [np.array([[3.0, 1.0, 0.0, 2.0],
                   [0.0, 0.0, 3.0, 0.0]]),
         np.ones((1, 4))]
    B = ALS.sort_components(A)
    # lambda = (3, 1, 3, 2): order 0, 2, 3, 1 -- index 0 before index 2 among the ties
    assert np.array_equal(B[0], A[0][:, [0, 2, 3, 1]])
    A_rev = [A[0][:, [2, 1, 0, 3]], A[1]]
    B_rev = ALS.sort_components(A_rev)
    assert np.array_equal(B_rev[0], A_rev[0][:, [0, 2, 3, 1]])


# ------------------------------------------------------------------ partial coarsening
UNEVEN = (40, 12, 40)


def _uneven_problem(eta=0.0):
    """A rank-3 tensor 40 x 12 x 40 with coarsest size 10 in every mode: mode 2 (size 12) is
    coarsened once, to 6, and then stops, while modes 1 and 3 go on to 10 -- so on level 1
    mode 2 is outside I_c (Section 4.5)."""
    p = synth.make_problem(UNEVEN, 3, eta_homo=eta, dtype=np.float64, seed=3)
    opts = MG.Options(coarsest=(10, 10, 10), max_setup_cycles=1, tol=1e-10)
    s = MG.mg_setup(p.Z, p.A0, p.tfms, opts)
    return p, opts, s


def test_uneven_hierarchy_stops_one_mode_early():
    _, _, s = _uneven_problem()
    assert [L.dims for L in s.levels] == [(40, 12, 40), (20, 6, 20), (10, 6, 10)]
    assert [L.Ic for L in s.levels] == [[True, True, True], [True, False, True], [False] * 3]


def _fixed_point_defect(Z, A, levels):
    A, _ = ALS.normalize(A)
    A = ALS.sort_components(A)
    B = MG.cp_fas(levels, 0, None, A, MG.Options(coarsest=(10, 10, 10), tol=1e-10))
    return max(np.max(np.abs(a - b)) / np.max(np.abs(a)) for a, b in zip(A, B))


def test_fas_rhs_of_non_coarsened_modes_keeps_the_fixed_point(monkeypatch):
    """Eq. FASrhs with R-hat = I for a mode outside I_c, F_c = H_c(A~_c) + F - H(A), leaves a
    stationary point of the fine problem a fixed point of a three-level CP-FAS cycle.  The
    alternative F_c = F for such modes, planted here in the oracle, does not: the coarse
    problem's solution is then no longer the restricted stationary point, and the correction
    moves it."""
    # a noisy tensor, so that no level tensor is an exact CP and H_c(A~_c) != 0 on the coarse
    # levels; the start is an ALS stationary point (H(A) = 0 to rounding) of the fine problem
    p, opts, s = _uneven_problem(eta=0.05)
    A, _ = ALS.als(p.Z, p.A0, 3000, tol=1e-13, g_fn=T.g_value)
    assert T.g_value(p.Z, A) < 1e-13
    assert _fixed_point_defect(p.Z, A, s.levels) < 1e-12
    real = MG.fas_rhs

    def planted(levels, lvl, F, A, At):
        Fc = real(levels, lvl, F, A, At)
        L = levels[lvl]
        for n in range(len(A)):
            if not L.Ic[n]:
                Fc[n] = np.zeros_like(Fc[n]) if F is None else F[n].copy()
        return Fc

    monkeypatch.setattr(MG, "fas_rhs", planted)
    assert _fixed_point_defect(p.Z, A, s.levels) > 1e-6


def test_uneven_hierarchy_multilevel_converges():
    """The full multilevel solver on the uneven exact problem reaches g < 1e-10 and the exact
    factors."""
    p = synth.make_problem(UNEVEN, 3, dtype=np.float64, seed=3)
    r = MG.multilevel(p.Z, p.A0, p.tfms, MG.Options(coarsest=(10, 10, 10), tol=1e-10))
    assert r.converged
    assert align.factor_error(p.truth, r.A) <= 1e-9
