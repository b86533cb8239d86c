"""GPU parity of the solver calls (cp_als_sweep, mg_setup, mg_fas_solve, cpmg_decompose)
against the FP64 oracle, from identical starts."""
import numpy as np
import pytest

from oracle import tensor as T, als as ALS, multigrid as MG, align
from paper_1111_6091_gb300 import synth

pytestmark = pytest.mark.gpu


def dev(cpmg, arrs):
    return [cpmg.colmajor(a) for a in arrs]


def host(cpmg, ts):
    return [cpmg.to_numpy(t) for t in ts]


def assert_same_stationary_point(Z, got, ref, tol):
    """Both sides stopped at g < tol: relative f within 1e-9, and the factors within
    max(1e-10, 3 (g_gpu + g_oracle)) after alignment -- two iterates near one stationary point lie
    within kappa (g_1 + g_2) of each other, kappa = |A - A*| / g of a few units on these problems."""
    g1, g2 = T.g_value(Z, got), T.g_value(Z, ref)
    assert g1 < tol and g2 < tol
    f1, f2 = T.f_value(Z, got), T.f_value(Z, ref)
    # relative 1e-9; for exact data f itself is ~(g ||Z||)^2, so also 1e-18 of ||Z||^2 absolute
    assert abs(f1 - f2) <= 1e-9 * f2 + 1e-18 * np.sum(np.asarray(Z, dtype=np.float64) ** 2)
    assert align.factor_error(ref, got) <= max(1e-10, 3.0 * (g1 + g2))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_one_als_sweep_matches_oracle(cpmg_ctx, dt):
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((24, 20, 18), 4, congruence=0.5, eta_homo=0.01, dtype=dt, seed=1)
    Z64 = p.Z.astype(np.float64)
    ref = ALS.sort_components(ALS.als_sweep(Z64, p.A0))
    for prec, tol in ((cpmg.PREC_FP64, 1e-10), (cpmg.PREC_DF, 1e-9), (cpmg.PREC_FP32, 2e-4)):
        if prec == cpmg.PREC_DF and dt == np.float64:
            continue
        A = dev(cpmg, p.A0)
        cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(p.Z), A, 1, precision=prec, check_every=0)
        for a, b in zip(host(cpmg, A), ref):
            assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b)), prec


def test_als_exact_recovery_20cubed(cpmg_ctx):
    """Exact rank-3 20^3 tensor (float64): f -> 0 and factor error <= 1e-10 against the truth,
    and the same iterate count as the oracle (+-1)."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((20, 20, 20), 3, dtype=np.float64, seed=0)
    for prec in (cpmg.PREC_FP64, cpmg.PREC_MIXED):
        A = dev(cpmg, p.A0)
        r = cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(p.Z), A, 10000, precision=prec, tol=1e-10, check_every=1)
        got = host(cpmg, A)
        assert r["status"] == cpmg.OK
        assert T.g_value(p.Z, got) < 1e-10
        assert align.factor_error(p.truth, got) <= 1e-10
        assert r["f"] <= 1e-16 * np.sum(p.Z ** 2)
    _, it = ALS.als(p.Z, p.A0, 10000, tol=1e-10, g_fn=T.g_value)
    A = dev(cpmg, p.A0)
    r = cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(p.Z), A, 10000, precision=cpmg.PREC_FP64, tol=1e-10, check_every=1)
    assert abs(r["iters_als"] - it) <= 1


def test_als_f_monotone(cpmg_ctx):
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((30, 25, 20), 4, congruence=0.8, eta_homo=0.05, dtype=np.float32, seed=2)
    A = dev(cpmg, p.A0)
    fprev = np.inf
    for _ in range(20):
        r = cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(p.Z), A, 1, precision=cpmg.PREC_DF, check_every=0)
        assert r["f"] <= fprev * (1 + 1e-10)
        fprev = r["f"]


def test_setup_cycle_matches_oracle(cpmg_ctx):
    """One CP-AMG-mult cycle (float64 arithmetic): the boot factors, the updated TFMs and the
    level-0 operators R-hat agree with the oracle's."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((20, 20, 20), 3, dtype=np.float64, seed=0)
    o = MG.Options(coarsest=(10, 10, 10), max_setup_cycles=1)
    ref = MG.mg_setup(p.Z, p.A0, p.tfms, o)
    A = dev(cpmg, p.A0)
    tf = [dev(cpmg, b) for b in p.tfms]
    h, r = cpmg.mg_setup(cpmg_ctx, cpmg.colmajor(p.Z), A, tf, precision=cpmg.PREC_FP64, max_setup_cycles=1,
                         coarsest=(10, 10, 10))
    assert r["levels"] == len(ref.levels) == 2
    for a, b in zip(host(cpmg, A), ref.A):
        assert np.max(np.abs(a - b)) <= 1e-8 * np.max(np.abs(b))
    for blk_g, blk_r in zip(tf, ref.tfms):
        for a, b in zip(host(cpmg, blk_g), blk_r):
            assert np.max(np.abs(a - b)) <= 1e-8 * np.max(np.abs(b))
    Rh = h.rhat(0, 3)
    for n in range(3):
        assert np.allclose(Rh[n], ref.levels[0].Rhat[n], rtol=1e-8, atol=1e-10)
    Y, shape, co = h.level_tensor(1, 3, __import__("torch").float64)
    assert shape == (10, 10, 10)
    assert np.allclose(cpmg.to_numpy(Y), ref.levels[1].Z, rtol=1e-8, atol=1e-8 * np.max(np.abs(ref.levels[1].Z)))
    h.free()


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_two_level_multilevel_20cubed(cpmg_ctx, prec):
    """The float64 20^3 rank-3 configuration: two-level multilevel solve to g < 1e-10, factor
    error <= 1e-10 against the exact factors, same cycle counts as the oracle."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((20, 20, 20), 3, dtype=np.float64, seed=0)
    ref = MG.multilevel(p.Z, p.A0, p.tfms, MG.Options(coarsest=(10, 10, 10), tol=1e-10))
    A = dev(cpmg, p.A0)
    tf = [dev(cpmg, b) for b in p.tfms]
    r = cpmg.cpmg_decompose(cpmg_ctx, cpmg.colmajor(p.Z), A, tf, precision=getattr(cpmg, "PREC_" + prec),
                            tol=1e-10, coarsest=(10, 10, 10))
    got = host(cpmg, A)
    assert r["status"] == cpmg.OK and r["levels"] == 2
    assert T.g_value(p.Z, got) < 1e-10
    assert align.factor_error(p.truth, got) <= 1e-10
    assert align.factor_error(ref.A, got) <= 1e-10
    if prec == "FP64":
        assert r["iters_setup"] == ref.setup_cycles and r["iters_solve"] == ref.solve_cycles


def test_fas_solve_from_setup_matches_oracle(cpmg_ctx):
    """mg_setup then mg_fas_solve as two calls on a 3-level float64 problem (coarsest 8)."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((32, 30, 28), 3, congruence=0.5, eta_homo=0.001, dtype=np.float64, seed=4)
    o = MG.Options(coarsest=(8, 8, 8), tol=1e-10)
    ref = MG.multilevel(p.Z, p.A0, p.tfms, o)
    A = dev(cpmg, p.A0)
    tf = [dev(cpmg, b) for b in p.tfms]
    h, r1 = cpmg.mg_setup(cpmg_ctx, cpmg.colmajor(p.Z), A, tf, precision=cpmg.PREC_FP64, tol=1e-10,
                          coarsest=(8, 8, 8))
    r2 = cpmg.mg_fas_solve(cpmg_ctx, h, cpmg.colmajor(p.Z), A, precision=cpmg.PREC_FP64, tol=1e-10,
                           coarsest=(8, 8, 8))
    h.free()
    got = host(cpmg, A)
    assert r1["levels"] == len(ref.levels)
    assert r2["g"] < 1e-10 and ref.converged
    assert_same_stationary_point(p.Z, got, ref.A, 1e-10)


def test_invalid_arguments(cpmg_ctx):
    import torch
    from paper_1111_6091_gb300 import cpmg
    Z = torch.zeros((4, 5, 6), dtype=torch.float32, device="cuda")
    A = [torch.zeros((2, I), dtype=torch.float64, device="cuda") for I in (6, 5, 4)]
    with pytest.raises(cpmg.CpmgError) as e:
        cpmg.cp_als_sweep(cpmg_ctx, Z, A, 1, precision=7)
    assert e.value.status == cpmg.INVALID_ARG
    A17 = [torch.zeros((17, I), dtype=torch.float64, device="cuda") for I in (6, 5, 4)]
    with pytest.raises(cpmg.CpmgError):
        cpmg.cp_als_sweep(cpmg_ctx, Z, A17, 1)
    Z1 = torch.zeros((4,), dtype=torch.float32, device="cuda")
    with pytest.raises(cpmg.CpmgError):
        cpmg.cp_als_sweep(cpmg_ctx, Z1, [torch.zeros((2, 4), dtype=torch.float64, device="cuda")], 1)


def test_host_buffers_roundtrip(cpmg_ctx):
    """cpmg_decompose with host (pinned) buffers equals the device-buffer call bitwise."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((20, 20, 20), 3, dtype=np.float64, seed=0)
    kw = dict(precision=cpmg.PREC_FP64, tol=1e-10, coarsest=(10, 10, 10))
    A = dev(cpmg, p.A0)
    cpmg.cpmg_decompose(cpmg_ctx, cpmg.colmajor(p.Z), A, [dev(cpmg, b) for b in p.tfms], **kw)
    Ah = [cpmg.colmajor(a, device="cpu", pin=True) for a in p.A0]
    tfh = [[cpmg.colmajor(a, device="cpu", pin=True) for a in b] for b in p.tfms]
    cpmg.cpmg_decompose(cpmg_ctx, cpmg.colmajor(p.Z, device="cpu", pin=True), Ah, tfh, **kw)
    for a, b in zip(host(cpmg, A), host(cpmg, Ah)):
        assert np.array_equal(a, b)


def test_graph_replay_matches_eager(cpmg_ctx):
    """The same solve with CUDA-graph replay (context on a dedicated stream) and without graphs
    gives bitwise identical factors: the graphs only change how launches are issued."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((32, 30, 28), 3, congruence=0.5, eta_homo=0.001, dtype=np.float32, seed=4)
    outs = []
    for graphs in (0, 1):
        stream = torch.cuda.Stream()
        ctx = cpmg.Context(0, stream=stream.cuda_stream)
        with torch.cuda.stream(stream):
            A = dev(cpmg, p.A0)
            tf = [dev(cpmg, b) for b in p.tfms]
            r = cpmg.cpmg_decompose(ctx, cpmg.colmajor(p.Z), A, tf, precision=cpmg.PREC_MIXED, tol=1e-7,
                                    coarsest=(8, 8, 8), als_fallback=1, use_graphs=graphs)
            B = dev(cpmg, p.A0)
            cpmg.cp_als_sweep(ctx, cpmg.colmajor(p.Z), B, 40, precision=cpmg.PREC_MIXED, check_every=5,
                              use_graphs=graphs)
            stream.synchronize()
        outs.append(([cpmg.to_numpy(a) for a in A], [cpmg.to_numpy(b) for b in B], r))
        ctx.close()
    (A0, B0, r0), (A1, B1, r1) = outs
    assert r0["iters_setup"] == r1["iters_setup"] and r0["iters_solve"] == r1["iters_solve"]
    for a, b in zip(A0 + B0, A1 + B1):
        assert np.array_equal(a, b)


def test_restriction_on_tensor_cores_keeps_the_fixed_point(cpmg_ctx):
    """The coarse tensors only shape the FAS corrections (Algorithm 2), so the multilevel solve
    with the split-BF16 tensor-core restriction reaches the same factors as with the FP32
    CUDA-core restriction, and both match the oracle's solution."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((64, 40, 36), 3, congruence=0.5, eta_homo=0.001, dtype=np.float32, seed=5)
    ref = MG.multilevel(p.Z.astype(np.float64), p.A0, p.tfms, MG.Options(coarsest=(8, 8, 8), tol=1e-9))
    got = []
    for tc in (0, 1):
        A = dev(cpmg, p.A0)
        tf = [dev(cpmg, b) for b in p.tfms]
        r = cpmg.cpmg_decompose(cpmg_ctx, cpmg.colmajor(p.Z), A, tf, precision=cpmg.PREC_MIXED, tol=1e-9,
                                coarsest=(8, 8, 8), als_fallback=1, ttm_tensor_cores=tc)
        assert r["status"] == cpmg.OK and r["g"] < 1e-9
        got.append(host(cpmg, A))
    assert align.factor_error(got[0], got[1]) <= 1e-6
    if ref.converged:
        assert align.factor_error(ref.A, got[1]) <= 1e-6


def test_multilevel_fmg_on_the_papers_dense_tensor(cpmg_ctx):
    """'Multilevel + FMG' (Section 6.1) on the paper's dense tensor z_ijk = (i^2+j^2+k^2)^(-1/2)
    (Section 6.3), s = 50, R = 3, float64, as three calls: mg_setup, mg_fmg (Algorithm 3 plus the
    down-sweep rebuild), mg_fas_solve.  Each stage is compared with the oracle's from identical
    inputs (uniform [0,1] starts as in the paper), and the multilevel cycle count is far below the
    ALS iteration count (the gap of Table tab:IJK)."""
    from paper_1111_6091_gb300 import cpmg
    s, R = 50, 3
    Z = synth.ijk_tensor(s)
    rng = np.random.default_rng(0)
    A0 = [rng.uniform(size=(s, R)) for _ in range(3)]
    tfms = [[rng.uniform(size=(s, R)) for _ in range(3)] for _ in range(2)]
    Ac0 = [rng.uniform(size=(4, R)) for _ in range(3)]
    o = MG.Options(coarsest=(4, 4, 4), tol=1e-10)
    kw = dict(precision=cpmg.PREC_FP64, tol=1e-10, coarsest=(4, 4, 4))
    # oracle, stage by stage (the body of multilevel_fmg)
    su = MG.mg_setup(Z, A0, tfms, o)
    A_fmg = MG.fmg_cp_fas(su.levels, Ac0, 100, o)
    levels, tf2 = MG.down_sweep(Z, A_fmg, su.tfms, o)
    ref = MG.mg_fas_solve(Z, levels, A_fmg, tf2, o, cycles_done=su.setup_cycles + 1)
    assert ref.converged and len(levels) == 5
    # GPU
    Zd = cpmg.colmajor(Z)
    A = dev(cpmg, A0)
    tf = [dev(cpmg, b) for b in tfms]
    h, r1 = cpmg.mg_setup(cpmg_ctx, Zd, A, tf, **kw)
    try:
        assert r1["levels"] == 5 and r1["iters_setup"] == su.setup_cycles
        dims, _ = h.level_info(4)
        assert tuple(int(dims[n]) for n in range(3)) == (4, 4, 4)
        rf = cpmg.mg_fmg(cpmg_ctx, h, Zd, dev(cpmg, Ac0), A, nu=100, **kw)
        got_fmg = host(cpmg, A)
        for a, b in zip(got_fmg, A_fmg):
            assert np.max(np.abs(a - b)) <= 1e-8 * np.max(np.abs(b))
        assert np.isclose(rf["g"], T.g_value(Z, A_fmg), rtol=1e-6)
        r2 = cpmg.mg_fas_solve(cpmg_ctx, h, Zd, A, **kw)
    finally:
        h.free()
    got = host(cpmg, A)
    assert r2["status"] == cpmg.OK and T.g_value(Z, got) < 1e-10
    assert r2["iters_solve"] == ref.solve_cycles
    assert_same_stationary_point(Z, got, ref.A, 1e-10)
    _, it_als = ALS.als(Z, A0, 10000, tol=1e-10, g_fn=T.g_value)
    assert (r1["iters_setup"] + 1 + r2["iters_solve"]) * 20 < it_als


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_dimension_tree_sweeps_match_oracle(cpmg_ctx, dt):
    """Third-order tensor with I_3 > 6R, so the sweeps take modes 1 and 2 from W = Z x_3 A^(3)^T:
    three ALS sweeps with and without the dimension tree both match the oracle's ALS, and f and g
    of the result (Eq. CPfunctional, Eq. gradConv) match the oracle's."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((36, 28, 44), 4, congruence=0.6, eta_homo=0.01, dtype=dt, seed=6)
    Z64 = p.Z.astype(np.float64)
    ref = p.A0
    for _ in range(3):
        ref = ALS.als_sweep(Z64, ref)
    ref = ALS.sort_components(ref)
    precs = ((cpmg.PREC_FP64, 1e-10),) + (((cpmg.PREC_DF, 1e-9), (cpmg.PREC_FP32, 2e-4)) if dt == np.float32 else ())
    for prec, tol in precs:
        for tree in (0, 1):
            A = dev(cpmg, p.A0)
            r = cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(p.Z), A, 3, precision=prec, check_every=0,
                                  dimension_tree=tree)
            got = host(cpmg, A)
            for a, b in zip(got, ref):
                assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b)), (prec, tree)
            f_got, f_ref = T.f_value(Z64, got), T.f_value(Z64, ref)
            assert abs(r["f"] - f_got) <= 1e-9 * f_got
            assert abs(r["g"] - T.g_value(Z64, got)) <= 1e-6 * T.g_value(Z64, got)
            if prec != cpmg.PREC_FP32:
                assert abs(f_got - f_ref) <= 1e-9 * f_ref


@pytest.mark.parametrize("eta", [0.0, 0.05])
def test_uneven_hierarchy_matches_oracle(cpmg_ctx, eta):
    """40 x 12 x 40, rank 3, coarsest 10: mode 2 stops coarsening at level 1 (Section 4.5), so the
    FAS right-hand side of that mode takes the branch with R-hat = I (Eq. FASrhs) on the GPU as in
    the oracle.  Exact data (eta = 0) and 5% noise, float64, to g < 1e-10."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((40, 12, 40), 3, eta_homo=eta, dtype=np.float64, seed=3)
    o = MG.Options(coarsest=(10, 10, 10), tol=1e-10)
    ref = MG.multilevel(p.Z, p.A0, p.tfms, o)
    assert ref.converged and [L.Ic for L in ref.levels][1] == [True, False, True]
    A = dev(cpmg, p.A0)
    tf = [dev(cpmg, b) for b in p.tfms]
    r = cpmg.cpmg_decompose(cpmg_ctx, cpmg.colmajor(p.Z), A, tf, precision=cpmg.PREC_FP64, tol=1e-10,
                            coarsest=(10, 10, 10))
    assert r["status"] == cpmg.OK and r["levels"] == 3
    assert r["iters_setup"] == ref.setup_cycles
    assert_same_stationary_point(p.Z, host(cpmg, A), ref.A, 1e-10)


def test_split_bf16_sweeps_match_oracle(cpmg_ctx):
    """CPMG_PREC_BF16X3: both passes over Z of each sweep are tcgen05 mode products in split BF16
    (x = hi + lo, products hi*hi + hi*lo + lo*hi in FP32), about 2^-17 relative per product, the
    FP32 class of accuracy.  Three sweeps stay within the FP32 test's bound of the oracle's ALS, and
    MIXED_BF16 (split-BF16 sweeps, then float-pair ones) reaches g < 1e-10."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((36, 28, 44), 4, congruence=0.6, eta_homo=0.01, dtype=np.float32, seed=6)
    Z64 = p.Z.astype(np.float64)
    ref = p.A0
    for _ in range(3):
        ref = ALS.als_sweep(Z64, ref)
    ref = ALS.sort_components(ref)
    A = dev(cpmg, p.A0)
    cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(p.Z), A, 3, precision=cpmg.PREC_BF16X3, check_every=0)
    for a, b in zip(host(cpmg, A), ref):
        assert np.max(np.abs(a - b)) <= 5e-4 * np.max(np.abs(b))
    A = dev(cpmg, p.A0)
    r = cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(p.Z), A, 5000, precision=cpmg.PREC_MIXED_BF16, tol=1e-10,
                          check_every=1)
    assert r["status"] == cpmg.OK and T.g_value(Z64, host(cpmg, A)) < 1e-10
    ref_c, _ = ALS.als(Z64, p.A0, 5000, tol=1e-10, g_fn=T.g_value)
    assert_same_stationary_point(Z64, host(cpmg, A), ref_c, 1e-10)


@pytest.mark.parametrize("dims,R", [((400, 400, 64), 10), ((200, 300, 37), 7)])
def test_dimension_tree_w_pass_large_fp32(cpmg_ctx, dims, R):
    """Tensors with enough rows for the FP32 W pass's streamed ring: at least 256 rows per SM, each
    CTA's rows read column by column through bulk copies. The second shape leaves a short last block
    of rows (60 000 rows in blocks of 396) and a short last stage of columns (37 = 4 x 8 + 5). One
    FP32 sweep with the tree matches the sweep without it, and the oracle's ALS."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem(dims, R, congruence=0.5, eta_homo=0.01, dtype=np.float32, seed=8, n_t=0)
    Z64 = p.Z.astype(np.float64)
    ref = ALS.sort_components(ALS.als_sweep(Z64, p.A0))
    out = []
    for tree in (1, 0):
        A = dev(cpmg, p.A0)
        cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(p.Z), A, 1, precision=cpmg.PREC_FP32, check_every=0,
                          dimension_tree=tree)
        out.append(host(cpmg, A))
        for a, b in zip(out[-1], ref):
            assert np.max(np.abs(a - b)) <= 2e-4 * np.max(np.abs(b)), tree
    for a, b in zip(*out):
        assert np.max(np.abs(a - b)) <= 2e-4 * np.max(np.abs(b))
