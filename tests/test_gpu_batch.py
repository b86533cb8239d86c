"""Batched CP-ALS (cpmg_batch_solve) against the FP64 oracle's ALS, tensor by tensor, and the
independence of each tensor's result from the rest of the batch."""
import numpy as np
import pytest

from oracle import tensor as T, als as ALS, align
from paper_1111_6091_gb300 import synth

pytestmark = pytest.mark.gpu


def problems(specs, dtype=np.float32):
    out = []
    for k, (dims, R, c) in enumerate(specs):
        out.append(synth.make_problem(dims, R, congruence=c, eta_homo=0.01, dtype=dtype, seed=40 + k))
    return out


SPECS = [((20, 17, 33), 3, 0.5), ((16, 40, 24, 18), 2, 0.7), ((70, 65, 16), 8, 0.6),
         ((33, 30), 4, 0.5), ((130, 20, 18), 5, 0.8), ((18, 16, 17, 20), 6, 0.6)]


def run_batch(ctx, probs, **kw):
    from paper_1111_6091_gb300 import cpmg
    Zs = [cpmg.colmajor(p.Z) for p in probs]
    As = [[cpmg.colmajor(a) for a in p.A0] for p in probs]
    st, res = cpmg.cpmg_batch_solve(ctx, Zs, As, **kw)
    return st, res, [[cpmg.to_numpy(a) for a in A] for A in As]


def test_fixed_sweeps_match_oracle_fp64(cpmg_ctx):
    """30 FP64 sweeps of every tensor (tol 0, so the cap stops them) equal the oracle's 30 ALS
    iterations (normalize after each, sort at the end) to 1e-9 relative."""
    from paper_1111_6091_gb300 import cpmg
    probs = problems(SPECS)
    st, res, got = run_batch(cpmg_ctx, probs, precision=cpmg.PREC_FP64, tol=0.0, max_als_iters=30,
                             check_every=1)
    for p, r, A in zip(probs, res, got):
        ref, it = ALS.als(p.Z.astype(np.float64), p.A0, 30)
        assert r["iters_als"] == 30 and r["status"] == cpmg.NOT_CONVERGED
        for a, b in zip(A, ref):
            assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(b))
        assert np.isclose(r["f"], T.f_value(p.Z.astype(np.float64), ref), rtol=1e-9)
        assert np.isclose(r["g"], T.g_value(p.Z.astype(np.float64), ref), rtol=1e-6)


@pytest.mark.parametrize("prec", ["FP32", "DF"])
def test_fixed_sweeps_float_paths(cpmg_ctx, prec):
    """Ten sweeps in FP32 (float products and sums) and float-pair arithmetic: factors within the
    accuracy of the arithmetic of the oracle's."""
    from paper_1111_6091_gb300 import cpmg
    probs = problems(SPECS)
    tol = {"FP32": 2e-4, "DF": 1e-9}[prec]
    st, res, got = run_batch(cpmg_ctx, probs, precision=getattr(cpmg, "PREC_" + prec), tol=0.0, max_als_iters=10,
                             check_every=1)
    for p, A in zip(probs, got):
        ref, _ = ALS.als(p.Z.astype(np.float64), p.A0, 10)
        for a, b in zip(A, ref):
            assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b)), prec


def test_converges_to_tolerance_mixed(cpmg_ctx):
    """MIXED precision to g < 1e-8 on exact low-rank tensors plus noise: every tensor stops with
    g < tol (verified by the oracle's g) and matches the oracle's ALS solution from the same
    start to 1e-6 after alignment."""
    from paper_1111_6091_gb300 import cpmg
    specs = [((24, 20, 18), 3, 0.3), ((16, 18, 20, 17), 2, 0.3), ((40, 30, 20), 4, 0.3)]
    probs = problems(specs)
    st, res, got = run_batch(cpmg_ctx, probs, precision=cpmg.PREC_MIXED, tol=1e-8, max_als_iters=5000,
                             check_every=1)
    assert st == cpmg.OK
    for p, r, A in zip(probs, res, got):
        Z64 = p.Z.astype(np.float64)
        assert r["status"] == cpmg.OK
        assert T.g_value(Z64, A) < 2e-8
        ref, _ = ALS.als(Z64, p.A0, 5000, tol=1e-8, g_fn=T.g_value)
        assert align.factor_error(ref, A) <= 1e-6


def test_result_independent_of_batch(cpmg_ctx):
    """Each tensor's factors are bitwise the same solved alone and inside a larger batch."""
    from paper_1111_6091_gb300 import cpmg
    probs = problems(SPECS)
    kw = dict(precision=cpmg.PREC_MIXED, tol=1e-6, max_als_iters=300, check_every=4)
    _, res_all, got_all = run_batch(cpmg_ctx, probs, **kw)
    for k in (0, 3, 5):
        _, res1, got1 = run_batch(cpmg_ctx, [probs[k]], **kw)
        assert res1[0]["iters_als"] == res_all[k]["iters_als"]
        for a, b in zip(got1[0], got_all[k]):
            assert np.array_equal(a, b)


def test_batch_matches_per_tensor_loop(cpmg_ctx):
    """The batched FP64 solve and a loop of cp_als_sweep calls (the per-tensor launch path)
    reach the same factors."""
    from paper_1111_6091_gb300 import cpmg
    probs = problems(SPECS[:3])
    _, res, got = run_batch(cpmg_ctx, probs, precision=cpmg.PREC_FP64, tol=0.0, max_als_iters=20,
                            check_every=1)
    for p, A in zip(probs, got):
        B = [cpmg.colmajor(a) for a in p.A0]
        cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(p.Z), B, 20, precision=cpmg.PREC_FP64, check_every=0)
        for a, b in zip(A, [cpmg.to_numpy(x) for x in B]):
            assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_batch_invalid_arguments(cpmg_ctx):
    import torch
    from paper_1111_6091_gb300 import cpmg
    Z = torch.zeros((4, 5, 6), dtype=torch.float32, device="cuda")
    A9 = [torch.zeros((9, I), dtype=torch.float64, device="cuda") for I in (6, 5, 4)]
    with pytest.raises(cpmg.CpmgError) as e:
        cpmg.cpmg_batch_solve(cpmg_ctx, [Z], [A9])
    assert e.value.status == cpmg.INVALID_ARG
