"""The request server (continuous batching): results equal to the oracle's ALS and bitwise
equal alone and in a mix, admission by HBM budget, requests joining while others run, and the
latency statistics."""
import time

import numpy as np
import pytest

from oracle import tensor as T, als as ALS, align
from paper_1111_6091_gb300 import synth

pytestmark = pytest.mark.gpu


def mix(n, seed=7, hi3=64, hi4=32):
    """Requests of the batched workload: order 3 or 4, modes in [16, hi3] (4-way: [16, hi4]),
    R in 2..6, congruence in [0.3, 0.6], 1% noise, float32."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        N = int(rng.integers(3, 5))
        hi = hi3 if N == 3 else hi4
        dims = tuple(int(v) for v in rng.integers(16, hi + 1, N))
        R = int(rng.integers(2, 7))
        c = float(rng.uniform(0.3, 0.6))
        out.append(synth.make_problem(dims, R, congruence=c, eta_homo=0.01, dtype=np.float32, seed=500 + k))
    return out


def new_server(**kw):
    import torch
    from paper_1111_6091_gb300 import cpmg
    stream = torch.cuda.Stream()
    ctx = cpmg.Context(0, stream=stream.cuda_stream)
    return ctx, cpmg.Server(ctx, **kw), stream


def submit(srv, p, **kw):
    import torch
    from paper_1111_6091_gb300 import cpmg
    Z = cpmg.colmajor(p.Z)
    A = [cpmg.colmajor(a) for a in p.A0]
    torch.cuda.synchronize()  # inputs written on torch's stream before the server's stream reads them
    return srv.submit(Z, A, **kw), A


OPTS = dict(tol=1e-8, max_als_iters=4000)


def collect(srv, tickets):
    from paper_1111_6091_gb300 import cpmg
    assert srv.wait(600.0) == 0
    out = []
    for t, A in tickets:
        r = srv.poll(t)
        assert r is not None
        out.append((r, [cpmg.to_numpy(a) for a in A]))
    return out


def test_mix_matches_oracle_and_alone():
    from paper_1111_6091_gb300 import cpmg
    probs = mix(10)
    ctx, srv, stream = new_server(sweeps_per_launch=4)
    try:
        res = collect(srv, [submit(srv, p, precision=cpmg.PREC_MIXED, **OPTS) for p in probs])
        for k, (p, (r, A)) in enumerate(zip(probs, res)):
            Z64 = p.Z.astype(np.float64)
            assert r["status"] == cpmg.OK, r
            assert T.g_value(Z64, A) < 2e-8
            if k % 3 == 0:
                ref, _ = ALS.als(Z64, p.A0, 4000, tol=1e-8, g_fn=T.g_value)
                assert align.factor_error(ref, A) <= 1e-6
        # the same requests one at a time: bitwise the same factors and sweep counts
        for k in (0, 4, 9):
            (r1, A1), = collect(srv, [submit(srv, probs[k], precision=cpmg.PREC_MIXED, **OPTS)])
            assert r1["iters_als"] == res[k][0]["iters_als"]
            for a, b in zip(A1, res[k][1]):
                assert np.array_equal(a, b)
        st = srv.stats()
        assert st["completed"] == 13 and 0 < st["p50_s"] <= st["p99_s"] and st["req_per_s"] > 0
    finally:
        ctx.close()


def test_requests_join_while_others_run():
    """A second wave submitted while the first is on the GPU is admitted into the running batch;
    every result equals the one from a server that saw all requests at once."""
    from paper_1111_6091_gb300 import cpmg
    probs = mix(8, seed=11)
    ctx, srv, stream = new_server(sweeps_per_launch=2)
    try:
        first = [submit(srv, p, precision=cpmg.PREC_MIXED, **OPTS) for p in probs[:4]]
        time.sleep(0.02)
        second = [submit(srv, p, precision=cpmg.PREC_MIXED, **OPTS) for p in probs[4:]]
        staggered = collect(srv, first + second)
        together = collect(srv, [submit(srv, p, precision=cpmg.PREC_MIXED, **OPTS) for p in probs])
        for (r1, A1), (r2, A2) in zip(staggered, together):
            assert r1["status"] == r2["status"] == cpmg.OK
            assert r1["iters_als"] == r2["iters_als"]
            for a, b in zip(A1, A2):
                assert np.array_equal(a, b)
    finally:
        ctx.close()


def test_budget_admission():
    """A request larger than the budget is refused; under a budget that fits about two requests
    at a time every request still completes with the same result as unbounded."""
    from paper_1111_6091_gb300 import cpmg
    probs = mix(6, seed=3, hi3=32, hi4=16)
    big = synth.make_problem((64, 64, 64), 4, congruence=0.3, eta_homo=0.01, dtype=np.float32, seed=9)
    ctx, srv, stream = new_server(sweeps_per_launch=4, budget_bytes=400_000, unit_elements=8192)
    try:
        with pytest.raises(cpmg.CpmgError) as e:
            submit(srv, big, precision=cpmg.PREC_MIXED, **OPTS)
        assert e.value.status == cpmg.OUT_OF_BUDGET
        tight = collect(srv, [submit(srv, p, precision=cpmg.PREC_MIXED, **OPTS) for p in probs])
    finally:
        ctx.close()
    ctx, srv, stream = new_server(sweeps_per_launch=4, unit_elements=8192)
    try:
        free = collect(srv, [submit(srv, p, precision=cpmg.PREC_MIXED, **OPTS) for p in probs])
    finally:
        ctx.close()
    for (r1, A1), (r2, A2) in zip(tight, free):
        assert r1["status"] == r2["status"] == cpmg.OK
        assert r1["iters_als"] == r2["iters_als"]
        for a, b in zip(A1, A2):
            assert np.array_equal(a, b)


def test_multilevel_requests_match_decompose_alone_and_in_the_mix(cpmg_ctx):
    """A multilevel request (the Section 6.1 driver, hierarchy resident while it runs) gives the
    factors of a direct cpmg_decompose call bitwise, whether it is served alone or beside batched
    ALS requests and another multilevel request."""
    import torch
    from paper_1111_6091_gb300 import cpmg, synth
    p = synth.make_problem((32, 30, 28), 3, congruence=0.5, eta_homo=0.001, dtype=np.float32, seed=4)
    kw = dict(precision=cpmg.PREC_MIXED, tol=1e-9, coarsest=(8, 8, 8), als_fallback=1)
    Z = cpmg.colmajor(p.Z)
    A_ref = [cpmg.colmajor(a) for a in p.A0]
    r_ref = cpmg.cpmg_decompose(cpmg_ctx, Z, A_ref, [[cpmg.colmajor(a) for a in b] for b in p.tfms], **kw)
    assert r_ref["status"] == cpmg.OK
    others = [synth.make_problem(d, 3, congruence=0.6, eta_homo=0.01, dtype=np.float32, seed=70 + k, n_t=2)
              for k, d in enumerate([(24, 20, 18), (40, 36, 30), (30, 30, 30)])]
    for mix in (False, True):
        ctx = cpmg.Context(0)
        try:
            srv = cpmg.Server(ctx)
            A = [cpmg.colmajor(a) for a in p.A0]
            TF = [[cpmg.colmajor(a) for a in b] for b in p.tfms]
            keep = []
            if mix:
                for q in others[:2]:
                    Aq = [cpmg.colmajor(a) for a in q.A0]
                    keep.append((srv.submit(cpmg.colmajor(q.Z), Aq, precision=cpmg.PREC_MIXED, tol=1e-8,
                                            max_als_iters=2000), Aq))
            t = srv.submit_multilevel(Z, A, TF, **kw)
            if mix:
                q = others[2]
                Aq = [cpmg.colmajor(a) for a in q.A0]
                keep.append((srv.submit_multilevel(cpmg.colmajor(q.Z), Aq, [[cpmg.colmajor(a) for a in b]
                                                                              for b in q.tfms], **kw), Aq))
            assert srv.wait(300.0) == cpmg.OK
            r = srv.poll(t)
            assert r["status"] == cpmg.OK and r["iters_setup"] == r_ref["iters_setup"]
            for tk, _ in keep:
                assert srv.poll(tk)["status"] in (cpmg.OK, cpmg.NOT_CONVERGED)
            torch.cuda.synchronize()
            for a, b in zip(A, A_ref):
                assert np.array_equal(cpmg.to_numpy(a), cpmg.to_numpy(b)), mix
        finally:
            ctx.close()
