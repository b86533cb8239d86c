"""Failure paths on the GPU, each made on the host or through a bounded wait, never by a fault:
a NaN in the data (CPMG_NUMERIC), an exactly singular Gamma (the pseudoinverse of Section 3),
a grid barrier that cannot complete (CPMG_TIMEOUT, the context stays usable), and cancelling
served requests (CPMG_CANCELLED)."""
import time

import numpy as np
import pytest

from oracle import als as ALS
from paper_1111_6091_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(cpmg, arrs):
    return [cpmg.colmajor(a) for a in arrs]


def test_nan_in_tensor_reports_numeric(cpmg_ctx):
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((20, 18, 16), 3, congruence=0.5, eta_homo=0.01, dtype=np.float32, seed=31)
    Z = p.Z.copy()
    Z[3, 4, 5] = np.nan
    with pytest.raises(cpmg.CpmgError) as e:
        cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(Z), _dev(cpmg, p.A0), 5, precision=cpmg.PREC_MIXED,
                          check_every=1, tol=1e-12)
    assert e.value.status == cpmg.NUMERIC


def test_nan_tensor_in_a_batch_leaves_the_others_alone(cpmg_ctx):
    """One poisoned tensor in a batch gets CPMG_NUMERIC; every other tensor's factors are bitwise
    those of the same batch without it."""
    from paper_1111_6091_gb300 import cpmg
    probs = [synth.make_problem(d, 3, congruence=0.5, eta_homo=0.01, dtype=np.float32, seed=40 + k, n_t=0)
             for k, d in enumerate([(20, 18, 16), (24, 20, 18), (16, 16, 16, 16)])]
    Zs = [cpmg.colmajor(p.Z) for p in probs]
    clean = [_dev(cpmg, p.A0) for p in probs]
    _, rc = cpmg.cpmg_batch_solve(cpmg_ctx, Zs, clean, precision=cpmg.PREC_MIXED, tol=1e-8, max_als_iters=200)
    Zbad = probs[1].Z.copy()
    Zbad[0, 0, 0] = np.nan
    Zs2 = [Zs[0], cpmg.colmajor(Zbad), Zs[2]]
    mixed = [_dev(cpmg, p.A0) for p in probs]
    st, rm = cpmg.cpmg_batch_solve(cpmg_ctx, Zs2, mixed, precision=cpmg.PREC_MIXED, tol=1e-8, max_als_iters=200)
    assert st == cpmg.NUMERIC and rm[1]["status"] == cpmg.NUMERIC
    for t in (0, 2):
        assert rm[t]["status"] == rc[t]["status"] and rm[t]["iters_als"] == rc[t]["iters_als"]
        for a, b in zip(mixed[t], clean[t]):
            assert np.array_equal(cpmg.to_numpy(a), cpmg.to_numpy(b))


def test_singular_gamma_takes_the_pseudoinverse(cpmg_ctx):
    """Two identical rank-one terms make every Gamma^(n) exactly singular: the update of Section 3
    is then A = M Gamma^+ (Cholesky fails its pivot test), on the GPU as in the oracle."""
    from paper_1111_6091_gb300 import cpmg
    p = synth.make_problem((22, 19, 17), 4, congruence=0.4, eta_homo=0.02, dtype=np.float64, seed=33)
    A0 = [a.copy() for a in p.A0]
    for a in A0:
        a[:, 3] = a[:, 1]
    ref = ALS.sort_components(ALS.als_sweep(p.Z, A0))
    A = _dev(cpmg, A0)
    cpmg.cp_als_sweep(cpmg_ctx, cpmg.colmajor(p.Z), A, 1, precision=cpmg.PREC_FP64, check_every=0)
    for a, b in zip(A, ref):
        a = cpmg.to_numpy(a)
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(b))


def test_unreachable_barrier_times_out_and_the_context_recovers():
    """The batched kernel's grid barriers are bounded waits.  With the test hook, the first barrier
    of every launch waits for one CTA more than the launch has: each wait runs out after 50 ms, the
    call returns CPMG_TIMEOUT, and with the hook off the same context solves the batch again with
    the results of a clean run."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    probs = [synth.make_problem(d, 3, congruence=0.5, eta_homo=0.01, dtype=np.float32, seed=50 + k, n_t=0)
             for k, d in enumerate([(20, 18, 16), (24, 20, 18)])]
    ctx = cpmg.Context(0)
    try:
        Zs = [cpmg.colmajor(p.Z) for p in probs]
        ref = [_dev(cpmg, p.A0) for p in probs]
        cpmg.cpmg_batch_solve(ctx, Zs, ref, precision=cpmg.PREC_MIXED, tol=1e-8, max_als_iters=100)
        ctx.debug_config(0.05, True)
        A = [_dev(cpmg, p.A0) for p in probs]
        t0 = time.perf_counter()
        with pytest.raises(cpmg.CpmgError) as e:
            cpmg.cpmg_batch_solve(ctx, Zs, A, precision=cpmg.PREC_MIXED, tol=1e-8, max_als_iters=100)
        assert e.value.status == cpmg.TIMEOUT
        assert time.perf_counter() - t0 < 30.0
        ctx.debug_config(2.0, False)
        A = [_dev(cpmg, p.A0) for p in probs]
        st, _ = cpmg.cpmg_batch_solve(ctx, Zs, A, precision=cpmg.PREC_MIXED, tol=1e-8, max_als_iters=100)
        torch.cuda.synchronize()
        for X, Y in zip(A, ref):
            for a, b in zip(X, Y):
                assert np.array_equal(cpmg.to_numpy(a), cpmg.to_numpy(b))
    finally:
        ctx.close()


def test_server_cancels_queued_and_running_requests():
    import torch
    from paper_1111_6091_gb300 import cpmg
    ctx = cpmg.Context(0)
    try:
        srv = cpmg.Server(ctx, max_active=1, sweeps_per_launch=8)
        long = synth.make_problem((64, 60, 56), 8, congruence=0.9, eta_homo=0.05, dtype=np.float32, seed=61, n_t=0)
        small = synth.make_problem((20, 18, 16), 3, congruence=0.5, eta_homo=0.01, dtype=np.float32, seed=62, n_t=0)
        Zl, Zs = cpmg.colmajor(long.Z), cpmg.colmajor(small.Z)
        Al, Aq = _dev(cpmg, long.A0), _dev(cpmg, small.A0)
        torch.cuda.synchronize()
        # the first request cannot reach tol = 0 and runs up to 1e4 sweeps; the second waits behind it
        t_run = srv.submit(Zl, Al, precision=cpmg.PREC_MIXED, tol=0.0, max_als_iters=10000)
        t_q = srv.submit(Zs, Aq, precision=cpmg.PREC_MIXED, tol=1e-8, max_als_iters=1000)
        srv.cancel(t_q)
        rq = srv.poll(t_q)
        assert rq is not None and rq["status"] == cpmg.CANCELLED
        for a, a0 in zip(Aq, small.A0):
            assert np.array_equal(cpmg.to_numpy(a), a0)
        time.sleep(0.2)
        srv.cancel(t_run)
        assert srv.wait(120.0) == cpmg.OK
        rr = srv.poll(t_run)
        assert rr["status"] == cpmg.CANCELLED and 0 < rr["iters_als"] < 10000
        assert all(np.all(np.isfinite(cpmg.to_numpy(a))) for a in Al)
        # the server goes on serving
        A2 = _dev(cpmg, small.A0)
        t2 = srv.submit(Zs, A2, precision=cpmg.PREC_MIXED, tol=1e-8, max_als_iters=1000)
        assert srv.wait(120.0) == cpmg.OK
        assert srv.poll(t2)["status"] == cpmg.OK
        with pytest.raises(cpmg.CpmgError):
            srv.cancel(t2)  # polled: the ticket is released
    finally:
        ctx.close()
