#!/usr/bin/env python3
"""Benchmark: time-to-tolerance of the batched CP-ALS form on one GPU.

Workload (one step): 512 independent dense tensors (order 3 or 4 with probability 1/2, mode sizes
uniform in [16, 128] ([16, 48] for order 4), rank uniform in 2..8, factor columns with pairwise
congruence uniform in [0.5, 0.95], 1% noise; seeded synthetic float32 data) decomposed by CP-ALS
(Section 3) from fixed N(0,1) starts until every tensor's g of Eq. gradConv is below 1e-8, or it
has run the 1e4 ALS iterations of Section 6.1, all in one cooperative persistent kernel per check
interval, MIXED precision (FP32 sweeps, float64-accurate sweeps near the FP32 floor; float64 Grams,
solves and g).  `value` is the seconds one step takes with the tensors resident in HBM (1.3 GB,
larger than the 126 MB L2); the batched kernel's launches are timed with CUDA events inside the
timed steps (roofline).  `e2e` repeats the step through the same C ABI call with pinned host
buffers, the copies inside the call.  The same batch in plain FP64 on the GPU, and as a loop of
per-tensor calls, is reported beside it.

Further measurements on the same line: the 100^3 rank-5 multilevel solve (Section 6.1 driver), the
400^3 rank-10 sweep and its MTTKRP against the measured HBM peak, the tensor-core restriction, the
served request stream and the paper's dense test tensor.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-tol (rel err 1e-8)"
BATCH_COUNT, BATCH_TOL, BATCH_MAX_IT, BATCH_CHECK = 512, 1e-8, 10000, 8
WORKLOAD = ("batched CP-ALS: 512 dense tensors, order 3/4, sizes U[16,128] (U[16,48] for order 4), "
            "R U{2..8}, congruence U[0.5,0.95], 1% noise, fp32, g<1e-8, at most 1e4 sweeps")

# the 100^3 rank-5 multilevel workload (congruence 0.9, 1% + 5% noise, levels 100/50/25/13)
DIMS, RANK, CONG, ETA1, ETA2, SEED = (100, 100, 100), 5, 0.9, 0.01, 0.05, 0
COARSEST = (13, 13, 13)
TOL = 1e-8


def problem():
    from paper_1111_6091_gb300 import synth
    return synth.make_problem(DIMS, RANK, congruence=CONG, eta_homo=ETA1, eta_hetero=ETA2,
                              dtype=np.float32, seed=SEED)


def config(extra=None):
    c = {"workload": WORKLOAD, "count": BATCH_COUNT, "order": [3, 4], "dims": "U[16,128] (order 4: U[16,48])",
         "rank": "U{2..8}", "congruence": "U[0.5,0.95]", "noise": 0.01, "tol": BATCH_TOL,
         "max_sweeps": BATCH_MAX_IT, "check_every": BATCH_CHECK,
         "solver": "CP-ALS (Section 3), one cooperative persistent kernel per check interval",
         "precision": "mixed fp32 / float-pair sweeps, float64 Grams, solves and g",
         "l2": "inputs larger than L2 (1.3 GB resident)"}
    if extra:
        c.update(extra)
    return c


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle (CPU)
def oracle_solve(p):
    """The FP64 oracle's multilevel solve (Section 6.1 driver) of the 100^3 workload."""
    from oracle import multigrid as MG
    o = MG.Options(coarsest=COARSEST, tol=TOL, als_fallback=True)
    t = time.perf_counter()
    r = MG.multilevel(p.Z.astype(np.float64), p.A0, p.tfms, o)
    return time.perf_counter() - t, r


def oracle_batch_tensor(p):
    """The FP64 oracle's ALS on one tensor of the batch, from the same start as the GPU, to g < 1e-8
    checked every 8 iterations (as the batched kernel checks), at most 1e4 iterations.  Returns
    (seconds, factors, iterations, g)."""
    from oracle import als as ALS, tensor as T
    Z64 = p.Z.astype(np.float64)
    t = time.perf_counter()
    A, it, g = p.A0, 0, T.g_value(Z64, p.A0)
    while it < BATCH_MAX_IT and g >= BATCH_TOL:
        A, _ = ALS.als(Z64, A, BATCH_CHECK, sort_at_end=False)
        it += BATCH_CHECK
        g = T.g_value(Z64, A)
    A = ALS.sort_components(A)
    return time.perf_counter() - t, A, it, g


def oracle_sweep_cost(probs, count=16, sweeps=4):
    """Seconds per (mode x element) of one oracle ALS iteration, measured on the first `count`
    tensors of the batch (`sweeps` iterations each): the oracle's cost of a sweep is N MTTKRPs,
    each a pass over the tensor."""
    from oracle import als as ALS
    t = time.perf_counter()
    work = 0
    for p in probs[:count]:
        Z64 = p.Z.astype(np.float64)
        A = p.A0
        for _ in range(sweeps):
            A = ALS.als_sweep(Z64, A)
        work += sweeps * p.Z.ndim * p.Z.size
    return (time.perf_counter() - t) / work


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        return max(n) if n else 1
    except Exception:
        return os.cpu_count() or 1


REF_SAMPLE = 4     # tensors the oracle solves per reference step
REF_POOL = 64      # the reference steps cycle through the first 64 tensors of the batch


def run_reference(args):
    """The oracle arm: each step, the FP64 NumPy oracle solves REF_SAMPLE tensors of the batch to
    tolerance (the same problems and starts as the GPU); the step's value is their total time
    scaled to the 512 tensors of the workload."""
    _, rank, _ = rank_env()
    if rank != 0:
        return
    probs = batch_problems(REF_POOL)

    def one(step):
        idx = [(REF_SAMPLE * step + j) % REF_POOL for j in range(REF_SAMPLE)]
        return sum(oracle_batch_tensor(probs[i])[0] for i in idx) * BATCH_COUNT / REF_SAMPLE

    for w in range(min(args.warmup, 1)):
        one(REF_POOL // REF_SAMPLE - 1 - w)
    vals = [one(s) for s in range(args.steps)]
    v = statistics.mean(vals)
    sample = (f"per step, the FP64 NumPy oracle's ALS solves {REF_SAMPLE} tensors of the batch (cycling through "
              f"the first {REF_POOL}) to g<1e-8; value = their time x {BATCH_COUNT}/{REF_SAMPLE}")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * v,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config(),
        "cpu_baseline": {"value": v, "unit": "s", "cores": blas_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "step_values": vals,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU
class Clocks:
    def __init__(self):
        self.f = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def rank_env():
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def ranks_barrier():
    """Barrier over the process group, if one is running (the timed region's edges)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x, device="cpu"):
    """The largest per-rank value over the process group: the job's step time is its slowest
    replica's.  Without a process group, x itself."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


PARITY_SAMPLE = 8     # tensors of the batch whose GPU result is compared with the oracle's
TRAFFIC_RATIO = 1.11  # DRAM bytes / algorithmic bytes of a full-batch k_batch launch (ncu capture)


def run_gpu(args):
    import torch
    from paper_1111_6091_gb300 import cpmg

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    ctx = cpmg.Context(local, stream=stream.cuda_stream)
    probs = batch_problems(BATCH_COUNT)
    with torch.cuda.stream(stream):
        Zs = [cpmg.colmajor(p.Z) for p in probs]
        A0 = [[cpmg.colmajor(a) for a in p.A0] for p in probs]
        As = [[a.clone() for a in A] for A in A0]
    torch.cuda.synchronize()

    def reset():
        with torch.cuda.stream(stream):
            for A, B in zip(As, A0):
                for a, b in zip(A, B):
                    a.copy_(b)
        torch.cuda.synchronize()

    def step(prec, Z=Zs, A=As):
        return cpmg.cpmg_batch_solve(ctx, Z, A, precision=prec, tol=BATCH_TOL, max_als_iters=BATCH_MAX_IT,
                                     check_every=BATCH_CHECK)

    def timed(prec):
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, res = step(prec)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), res

    for _ in range(args.warmup):  # the first call also tunes the unit sizes of the shape classes
        reset()
        step(cpmg.PREC_MIXED)
    torch.cuda.synchronize()
    ranks_barrier()
    clocks = Clocks()
    clocks.start()
    launches0 = ctx.launches()
    ctx.profile_reset()
    ctx.profile(True)
    ms, res = [], None
    for _ in range(args.steps):
        t, res = timed(cpmg.PREC_MIXED)
        ms.append(t)
    torch.cuda.synchronize()
    ranks_barrier()
    clk = clocks.stop()
    launches = (ctx.launches() - launches0) // max(args.steps, 1)
    prof_ms, prof_n, prof_bytes = ctx.profile_read(4)
    ctx.profile(False)
    t_step = max_over_ranks(statistics.mean(ms), device="cuda")
    A_gpu = [[cpmg.to_numpy(a) for a in As[i]] for i in range(PARITY_SAMPLE)]
    res_mixed = res
    zbytes = sum(p.Z.nbytes for p in probs)

    def summary(r, seconds):
        it = [x["iters_als"] for x in r]
        return {"seconds": seconds, "converged": sum(x["status"] == cpmg.OK for x in r),
                "tensor_sweeps": int(sum(it)), "max_sweeps": int(max(it)), "median_sweeps": float(np.median(it)),
                "worst_g": max(x["g"] for x in r)}

    batched = {"mixed": summary(res_mixed, t_step * 1e-3)}
    if args.solve_only:
        if rank == 0:
            print(json.dumps({"solve_only": True, "ms": ms, "launches": int(launches), **batched}), flush=True)
        ctx.close()
        return

    # the plain FP64 GPU path on the same batch
    t64, res64 = timed(cpmg.PREC_FP64)
    batched["fp64"] = summary(res64, t64 * 1e-3)
    batched["mixed_vs_fp64"] = batched["fp64"]["seconds"] / batched["mixed"]["seconds"]
    # the same MIXED solves as a loop of per-tensor calls
    if args.batch_loop:
        reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv = 0
        with torch.cuda.stream(stream):
            for Z, A in zip(Zs, As):
                r = cpmg.cp_als_sweep(ctx, Z, A, BATCH_MAX_IT, precision=cpmg.PREC_MIXED, tol=BATCH_TOL,
                                      check_every=BATCH_CHECK)
                conv += r["status"] == cpmg.OK
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        batched["per_tensor_loop_mixed"] = {"seconds": dt, "converged": conv}
        batched["speedup_vs_loop"] = dt / batched["mixed"]["seconds"]

    # end to end through the C ABI with pinned host buffers (copies inside the call)
    Zh = [cpmg.colmajor(p.Z, device="cpu", pin=True) for p in probs]
    Ah = [[cpmg.colmajor(a, device="cpu", pin=True) for a in p.A0] for p in probs]
    e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        for A, p in zip(Ah, probs):
            for a, a0 in zip(A, p.A0):
                a.copy_(torch.from_numpy(np.ascontiguousarray(a0.T)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(cpmg.PREC_MIXED, Zh, Ah)
        e2e.append(time.perf_counter() - t0)
    fbytes = sum(a.numel() * 8 for A in Ah for a in A)
    del Zh, Ah

    # parity of a sample of the batch against the oracle (same problems, same starts, same stopping test)
    parity = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import align, tensor as T
        rows = []
        for i in range(PARITY_SAMPLE):
            _, Ao, ito, go = oracle_batch_tensor(probs[i])
            Z64 = probs[i].Z.astype(np.float64)
            fo, fg = T.f_value(Z64, Ao), T.f_value(Z64, A_gpu[i])
            rows.append({"tensor": i, "factor_err": align.factor_error(Ao, A_gpu[i]),
                         "rel_f": abs(fg - fo) / fo, "g_gpu": res_mixed[i]["g"], "g_oracle": go,
                         "sweeps_gpu": res_mixed[i]["iters_als"], "sweeps_oracle": ito})
        parity = {"sample": f"tensors 0..{PARITY_SAMPLE - 1}", "max_factor_err": max(r["factor_err"] for r in rows),
                  "max_rel_f": max(r["rel_f"] for r in rows), "tensors": rows}
        # the oracle's cost of the whole workload: its measured seconds per (mode x element) of an ALS
        # iteration, times the MTTKRP passes each tensor needs to tolerance (the GPU's sweep counts,
        # plus the g evaluations every check interval)
        rate = oracle_sweep_cost(probs)
        work = sum((r["iters_als"] + r["iters_als"] / BATCH_CHECK) * p.Z.ndim * p.Z.size
                   for r, p in zip(res_mixed, probs))
        cpu = {"value": rate * work, "unit": "s", "cores": blas_threads(), "kind": "oracle",
               "sample": "FP64 NumPy ALS, 4 iterations of each of the first 16 tensors timed; value = that "
                         "cost per (mode x element) x the MTTKRP passes of the whole batch to tolerance"}

    # roofline of the batched kernel over the timed steps (CUDA events around every launch)
    hbm, how = peaks()
    avg_s = prof_ms * 1e-3 / max(prof_n, 1)
    achieved = prof_bytes / avg_s / 1e9 if prof_n else None
    roofline = {"bound": "hbm", "kernel": "k_batch (cooperative persistent batched CP-ALS)",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm if achieved else None,
                "traffic": TRAFFIC_RATIO * prof_bytes if prof_n else None, "launches_per_step": prof_n // max(args.steps, 1),
                "avg_us": avg_s * 1e6, "algorithmic_bytes_per_launch": prof_bytes, "peak_source": how,
                "note": "mean over every launch of the timed steps; late launches carry only the few tensors "
                        "still above tolerance, so the kernel is latency-bound there; traffic = the captured "
                        "DRAM/algorithmic ratio of a full-batch launch x the mean algorithmic bytes"}

    extra = {}
    if not args.no_extras:
        extra["multilevel_100cubed"] = run_multilevel_100cubed(ctx, stream, parity=rank == 0 and not args.no_cpu_baseline)
        extra.update(run_400cubed(ctx, stream, hbm, how))
        if args.serve_requests > 0:
            extra["served"] = run_served(args.serve_requests, parity=rank == 0 and not args.no_cpu_baseline)
        if not args.no_paper_dense:
            extra["paper_dense_ijk"] = run_paper_dense(ctx, stream)
            extra["paper_laplacian"] = run_paper_laplacian(ctx, stream)

    line = {
        "metric": METRIC, "value": t_step * 1e-3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": config({"parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
        "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": int(zbytes + fbytes),
                "d2h_bytes_per_step": int(fbytes)},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "err_vs_oracle": parity,
        "batched": batched,
        "gpu_launches": int(launches),
        "gpu_launches_note": "kernel launches per step issued by libcpmg",
        "clocks": clk,
        "step_ms": ms,
        **extra,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_multilevel_100cubed(ctx, stream, reps=3, parity=True):
    """The 100^3 rank-5 workload by the "Multilevel" driver of Section 6.1 (setup cycles, FAS solve
    cycles with the one-time rebuild, then plain ALS if stagnation persists), MIXED, to g < 1e-8;
    with `parity`, the oracle's solve from the same start beside it."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    p = problem()
    opts = cpmg.make_opts(precision=cpmg.PREC_MIXED, tol=TOL, coarsest=COARSEST, als_fallback=1)
    with torch.cuda.stream(stream):
        Z = cpmg.colmajor(p.Z)
        A0 = [cpmg.colmajor(a) for a in p.A0]
        T0 = [[cpmg.colmajor(a) for a in b] for b in p.tfms]
    A = [a.clone() for a in A0]
    T = [[a.clone() for a in b] for b in T0]
    ms, r = [], None
    for k in range(reps + 1):
        with torch.cuda.stream(stream):
            for a, a0 in zip(A, A0):
                a.copy_(a0)
            for b, b0 in zip(T, T0):
                for a, a0 in zip(b, b0):
                    a.copy_(a0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = cpmg.cpmg_decompose(ctx, Z, A, T, opts)
            e1.record(stream)
            e1.synchronize()
        if k:
            ms.append(e0.elapsed_time(e1))
    out = {"workload": "dense 100x100x100 fp32, R=5, congruence 0.9, noise 1%+5%, levels 100/50/25/13, g<1e-8",
           "seconds": statistics.mean(ms) * 1e-3, "solver": {k: r[k] for k in ("g", "f", "iters_setup", "iters_solve",
                                                                             "iters_als", "restarted", "levels", "status")}}
    if parity:
        from oracle import align, tensor as OT
        dt, ro = oracle_solve(p)
        got = [cpmg.to_numpy(a) for a in A]
        fo = OT.f_value(p.Z.astype(np.float64), ro.A)
        out["oracle"] = {"seconds": dt, "setup": ro.setup_cycles, "solve": ro.solve_cycles,
                         "als": getattr(ro, "als_iters", 0), "cores": blas_threads()}
        out["err_vs_oracle"] = {"factor_err": align.factor_error(ro.A, got), "rel_f": abs(r["f"] - fo) / fo}
    return out


def run_400cubed(ctx, stream, hbm, how):
    """The 400^3 rank-10 float32 tensor (256 MB, congruence 0.95, 1% noise): one ALS sweep with and
    without the dimension tree, the MTTKRP passes of the sweep against the measured HBM peak, the
    tensor-core restriction, and the "Multilevel" solve over five levels (400/200/100/50/25) to
    g < 1e-8 with the caps of Section 6.1 (500 cycles, 1e4 ALS iterations)."""
    import torch
    from paper_1111_6091_gb300 import cpmg, synth
    p4 = synth.make_problem((400, 400, 400), 10, congruence=0.95, eta_homo=0.01, dtype=np.float32, seed=0)
    out = {}
    with torch.cuda.stream(stream):
        Z4 = cpmg.colmajor(p4.Z)
        A0 = [cpmg.colmajor(a) for a in p4.A0]
    sweeps = {}
    for name, prec in (("fp32", cpmg.PREC_FP32), ("float_pair", cpmg.PREC_DF)):
        for tree in (1, 0):
            A = [a.clone() for a in A0]
            o = cpmg.make_opts(precision=prec, check_every=0, dimension_tree=tree)
            with torch.cuda.stream(stream):
                # the sweep time as the slope between a 10- and a 50-sweep call (each call also
                # captures its sweep graph and evaluates ||Z|| and f once), without timing events
                # (event nodes slow graph replay); then the MTTKRP passes timed with per-launch
                # events on another call
                cpmg.cp_als_sweep(ctx, Z4, A, 10, o)
                t = {}
                for nsw in (10, 50):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    cpmg.cp_als_sweep(ctx, Z4, A, nsw, o)
                    e1.record(stream)
                    e1.synchronize()
                    t[nsw] = e0.elapsed_time(e1)
                ctx.profile_reset()
                ctx.profile(True)
                cpmg.cp_als_sweep(ctx, Z4, A, 10, o)
                torch.cuda.synchronize()
                ms, n, b = ctx.profile_read(0 if prec == cpmg.PREC_FP32 else 1)
                ctx.profile(False)
            gbs = b / (ms * 1e-3 / n) / 1e9 if n else None
            sweeps[f"{name}_tree{tree}"] = {"ms_per_sweep": (t[50] - t[10]) / 40, "ms_per_call_fixed": t[10] - (t[50] - t[10]) / 4,
                                            "z_passes_per_sweep": n / 10,
                                            "mttkrp_gbs": gbs, "mttkrp_frac": gbs / hbm if gbs else None,
                                            "mttkrp_avg_us": ms * 1e3 / n if n else None}
    out["sweep_400cubed_r10"] = dict(sweeps, peak=hbm, peak_source=how)
    out["ttm_400cubed_tc"] = ttm_400cubed(ctx, stream, Z4, hbm, how)
    opts = cpmg.make_opts(precision=cpmg.PREC_MIXED, tol=TOL, coarsest=(25, 25, 25), als_fallback=1,
                          max_cycles=500, max_als_iters=10000)
    with torch.cuda.stream(stream):
        A = [a.clone() for a in A0]
        T = [[cpmg.colmajor(a) for a in b] for b in p4.tfms]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = cpmg.cpmg_decompose(ctx, Z4, A, T, opts)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    out["multilevel_400cubed_r10"] = {
        "workload": "dense 400^3 fp32, R=10, congruence 0.95, 1% noise, 5 levels, g<1e-8, Section 6.1 caps",
        "seconds": dt, "solver": {k: r[k] for k in ("g", "f", "iters_setup", "iters_solve", "iters_als", "restarted",
                                                    "refine_sweeps", "levels", "status")}}
    del Z4
    return out




TTM_DIMS, TTM_IC = (400, 400, 400), 200


def ttm_rhat(seed=3):
    import torch
    rng = np.random.default_rng(seed)
    return [torch.from_numpy(np.ascontiguousarray(rng.standard_normal((TTM_IC, I)).T)).cuda() for I in TTM_DIMS]


def ttm_400cubed(ctx, stream, Z4, hbm, how, reps=5):
    """Level-0 restriction of the 400^3 float tensor (modes 400 -> 200 in turn) on tcgen05 in
    split BF16: per-launch CUDA events around the three mode-product kernels."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    with torch.cuda.stream(stream):
        Rh = ttm_rhat()
        for _ in range(2):
            cpmg.cpmg_ttm(ctx, Z4, Rh, tensor_cores=1)
        ctx.profile(True)
        ctx.profile_reset()
        for _ in range(reps):
            cpmg.cpmg_ttm(ctx, Z4, Rh, tensor_cores=1)
        ms, n, bpl = ctx.profile_read(3)
        ctx.profile(False)
    I, c = TTM_DIMS[0], TTM_IC
    # useful flops of the three mode products, and the bytes each reads and writes once
    flops = 2.0 * c * I * (I * I) + 2.0 * c * I * (c * I) + 2.0 * c * I * (c * c)
    byts = 4.0 * (I ** 3 + c * I * I) + 4.0 * (c * I * I + c * c * I) + 4.0 * (c * c * I + c ** 3)
    t = ms * 1e-3 / reps
    npad = -(-c // 16) * 16
    tc_peak = peaks_tensor()
    return {"kernel": "ttm_tc (3 mode products 400->200, split BF16, FP32 accumulate)",
            "avg_us_per_restriction": t * 1e6, "launches": n,
            "achieved_gbs": byts / t / 1e9, "hbm_peak": hbm, "hbm_frac": byts / t / 1e9 / hbm,
            "useful_tflops": flops / t / 1e12,
            "tensor_tflops_issued": 3 * flops * npad / c / t / 1e12,
            "bf16_peak_tflops": tc_peak, "tensor_frac": 3 * flops * npad / c / t / 1e12 / tc_peak if tc_peak else None,
            "algorithmic_bytes": byts, "algorithmic_flops": flops, "peak_source": how}


def peaks_tensor():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d.get("bf16_tflops") or 0) or None
    except Exception:
        return 1900.0  # fallback burst figure




def batch_problems(count, seed=0):
    """The uneven batch workload (synth.batch_specs): 1% noise, float32, no test blocks."""
    from paper_1111_6091_gb300 import synth
    return [synth.make_problem(sp["dims"], sp["R"], congruence=sp["congruence"], eta_homo=0.01,
                               dtype=np.float32, seed=sp["seed"], n_t=0)
            for sp in synth.batch_specs(count, seed)]


def run_paper_dense(ctx, stream, s=100, R=3, reps=2):
    """The paper's dense tensor z_ijk = (i^2+j^2+k^2)^(-1/2) (Section 6.3, Table tab:IJK test 6:
    s = 100, R = 3), float64, to g < 1e-10 from uniform [0,1] starts: "Multilevel + FMG"
    (mg_setup, mg_fmg with 100 coarsest ALS iterations, mg_fas_solve; levels down to 4) against
    plain ALS (cp_als_sweep), both on the GPU in float64.  Wall time of the calls (each
    synchronizes), best of `reps` after one warm-up."""
    import torch
    from paper_1111_6091_gb300 import cpmg, synth
    Z = synth.ijk_tensor(s)
    rng = np.random.default_rng(0)
    A0 = [rng.uniform(size=(s, R)) for _ in range(3)]
    tfms = [[rng.uniform(size=(s, R)) for _ in range(3)] for _ in range(2)]
    lv, I = 1, s
    while (I + 1) // 2 >= 4:
        I = (I + 1) // 2
        lv += 1
    Ac0 = [rng.uniform(size=(I, R)) for _ in range(3)]
    kw = dict(precision=cpmg.PREC_FP64, tol=1e-10, coarsest=(I, I, I))
    with torch.cuda.stream(stream):
        Zd = cpmg.colmajor(Z)
        A0d = [cpmg.colmajor(a) for a in A0]
        T0d = [[cpmg.colmajor(a) for a in b] for b in tfms]
        Acd = [cpmg.colmajor(a) for a in Ac0]
    torch.cuda.synchronize()

    def ml_fmg():
        with torch.cuda.stream(stream):
            A = [a.clone() for a in A0d]
            T = [[a.clone() for a in b] for b in T0d]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            h, r1 = cpmg.mg_setup(ctx, Zd, A, T, **kw)
            dims, _ = h.level_info(h.levels() - 1)
            if tuple(int(dims[n]) for n in range(3)) != (I, I, I):
                h.free()
                raise RuntimeError("unexpected coarsest level %s" % (tuple(dims[:3]),))
            rf = cpmg.mg_fmg(ctx, h, Zd, Acd, A, nu=100, **kw)
            r2 = cpmg.mg_fas_solve(ctx, h, Zd, A, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        h.free()
        return dt, {"setup_cycles": r1["iters_setup"], "fmg_cycles": 1, "solve_cycles": r2["iters_solve"],
                    "als_fallback_iters": r2["iters_als"], "g": r2["g"], "levels": r1["levels"],
                    "status": r2["status"]}

    def als():
        with torch.cuda.stream(stream):
            A = [a.clone() for a in A0d]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            r = cpmg.cp_als_sweep(ctx, Zd, A, 20000, precision=cpmg.PREC_FP64, tol=1e-10, check_every=-1)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, {"iters": r["iters_als"], "g": r["g"], "status": r["status"]}

    best = {}
    for name, fn in (("ml_fmg", ml_fmg), ("als", als)):
        fn()
        runs = [fn() for _ in range(reps)]
        dt, info = min(runs, key=lambda x: x[0])
        best[name] = dict(seconds=dt, **info)
    return {"tensor": "z_ijk = (i^2+j^2+k^2)^(-1/2)", "s": s, "R": R, "tol": 1e-10, "precision": "fp64",
            "levels": lv, **best, "speedup": best["als"]["seconds"] / best["ml_fmg"]["seconds"],
            "paper_matlab_s": {"als": 80.2, "ml_fmg": 8.1, "note": "Table tab:IJK test 6, MATLAB on a 2.5 GHz "
                                                                  "Core 2 Duo; context only"}}


SERVE_RATE, SERVE_LARGE_FRAC = 2000.0, 0.05


# Table tab:LapParams tests run here, with the paper's Table tab:Laplacian results for context:
# (test, N, s, R, coarsest, paper ALS iterations / s, paper ML iterations / s)
LAPLACIAN_TESTS = [(1, 4, 20, 4, 10, 1897, 24.0, 37, 7.6), (2, 4, 20, 5, 10, 3329, 53.6, 64, 15.1),
                   (3, 4, 20, 6, 10, 3587, 70.3, 67, 17.5), (7, 6, 20, 2, 5, 1619, 187.0, 48, 111.4)]


def run_paper_laplacian(ctx, stream):
    """The paper's Laplacian tensor (Section 6.2), dense, float32 storage (exact), float64-accurate
    arithmetic (float pairs), uniform [0,1] starts, to g < 1e-10: the "Multilevel" solver against
    plain ALS (at most 1e4 iterations), per test of Table tab:LapParams."""
    import torch
    from paper_1111_6091_gb300 import cpmg, synth
    out = []
    for test, N, s, R, co, p_als_it, p_als_s, p_ml_it, p_ml_s in LAPLACIAN_TESTS:
        Z = synth.laplacian_tensor(N // 2, s, dtype=np.float32)
        A0 = synth.uniform_start(Z.shape, R, 0)
        tfms = [synth.uniform_start(Z.shape, R, 1 + t) for t in range(2)]
        with torch.cuda.stream(stream):
            Zd = cpmg.colmajor(Z)
            A = [cpmg.colmajor(a) for a in A0]
            tf = [[cpmg.colmajor(a) for a in b] for b in tfms]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = cpmg.cpmg_decompose(ctx, Zd, A, tf, precision=cpmg.PREC_DF, tol=1e-10, coarsest=(co,) * N)
            torch.cuda.synchronize()
            t_ml = time.perf_counter() - t0
            A = [cpmg.colmajor(a) for a in A0]
            t0 = time.perf_counter()
            ra = cpmg.cp_als_sweep(ctx, Zd, A, 10000, precision=cpmg.PREC_DF, tol=1e-10, check_every=-1)
            torch.cuda.synchronize()
            t_als = time.perf_counter() - t0
        del Zd
        out.append({"test": test, "N": N, "s": s, "R": R, "levels": r["levels"],
                    "multilevel": {"seconds": t_ml, "setup": r["iters_setup"], "solve": r["iters_solve"],
                                   "g": r["g"], "status": r["status"]},
                    "als": {"seconds": t_als, "iters": ra["iters_als"], "g": ra["g"], "status": ra["status"]},
                    "speedup": t_als / t_ml,
                    "paper_matlab": {"als_iters": p_als_it, "als_s": p_als_s, "ml_iters": p_ml_it, "ml_s": p_ml_s}})
    return {"tensor": "finite-difference Laplacian, order N = 2d, s^N dense", "tol": 1e-10, "precision": "float-pair",
            "tests": out, "note": "paper: MATLAB on a 2.5 GHz Core 2 Duo, sparse tensors, averages of 10 starts; context only"}


def run_served(nreq, pool_small=96, pool_large=4, seed=12345, precisions=("mixed", "fp64"), large_multilevel=False,
               parity=False):
    """Poisson arrivals (2000 requests/s) of CP-ALS requests to g < 1e-8 (at most 1e4 sweeps):
    95% drawn from a pool of tensors of the batch workload, 5% 256^3 R=8 tensors; admission
    budget 120 GB.  Served with MIXED and with plain FP64 arithmetic; p50/p99 latency and
    throughput of each.

    parity (the oracle leg): for the MIXED arm, the served results of a 1 % sample of the small
    requests against the oracle's ALS from the same start with the same stopping test (factor
    error, relative f), and for every large tensor served the oracle's own FP64 g (Eq. gradConv)
    and f of the served factors (an oracle solve of a 256^3 tensor takes far longer than the run;
    requests for the same tensor and start give bitwise the same factors)."""
    import torch
    from paper_1111_6091_gb300 import cpmg, synth
    small = batch_problems(pool_small, seed=1)
    rng = np.random.default_rng(seed)
    large = [synth.make_problem((256, 256, 256), 8, congruence=float(rng.uniform(0.5, 0.95)), eta_homo=0.01,
                                dtype=np.float32, seed=1000 + k, n_t=2 if large_multilevel else 0)
             for k in range(pool_large)]
    arrivals = np.cumsum(rng.exponential(1.0 / SERVE_RATE, nreq))
    picks = [("L", int(rng.integers(0, pool_large))) if rng.random() < SERVE_LARGE_FRAC
             else ("S", int(rng.integers(0, pool_small))) for _ in range(nreq)]
    out = {"requests": nreq, "rate_per_s": SERVE_RATE, "large_fraction": SERVE_LARGE_FRAC, "tol": BATCH_TOL,
           "max_sweeps": BATCH_MAX_IT, "budget_gb": 120,
           "large_solver": "multilevel (Section 6.1 driver, hierarchy resident per request)" if large_multilevel
           else "batched ALS"}
    arms = {"mixed": cpmg.PREC_MIXED, "fp64": cpmg.PREC_FP64}
    for name, prec in ((k, arms[k]) for k in precisions):
        stream = torch.cuda.Stream()
        ctx = cpmg.Context(0, stream=stream.cuda_stream)
        srv = cpmg.Server(ctx, budget_bytes=120 * 10**9, sweeps_per_launch=BATCH_CHECK)
        Zd = {("S", k): cpmg.colmajor(p.Z) for k, p in enumerate(small)}
        Zd.update({("L", k): cpmg.colmajor(p.Z) for k, p in enumerate(large)})
        A0 = {key: [cpmg.colmajor(a) for a in (small if key[0] == "S" else large)[key[1]].A0] for key in Zd}
        As = [[a.clone() for a in A0[key]] for key in picks]
        torch.cuda.synchronize()
        T0 = {("L", k): [[cpmg.colmajor(a) for a in b] for b in p.tfms] for k, p in enumerate(large)} \
            if large_multilevel else {}

        def submit(key, A):
            if large_multilevel and key[0] == "L":
                return srv.submit_multilevel(Zd[key], A, T0[key], precision=prec, tol=BATCH_TOL,
                                             max_als_iters=BATCH_MAX_IT, als_fallback=1,
                                             coarsest=(32, 32, 32))
            return srv.submit(Zd[key], A, precision=prec, tol=BATCH_TOL, max_als_iters=BATCH_MAX_IT)

        # warm: one request per shape class, so the unit-size tuning is not in the timed run
        warm = [submit(key, [a.clone() for a in A0[key]]) for key in Zd if key[0] == "S" or not large_multilevel]
        torch.cuda.synchronize()
        srv.wait(600.0)
        for t in warm:
            srv.poll(t)
        t0 = time.perf_counter()
        tickets = []
        for i, key in enumerate(picks):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            tickets.append(submit(key, As[i]))
        srv.wait(900.0)
        dt = time.perf_counter() - t0
        lats, conv, results = [], 0, []
        for t in tickets:
            r = srv.poll(t)
            results.append(r)
            lats.append(r["seconds"])
            conv += r["status"] == cpmg.OK
        lat_l = [l for l, key in zip(lats, picks) if key[0] == "L"]
        if parity and name == "mixed":
            out["err_vs_oracle"] = served_parity(results, picks, small, large, As, nreq)
        lats = np.sort(np.array(lats))
        out[name] = {"p50_s": float(np.percentile(lats, 50)), "p99_s": float(np.percentile(lats, 99)),
                     "req_per_s": nreq / dt, "seconds": dt, "converged": conv,
                     "large_p50_s": float(np.percentile(lat_l, 50)) if lat_l else None,
                     "large_requests": len(lat_l)}
        ctx.close()
    return out


def served_parity(results, picks, small, large, As, nreq):
    """Served results (the polled result dicts, in request order) against the oracle (see
    run_served)."""
    from paper_1111_6091_gb300 import cpmg
    from oracle import align, tensor as T
    step = max(1, nreq // max(1, nreq // 100))
    rows, seen = [], set()
    for i in range(0, nreq, step):
        key = picks[i]
        if key[0] != "S" or key in seen:
            continue
        seen.add(key)
        r = results[i]
        _, Ao, ito, go = oracle_batch_tensor(small[key[1]])
        got = [cpmg.to_numpy(a) for a in As[i]]
        Z64 = small[key[1]].Z.astype(np.float64)
        fo, fg = T.f_value(Z64, Ao), T.f_value(Z64, got)
        rows.append({"request": i, "pool_tensor": key[1], "factor_err": align.factor_error(Ao, got),
                     "rel_f": abs(fg - fo) / fo, "sweeps_gpu": r["iters_als"], "sweeps_oracle": ito})
    large_rows = []
    for k in range(len(large)):
        idx = [i for i, key in enumerate(picks) if key == ("L", k)]
        if not idx:
            continue
        i = idx[0]
        r = results[i]
        got = [cpmg.to_numpy(a) for a in As[i]]
        Z64 = large[k].Z.astype(np.float64)
        g_o, f_o = T.g_value(Z64, got), T.f_value(Z64, got)
        same = all(all(np.array_equal(cpmg.to_numpy(a), b) for a, b in zip(As[j], got)) for j in idx[1:])
        large_rows.append({"pool_tensor": k, "requests": len(idx), "g_oracle": g_o, "g_reported": r["g"],
                           "rel_f_reported_vs_oracle": abs(r["f"] - f_o) / f_o, "all_requests_bitwise_equal": same})
    return {"small_sample": f"{len(rows)} requests (every {step}th, one per pool tensor)",
            "max_factor_err": max((x["factor_err"] for x in rows), default=None),
            "max_rel_f": max((x["rel_f"] for x in rows), default=None), "small": rows, "large": large_rows}


def run_ttm_case(args):
    """Small case for profiler captures: one level-0 restriction of the 400^3 float tensor on
    tensor cores (three k_ttm_tc launches)."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    rng = np.random.default_rng(23)
    Zn = np.asfortranarray(rng.standard_normal(TTM_DIMS).astype(np.float32))
    ctx = cpmg.Context(0)
    Y = cpmg.cpmg_ttm(ctx, cpmg.colmajor(Zn), ttm_rhat(), tensor_cores=1)
    torch.cuda.synchronize()
    print(json.dumps({"case": "ttm 400^3 -> 200^3 tensor cores", "y00": float(Y.flatten()[0])}))
    ctx.close()


def run_sweep_case(args):
    """Small case for launch-list captures: 20 FP32 and 20 float-pair ALS sweeps of the 100^3
    rank-5 workload tensor (about 250 kernel launches)."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    p = problem()
    stream = torch.cuda.Stream()
    ctx = cpmg.Context(0, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        Z = cpmg.colmajor(p.Z)
        A = [cpmg.colmajor(a) for a in p.A0]
        for prec in (cpmg.PREC_FP32, cpmg.PREC_DF):
            cpmg.cp_als_sweep(ctx, Z, A, 20, precision=prec, check_every=0)
    torch.cuda.synchronize()
    print(json.dumps({"case": "als sweeps 100^3 R=5", "sweeps": 40}))
    ctx.close()


def run_batch_case(args):
    """Profiler case: the 512-tensor batch workload, 8 MIXED sweeps of every tensor plus one g
    evaluation.  Launches: the unit-size autotuner (5 candidates x (k_batch_init + 3 MTTKRP-only
    k_batch)), then one k_batch of 8 sweeps + g, then k_batch_sort."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    probs = batch_problems(BATCH_COUNT)
    ctx = cpmg.Context(0)
    Zs = [cpmg.colmajor(p.Z) for p in probs]
    As = [[cpmg.colmajor(a) for a in p.A0] for p in probs]
    # tol 1e-8 as in the benchmark; with --batch-case-sweeps S the last of the S/8 launches carries
    # the tensors still above tolerance after S - 8 sweeps (S = 1024: about 90 of the 512)
    st, res = cpmg.cpmg_batch_solve(ctx, Zs, As, precision=cpmg.PREC_MIXED, tol=BATCH_TOL if args.batch_case_sweeps > 8
                                    else 0.0, max_als_iters=args.batch_case_sweeps, check_every=8)
    torch.cuda.synchronize()
    print(json.dumps({"case": "batched %d tensors" % BATCH_COUNT, "sweeps": sum(r["iters_als"] for r in res),
                      "running_at_cap": sum(r["iters_als"] >= args.batch_case_sweeps for r in res)}))
    ctx.close()


def run_mttkrp_case(args):
    """Small case for profiler captures: two ALS sweeps on the 400^3 rank-10 tensor in the chosen
    arithmetic; with the dimension tree each sweep is the W pass (k_dt_w, or a tensor-core mode
    product for bf16x3) and one mode-3 pass."""
    import torch
    from paper_1111_6091_gb300 import cpmg, synth
    p4 = synth.make_problem((400, 400, 400), 10, congruence=0.95, eta_homo=0.01, dtype=np.float32, seed=0)
    ctx = cpmg.Context(0)
    Z4 = cpmg.colmajor(p4.Z)
    A4 = [cpmg.colmajor(a) for a in p4.A0]
    prec = {"fp32": cpmg.PREC_FP32, "df": cpmg.PREC_DF, "fp64": cpmg.PREC_FP64,
            "bf16x3": cpmg.PREC_BF16X3}[args.case_prec]
    r = cpmg.cp_als_sweep(ctx, Z4, A4, 2, precision=prec, check_every=0)
    torch.cuda.synchronize()
    print(json.dumps({"case": "mttkrp 400^3 R=10", "precision": args.case_prec, "f": r["f"]}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mttkrp-case", action="store_true", help="profiler case: 2 sweeps at 400^3")
    ap.add_argument("--case-prec", default="fp32", choices=["fp32", "df", "fp64", "bf16x3"])
    ap.add_argument("--ttm-case", action="store_true", help="profiler case: one 400^3 restriction")
    ap.add_argument("--sweep-case", action="store_true", help="profiler case: 40 ALS sweeps at 100^3")
    ap.add_argument("--batch-case", action="store_true", help="profiler case: one 8-sweep launch of the 512-tensor batch")
    ap.add_argument("--batch-case-sweeps", type=int, default=8,
                    help="batch case: solve to g < 1e-8 with this sweep cap (the last launch then carries the slow tensors)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paper-dense", action="store_true", help="skip the paper's dense-tensor comparison")
    ap.add_argument("--paper-dense", action="store_true", help="run only the paper's dense-tensor comparison")
    ap.add_argument("--solve-only", action="store_true", help="profiler case: the timed solves only")
    ap.add_argument("--no-batch-loop", dest="batch_loop", action="store_false",
                    help="skip the per-tensor launch loop over the batch")
    ap.add_argument("--served-only", action="store_true",
                    help="only the served request stream (--serve-requests, --serve-precisions, --serve-large-multilevel)")
    ap.add_argument("--serve-precisions", default="mixed,fp64")
    ap.add_argument("--serve-large-multilevel", action="store_true",
                    help="serve the 256^3 requests with the multilevel driver instead of batched ALS")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the batched workload (no 100^3 / 400^3 / served / paper-tensor measurements)")
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="requests of the served workload (20000 for the full stream; 0: skip)")
    args = ap.parse_args()
    if args.impl != "reference":
        from paper_1111_6091_gb300 import build
        build.build()
    if args.mttkrp_case:
        run_mttkrp_case(args)
    elif args.ttm_case:
        run_ttm_case(args)
    elif args.sweep_case:
        run_sweep_case(args)
    elif args.batch_case:
        run_batch_case(args)
    elif args.paper_dense:
        import torch
        from paper_1111_6091_gb300 import cpmg
        stream = torch.cuda.Stream()
        ctx = cpmg.Context(0, stream=stream.cuda_stream)
        print(json.dumps(run_paper_dense(ctx, stream)), flush=True)
        ctx.close()
    elif args.served_only:
        print(json.dumps({"served": run_served(args.serve_requests, precisions=tuple(args.serve_precisions.split(",")),
                                               large_multilevel=args.serve_large_multilevel,
                                               parity=not args.no_cpu_baseline)}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
