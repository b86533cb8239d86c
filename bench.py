#!/usr/bin/env python3
"""Benchmark: time-to-tolerance of the multilevel CP solver on one GPU.

Workload (one step): the 100x100x100 float32 tensor of rank 5 whose factor columns have
pairwise congruence 0.9, with 1% homoscedastic and 5% heteroscedastic noise (seeded
synthetic data), decomposed by the "Multilevel" solver (CP-AMG-mult setup cycles, then
CP-FAS solve cycles with the one-time rebuild, then plain ALS if stagnation persists)
from a fixed N(0,1) start until g < 1e-8 (Eq. gradConv), levels 100/50/25/13, MIXED
precision (FP32 sweeps, float64-accurate sweeps near the FP32 floor).

Timing: W untimed steps, then K steps each bracketed by CUDA events on the library's
stream, with a 512 MB write between steps to flush the 126 MB L2 (the tensor is 4 MB).
The finest-level MTTKRP launches inside the timed steps are timed with events by the
library (roofline).  The end-to-end number repeats the solve through the same C ABI call
with pinned host buffers, the copies inside the timed region.  A second measurement
times the FP32 MTTKRP of the 400x400x400 rank-10 tensor (256 MB, larger than L2) against
the measured HBM peak.

``--impl reference`` times the FP64 CPU oracle on the same workload instead.
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

DIMS, RANK, CONG, ETA1, ETA2, SEED = (100, 100, 100), 5, 0.9, 0.01, 0.05, 0
COARSEST = (13, 13, 13)
TOL = 1e-8
METRIC = "time-to-tol (rel err 1e-8)"
WORKLOAD = "dense 100x100x100 fp32, R=5, congruence 0.9, noise 1%+5%, multilevel 4 levels, g<1e-8"


def problem():
    from paper_1111_6091_gb300 import synth
    return synth.make_problem(DIMS, RANK, congruence=CONG, eta_homo=ETA1, eta_hetero=ETA2,
                              dtype=np.float32, seed=SEED)


def config(extra=None):
    c = {"workload": WORKLOAD, "dims": list(DIMS), "rank": RANK, "congruence": CONG,
         "noise": [ETA1, ETA2], "tol": TOL, "solver": "multilevel (setup + FAS + ALS fallback)",
         "precision": "mixed fp32 / float-pair", "l2": "flushed between steps (512 MB write)"}
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
    from oracle import multigrid as MG
    o = MG.Options(coarsest=COARSEST, tol=TOL, als_fallback=True)
    t = time.perf_counter()
    r = MG.multilevel(p.Z.astype(np.float64), p.A0, p.tfms, o)
    return time.perf_counter() - t, r


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        return max(n) if n else 1
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return
    p = problem()
    for _ in range(min(args.warmup, 1)):
        oracle_solve(p)
    times = []
    r = None
    for _ in range(args.steps):
        dt, r = oracle_solve(p)
        times.append(dt)
    v = statistics.mean(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * v,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config(),
        "cpu_baseline": {"value": v, "unit": "s", "cores": blas_threads(), "kind": "oracle",
                         "sample": "full solve of the workload by the FP64 NumPy oracle"},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_cycles": {"setup": r.setup_cycles, "solve": r.solve_cycles,
                          "als": getattr(r, "als_iters", 0), "converged": bool(r.converged)},
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
    p = problem()
    opts = cpmg.make_opts(precision=cpmg.PREC_MIXED, tol=TOL, coarsest=COARSEST, als_fallback=1)

    with torch.cuda.stream(stream):
        Z = cpmg.colmajor(p.Z)
        A0 = [cpmg.colmajor(a) for a in p.A0]
        T0 = [[cpmg.colmajor(a) for a in b] for b in p.tfms]
        A = [a.clone() for a in A0]
        T = [[a.clone() for a in b] for b in T0]
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def reset():
        for a, a0 in zip(A, A0):
            a.copy_(a0)
        for b, b0 in zip(T, T0):
            for a, a0 in zip(b, b0):
                a.copy_(a0)

    def step():
        return cpmg.cpmg_decompose(ctx, Z, A, T, opts)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            reset()
            step()
        torch.cuda.synchronize()
        ranks_barrier()
        clocks = Clocks()
        clocks.start()
        launches0 = ctx.launches()
        ms, results = [], []
        for _ in range(args.steps):
            reset()
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            results.append(step())
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        ranks_barrier()
        launches = (ctx.launches() - launches0) // max(args.steps, 1)
        clk = clocks.stop()
        # One more identical step with per-launch CUDA events on the finest-level MTTKRP main
        # kernel (the event nodes slow graph replay, so the timed steps above run without them).
        reset()
        flush.fill_(1.0)
        ctx.profile(True)
        ctx.profile_reset()
        step()
        torch.cuda.synchronize()
        prof = [ctx.profile_read(k) for k in range(3)]
        ctx.profile(False)
    t_step = max_over_ranks(statistics.mean(ms), device="cuda")

    if args.solve_only:
        if rank == 0:
            print(json.dumps({"solve_only": True, "ms": ms, "launches": int(launches)}), flush=True)
        ctx.close()
        return

    # end to end through the C ABI with pinned host buffers
    Zh = cpmg.colmajor(p.Z, device="cpu", pin=True)
    Ah = [cpmg.colmajor(a, device="cpu", pin=True) for a in p.A0]
    Th = [[cpmg.colmajor(a, device="cpu", pin=True) for a in b] for b in p.tfms]
    e2e = []
    for _ in range(args.steps):
        for a, a0 in zip(Ah, p.A0):
            a.copy_(torch.from_numpy(np.ascontiguousarray(a0.T)))
        for b, b0 in zip(Th, p.tfms):
            for a, a0 in zip(b, b0):
                a.copy_(torch.from_numpy(np.ascontiguousarray(a0.T)))
        with torch.cuda.stream(stream):
            flush.fill_(2.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cpmg.cpmg_decompose(ctx, Zh, Ah, Th, opts)
            torch.cuda.synchronize()
            e2e.append(time.perf_counter() - t0)
    h2d = Zh.numel() * 4 + sum(a.numel() * 8 for a in Ah) + sum(a.numel() * 8 for b in Th for a in b)
    d2h = sum(a.numel() * 8 for a in Ah) + sum(a.numel() * 8 for b in Th for a in b)

    # bandwidth kernel of the timed steps: the finest-level MTTKRP (bulk-copy kernel)
    kinds = ["fp32", "float-pair", "fp64"]
    tot = [x[0] for x in prof]
    k = int(np.argmax(tot))
    ms_k, n_k, bytes_k = prof[k]
    hbm, how = peaks()
    avg_s = ms_k * 1e-3 / max(n_k, 1)
    achieved = bytes_k / avg_s / 1e9 if n_k else None

    # 400^3 rank-10 FP32 MTTKRP bandwidth (inputs larger than L2)
    from paper_1111_6091_gb300 import synth
    p4 = synth.make_problem((400, 400, 400), 10, congruence=0.95, eta_homo=0.01, dtype=np.float32, seed=0)
    with torch.cuda.stream(stream):
        Z4 = cpmg.colmajor(p4.Z)
        A4 = [cpmg.colmajor(a) for a in p4.A0]
        o4 = cpmg.make_opts(precision=cpmg.PREC_FP32, check_every=0)
        cpmg.cp_als_sweep(ctx, Z4, A4, 3, o4)
        ctx.profile(True)
        ctx.profile_reset()
        cpmg.cp_als_sweep(ctx, Z4, A4, 10, o4)
        ms4, n4, b4 = ctx.profile_read(0)
        ctx.profile(False)
    gbs4 = b4 / (ms4 * 1e-3 / n4) / 1e9
    ttm4 = ttm_400cubed(ctx, stream, Z4, hbm, how)
    del Z4, A4
    batched = run_batched(ctx, stream, args.batch_count) if args.batch_count > 0 else None
    served = run_served(args.serve_requests) if args.serve_requests > 0 else None
    dense_ijk = run_paper_dense(ctx, stream) if not args.no_paper_dense else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        if batched is not None:
            batched["cpu_oracle_sample"] = oracle_batch_sample()
        dt, r = oracle_solve(p)
        cpu = {"value": dt, "unit": "s", "cores": blas_threads(), "kind": "oracle",
               "sample": "one full solve of the workload by the FP64 NumPy oracle (same solver and start)",
               "oracle_cycles": {"setup": r.setup_cycles, "solve": r.solve_cycles,
                                 "als": getattr(r, "als_iters", 0)}}

    res = results[-1]
    line = {
        "metric": METRIC, "value": t_step * 1e-3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": config({"parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
        "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": {"bound": "hbm", "kernel": f"k_mttkrp_tma ({kinds[k]}, 100^3 finest level)",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm if achieved else None, "traffic": None,
                     "launches": n_k, "avg_us": avg_s * 1e6, "peak_source": how,
                     "note": "timed on one extra profiled step of the same workload; the 4 MB tensor is "
                             "L2-resident inside a solve; frac is against HBM"},
        "mttkrp_400cubed_fp32": {"achieved": gbs4, "peak": hbm, "unit": "GB/s", "frac": gbs4 / hbm,
                                 "avg_us": ms4 * 1e3 / n4, "launches": n4, "peak_source": how},
        "ttm_400cubed_tc": ttm4,
        "batched": batched,
        "served": served,
        "paper_dense_ijk": dense_ijk,
        "cpu_baseline": cpu,
        "gpu_launches": int(launches),
        "gpu_launches_note": "kernel launches per step issued by libcpmg (graph replays count their kernels)",
        "clocks": clk,
        "solver": {k2: res[k2] for k2 in ("g", "f", "iters_setup", "iters_solve", "iters_als", "restarted",
                                          "refine_sweeps", "levels", "status")},
        "step_ms": ms,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


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


BATCH_COUNT, BATCH_TOL, BATCH_MAX_IT, BATCH_CHECK = 512, 1e-8, 1000, 8


def batch_problems(count, seed=0):
    """The uneven batch workload (synth.batch_specs): 1% noise, float32, no test blocks."""
    from paper_1111_6091_gb300 import synth
    return [synth.make_problem(sp["dims"], sp["R"], congruence=sp["congruence"], eta_homo=0.01,
                               dtype=np.float32, seed=sp["seed"], n_t=0)
            for sp in synth.batch_specs(count, seed)]


def oracle_batch_sample(count=32, sweeps=5):
    """The FP64 oracle's ALS on a bounded sample of the batch workload (its first `count`
    tensors, `sweeps` sweeps each), as tensor-sweeps per second on the host cores."""
    from oracle import als as ALS
    probs = batch_problems(count)
    t = time.perf_counter()
    for p in probs:
        A = p.A0
        Z64 = p.Z.astype(np.float64)
        for _ in range(sweeps):
            A = ALS.als_sweep(Z64, A)
    dt = time.perf_counter() - t
    return {"value": count * sweeps / dt, "unit": "tensor-sweeps/s", "cores": blas_threads(), "kind": "oracle",
            "sample": f"FP64 NumPy ALS, {sweeps} sweeps of each of the first {count} tensors of the batch"}


def run_batched(ctx, stream, count=BATCH_COUNT):
    """Batched CP-ALS of `count` uneven tensors to g < 1e-8 (at most 1000 sweeps each) in MIXED
    and in FP64 arithmetic, and the same MIXED solves as a loop of per-tensor cp_als_sweep calls."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    probs = batch_problems(count)
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

    out = {"count": count, "tol": BATCH_TOL, "max_sweeps": BATCH_MAX_IT, "check_every": BATCH_CHECK}
    zbytes = [p.Z.nbytes for p in probs]
    for name, prec in (("mixed", cpmg.PREC_MIXED), ("fp64", cpmg.PREC_FP64)):
        reset()
        # first call tunes the unit sizes for these shape classes; time the second
        cpmg.cpmg_batch_solve(ctx, Zs, As, precision=prec, tol=BATCH_TOL, max_als_iters=BATCH_MAX_IT,
                              check_every=BATCH_CHECK)
        reset()
        t0 = time.perf_counter()
        st, res = cpmg.cpmg_batch_solve(ctx, Zs, As, precision=prec, tol=BATCH_TOL, max_als_iters=BATCH_MAX_IT,
                                        check_every=BATCH_CHECK)
        dt = time.perf_counter() - t0
        sweeps = sum(r["iters_als"] for r in res)
        zsw = sum(r["iters_als"] * len(p.Z.shape) * b for r, p, b in zip(res, probs, zbytes))
        out[name] = {"seconds": dt, "converged": sum(r["status"] == cpmg.OK for r in res),
                     "tensor_sweeps": sweeps, "tensor_sweeps_per_s": sweeps / dt,
                     "sweep_z_gbs": zsw / dt / 1e9}
    # per-tensor launch loop (the same MIXED solves one tensor at a time)
    reset()
    t0 = time.perf_counter()
    conv = 0
    with torch.cuda.stream(stream):
        for Z, A in zip(Zs, As):
            r = cpmg.cp_als_sweep(ctx, Z, A, BATCH_MAX_IT, precision=cpmg.PREC_MIXED, tol=BATCH_TOL,
                                  check_every=BATCH_CHECK)
            conv += r["status"] == cpmg.OK
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out["per_tensor_loop_mixed"] = {"seconds": dt, "converged": conv}
    out["speedup_vs_loop"] = dt / out["mixed"]["seconds"]
    out["mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    return out


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


def run_served(nreq, pool_small=96, pool_large=4, seed=12345):
    """Poisson arrivals (2000 requests/s) of CP-ALS requests to g < 1e-8 (at most 1000 sweeps):
    95% drawn from a pool of tensors of the batch workload, 5% 256^3 R=8 tensors; admission
    budget 120 GB.  Served with MIXED and with plain FP64 arithmetic; p50/p99 latency and
    throughput of each."""
    import torch
    from paper_1111_6091_gb300 import cpmg, synth
    small = batch_problems(pool_small, seed=1)
    rng = np.random.default_rng(seed)
    large = [synth.make_problem((256, 256, 256), 8, congruence=float(rng.uniform(0.5, 0.95)), eta_homo=0.01,
                                dtype=np.float32, seed=1000 + k, n_t=0) for k in range(pool_large)]
    arrivals = np.cumsum(rng.exponential(1.0 / SERVE_RATE, nreq))
    picks = [("L", int(rng.integers(0, pool_large))) if rng.random() < SERVE_LARGE_FRAC
             else ("S", int(rng.integers(0, pool_small))) for _ in range(nreq)]
    out = {"requests": nreq, "rate_per_s": SERVE_RATE, "large_fraction": SERVE_LARGE_FRAC, "tol": BATCH_TOL,
           "max_sweeps": BATCH_MAX_IT, "budget_gb": 120}
    for name, prec in (("mixed", cpmg.PREC_MIXED), ("fp64", cpmg.PREC_FP64)):
        stream = torch.cuda.Stream()
        ctx = cpmg.Context(0, stream=stream.cuda_stream)
        srv = cpmg.Server(ctx, budget_bytes=120 * 10**9, sweeps_per_launch=BATCH_CHECK)
        Zd = {("S", k): cpmg.colmajor(p.Z) for k, p in enumerate(small)}
        Zd.update({("L", k): cpmg.colmajor(p.Z) for k, p in enumerate(large)})
        A0 = {key: [cpmg.colmajor(a) for a in (small if key[0] == "S" else large)[key[1]].A0] for key in Zd}
        As = [[a.clone() for a in A0[key]] for key in picks]
        torch.cuda.synchronize()
        # warm: one request per shape class, so the unit-size tuning is not in the timed run
        warm = [srv.submit(Zd[key], [a.clone() for a in A0[key]], precision=prec, tol=BATCH_TOL,
                           max_als_iters=BATCH_MAX_IT) for key in Zd]
        torch.cuda.synchronize()
        srv.wait(600.0)
        for t in warm:
            srv.poll(t)
        t0 = time.perf_counter()
        tickets = []
        for i, key in enumerate(picks):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            tickets.append(srv.submit(Zd[key], As[i], precision=prec, tol=BATCH_TOL, max_als_iters=BATCH_MAX_IT))
        srv.wait(900.0)
        dt = time.perf_counter() - t0
        lats, conv = [], 0
        for t in tickets:
            r = srv.poll(t)
            lats.append(r["seconds"])
            conv += r["status"] == cpmg.OK
        lats = np.sort(np.array(lats))
        out[name] = {"p50_s": float(np.percentile(lats, 50)), "p99_s": float(np.percentile(lats, 99)),
                     "req_per_s": nreq / dt, "seconds": dt, "converged": conv}
        ctx.close()
    return out


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
    evaluation.  Launches: the unit-size autotuner (5 candidates x (k_batch_init + 2 MTTKRP-only
    k_batch)), then one k_batch of 8 sweeps + g, then k_batch_sort."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    probs = batch_problems(BATCH_COUNT)
    ctx = cpmg.Context(0)
    Zs = [cpmg.colmajor(p.Z) for p in probs]
    As = [[cpmg.colmajor(a) for a in p.A0] for p in probs]
    st, res = cpmg.cpmg_batch_solve(ctx, Zs, As, precision=cpmg.PREC_MIXED, tol=0.0, max_als_iters=8,
                                    check_every=8)
    torch.cuda.synchronize()
    print(json.dumps({"case": "batched %d tensors" % BATCH_COUNT, "sweeps": sum(r["iters_als"] for r in res)}))
    ctx.close()


def run_mttkrp_case(args):
    """Small case for profiler captures: two FP32 ALS sweeps on the 400^3 rank-10 tensor
    (six MTTKRP main-kernel launches)."""
    import torch
    from paper_1111_6091_gb300 import cpmg, synth
    p4 = synth.make_problem((400, 400, 400), 10, congruence=0.95, eta_homo=0.01, dtype=np.float32, seed=0)
    ctx = cpmg.Context(0)
    Z4 = cpmg.colmajor(p4.Z)
    A4 = [cpmg.colmajor(a) for a in p4.A0]
    prec = {"fp32": cpmg.PREC_FP32, "df": cpmg.PREC_DF, "fp64": cpmg.PREC_FP64}[args.case_prec]
    r = cpmg.cp_als_sweep(ctx, Z4, A4, 2, precision=prec, check_every=0)
    torch.cuda.synchronize()
    print(json.dumps({"case": "mttkrp 400^3 R=10", "precision": args.case_prec, "f": r["f"]}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mttkrp-case", action="store_true", help="profiler case: 2 sweeps at 400^3")
    ap.add_argument("--case-prec", default="fp32", choices=["fp32", "df", "fp64"])
    ap.add_argument("--ttm-case", action="store_true", help="profiler case: one 400^3 restriction")
    ap.add_argument("--sweep-case", action="store_true", help="profiler case: 40 ALS sweeps at 100^3")
    ap.add_argument("--batch-case", action="store_true", help="profiler case: one 8-sweep launch of the 512-tensor batch")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-paper-dense", action="store_true", help="skip the paper's dense-tensor comparison")
    ap.add_argument("--paper-dense", action="store_true", help="run only the paper's dense-tensor comparison")
    ap.add_argument("--solve-only", action="store_true", help="profiler case: the timed solves only")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT, help="batched workload size (0: skip)")
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
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
