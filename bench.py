"""Benchmark: biharmonic DOF/s to a fixed error on one or more B300s.

A step is one whole solve (Algorithm 1: Schur right-hand side, GMRES on the
Schur system to relative residual 1e-12, recovery of V and U) of the 3D
variable-coefficient clamped problem on a 1024^3 grid: u = prod_a
sin^2(pi x_a) sin(32 pi x_a), coefficient 1 + 0.5 * (6 seeded Fourier modes,
wavenumbers <= 4), FP64 throughout.  DOF = interior unknowns (N-1)^3 per
solve.  Beside it: the same workload through the mixed path (FP32 inner
solves, FP64 refinement), the 2D 4096^2 workload in both precisions, the
serving stream, and the oracle's timing sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME --n N] [--prec fp64|mixed]

Multi-GPU runs (torchrun) solve independent replicas, one per rank (the
solve does not shard on this pool: every box has one GPU); value is the sum
over ranks.  The reference arm times the CPU oracle (assembled coupled
system + SuperLU) on a bounded sample of the same workload (--cpu-n).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "biharmonic DOF/s to fixed error"
UNIT = "DOF/s"
# FP64 peak of the B300, derived from the FP64 pipe's issue rate (ncu: 2 FP64
# thread operations per clock per SM, an FMA counting 2 flops) at the maximum
# SM clock: 148 x 2 x 2 x 2.032e9 flop/s
FP64_PEAK_TFLOPS_DERIVED = 148 * 2 * 2 * 2.032e9 / 1e12

# Arrival rate of the serving stream as a fraction of the sequential FP64
# capacity estimated from one warm solve per shape.  The estimate leaves out
# the per-request data copy, plan load and error check and the spread of
# iteration counts over the requests' data (measured on B300: 26 ms per
# request served one at a time against 20.4 ms estimated), so at 0.8 the
# one-at-a-time arm saturated; at 0.6 every arm stays below its capacity.
SERVE_LOAD = 0.6

# DRAM bytes (read + write) per launch of the dominant kernel class from an
# ncu capture, scaled to the bench's grid by the points processed
# (profiles/k_dst_fp64_3d512x256x256.md): at 512 x 256 x 256 the x-DST moves
# 500.6 MB (`<2,0>`, M(V/alpha) load), 761.1 MB (`<0,1>`, 1/alpha store) and
# 473.1 MB (`<0,0>`) per launch; 1023^3 / (511 x 255 x 255) = 32.22 times the
# points; weighted by the finest grid's 19 / 19 / 8 launches of a solve
# (profiles/launches_fourier3d_k32_1024_fp64.md)
PROFILED_TRAFFIC = {("fourier3d_k32", (1024, 1024, 1024), "dst_x"):
                    32.22e6 * (19 * 500.6 + 19 * 761.1 + 8 * 473.1) / 46}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def dst_flops_per_line(N: int) -> float:
    """The algorithmic flop count of one DST-I line (N/2-point complex FFT
    with pre- and post-processing), fixed independently of how a kernel fuses
    the operations into FMAs: a complex product counts as 6 flops.

    pre-processing 8 per pair (N/2 pairs); radix-2 stage 4 per butterfly;
    radix-4 stage 34 per butterfly (16 without twiddles in the first stage);
    post-processing 14 per pair (M/2 pairs); prefix sum ~2 per odd output;
    output scaling 1 per element.
    """
    M = N // 2
    logM = int(round(math.log2(M)))
    f = 8 * (N // 2)
    stages = []
    ns = 1
    if logM % 2:
        f += 4 * (M // 2)
        ns = 2
    while ns < M:
        f += (34 if ns > 1 else 16) * (M // 4)
        ns *= 4
    f += 14 * (M // 2) + 2 * M + N
    return float(f)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except Exception:
                continue
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            sm.sort()
            out["sm_mhz"] = sm[len(sm) // 2]
            out["sm_max_mhz"] = max(mx)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(sm)
        try:
            os.unlink(self.path)
        except Exception:
            pass
        return out


def max_over_ranks(values, world, device):
    """The largest of each value over the ranks (the slowest rank's time
    decides a replicated run); one all-reduce on the initialised process
    group when world > 1."""
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


_HOST_GROUP = None  # gloo group of all ranks for the host barriers (None: the default group is gloo)


def host_barrier(world: int, timeout_s: float) -> None:
    """Bounded barrier of all ranks on the host.  A rank that raised, exited
    or never arrives makes the others raise within `timeout_s` (the error
    names the missing ranks) instead of waiting for the process group's own
    timeout.  The caller synchronises its device first."""
    if world <= 1:
        return
    import datetime

    import torch.distributed as dist

    dist.monitored_barrier(group=_HOST_GROUP, timeout=datetime.timedelta(seconds=timeout_s), wait_all_ranks=True)


def whole_job_rate(world: int, steps: int, units_per_step: float, ms: float) -> float:
    """Units all ranks processed per second: each rank runs `steps` steps of
    `units_per_step` units, the job takes the slowest rank's `ms`."""
    return world * steps * units_per_step / (ms / 1e3)


_SAMPLES = {}


def cpu_oracle_sample(name: str, N_cpu: int):
    """Time the CPU oracle (assembly + SuperLU) on workload `name` at N_cpu
    intervals per axis; returns (DOF/s, seconds, err against the exact u,
    assembly seconds, SuperLU factor-and-solve seconds).

    The synthetic inputs are generated once, outside the timed region."""
    import numpy as np

    from oracle import coupled
    from paper_2609_16478_b300 import inputs

    key = (name, N_cpu)
    prob = inputs.config_problem(name)
    if key not in _SAMPLES:
        _SAMPLES[key] = inputs.sample(prob, [N_cpu] * prob.dim)
    d = _SAMPLES[key]
    t0 = time.perf_counter()
    sys_ = coupled.assemble(d)
    t1 = time.perf_counter()
    sol = coupled.solve_direct(sys_, d)
    dt = time.perf_counter() - t0
    err = float(np.max(np.abs(sol.U - d["u_exact"])))
    return (N_cpu - 1) ** prob.dim / dt, dt, err, t1 - t0, dt - (t1 - t0)


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def run_reference(args, rank, world):
    """The oracle as the reference arm (rank 0 only): each step one direct
    solve of the bench's workload at the bounded size --cpu-n."""
    if rank != 0:
        return
    from paper_2609_16478_b300 import inputs

    name, N_cpu = args.workload, args.cpu_n
    dim = inputs.config_problem(name).dim
    for _ in range(args.warmup):
        cpu_oracle_sample(name, N_cpu)
    t0 = time.perf_counter()
    errs, t_asm, t_lu = [], 0.0, 0.0
    for _ in range(args.steps):
        _, _, e, ta, tl = cpu_oracle_sample(name, N_cpu)
        errs.append(e)
        t_asm += ta
        t_lu += tl
    dt = time.perf_counter() - t0
    value = args.steps * (N_cpu - 1) ** dim / dt
    sample = ("direct solve of the assembled coupled system (SuperLU, single-threaded; %d host cores visible) of "
              "the bench's workload at N=%d per step (the GPU arm solves N=%d)" % (_cores(), N_cpu, args.n))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload_name(name, args.n, dim) + ", oracle sample N=%d" % N_cpu,
                   "dim": dim, "N": N_cpu, "err_inf_vs_exact": max(errs),
                   "note": "a timing sample: the high-wavenumber u is not resolved at this N"
                   if name == "fourier3d_k32" else ""},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "split_s": {"assembly": t_asm, "superlu": t_lu}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def paper_suite(args, dev):
    """The paper's printed workloads at their largest sizes, one JSON line each:
    Example 1 (Table 1) at 4096^2, Examples 2-3 (Tables 2-3, variable beta/alpha)
    at 512^3, and Table 4's classical-biharmonic timing problems at 1024^3,
    FP64 and mixed; the error against the exact solution beside the printed one."""
    import torch

    from paper_2609_16478_b300 import ahoc, inputs
    printed = {("singular2d", 4096): 4.54e-10, ("singular2d_eps1e-5", 4096): 4.65e-9,
               ("peak3d_q10_p0.2", 512): 8.50e-7, ("peak3d_q5_p1", 512): 1.07e-8,
               ("sincos3d_var_5_1_5", 512): 1.05e-10, ("sincos3d_var_25_5_25", 512): 7.45e-8}
    paper_cpu_s = {("classic3d_peak", 1024): 362.76, ("classic3d_sincos", 1024): 161.88,
                   ("classic3d_peak", 512): 44.86, ("classic3d_sincos", 512): 19.89}
    runs = [("singular2d", 4096), ("singular2d_eps1e-5", 4096), ("peak3d_q10_p0.2", 512), ("peak3d_q5_p1", 512),
            ("sincos3d_var_5_1_5", 512), ("sincos3d_var_25_5_25", 512), ("classic3d_peak", 512),
            ("classic3d_sincos", 512), ("classic3d_peak", 1024), ("classic3d_sincos", 1024)]
    for name, N in runs:
        prob = inputs.config_problem(name)
        d = inputs.sample(prob, [N] * prob.dim, backend="torch", device=dev)
        f = d["f"].reshape(-1).contiguous()
        for prec in ("fp64", "mixed"):
            st = torch.cuda.Stream(device=dev)
            p = ahoc.plan_for(d, device=dev, prec=prec, restart=100, max_iters=1000, stream=st)
            u = torch.empty_like(f)
            p.solve(f, u, tol=1e-12, check=False)
            st.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _, info = p.solve(f, u, tol=1e-12)
            e1.record(st)
            st.synchronize()
            ms = e0.elapsed_time(e1)
            err = float((u.reshape(d["u_exact"].shape) - d["u_exact"]).abs().max())
            dof = (N - 1) ** prob.dim
            print(json.dumps({"suite": "paper", "workload": name, "N": N, "dim": prob.dim, "prec": prec,
                              "ms": ms, "dof_per_s": dof / (ms / 1e3), "err_inf_vs_exact": err,
                              "paper_err_inf": printed.get((name, N)),
                              "paper_cpu_s_16_threads": paper_cpu_s.get((name, N)),
                              "gmres_iters": info["iters"], "coarse_iters": info["coarse_iters"],
                              "refine_steps": info["refine_steps"], "vsolve_iters": info["vsolve_iters"]}),
                  flush=True)
            p.close()
        del d, f
        torch.cuda.empty_cache()


def serving_variant(args, dev):
    """The serving workload: a seeded Poisson stream of requests of mixed
    dimension, size, coefficient and right-hand side, at SERVE_LOAD of the
    measured sequential FP64 capacity (below the capacity of every arm), served three
    ways: the batched mixed-precision server, the same server in FP64 (same
    workers and batches: the precision gain apart from the batching gain),
    and one-at-a-time FP64 solves."""
    import torch

    from paper_2609_16478_b300 import ahoc, autotune, inputs, serving

    tol = args.serve_tol
    p3 = 0.3
    mix = {(2, n): (1 - p3) / len(inputs.SERVE_2D) for n in inputs.SERVE_2D}
    mix.update({(3, n): p3 / len(inputs.SERVE_3D) for n in inputs.SERVE_3D})
    # sequential capacity per precision, one warm solve per shape
    t_seq = {"mixed": {}, "fp64": {}}
    for prec in t_seq:
        for (dim, n) in mix:
            d = inputs.sample_request(inputs.RequestSpec(10 ** 6, dim, n, (1,) * dim, 0.0), device=dev)
            p = ahoc.Plan(dim, [n] * dim, d["alpha"], prec=prec, restart=60, max_iters=2000)
            p.solve(d["f"], tol=tol)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p.solve(d["f"], tol=tol)
            t_seq[prec][(dim, n)] = time.perf_counter() - t0
            p.close()
    cap = {prec: 1.0 / sum(mix[k] * t_seq[prec][k] for k in mix) for prec in t_seq}
    rate = SERVE_LOAD * min(cap.values())
    specs = inputs.request_stream(args.serve_requests, rate, seed=5)

    def warm_specs(batch_for, size, copies, rid0):
        # `copies` batches of `size` requests of every shape at once (at most
        # the shape's batch): with as many workers, the pool then holds that
        # many plans of that size per shape
        out, rid = [], rid0
        for (dim, n) in mix:
            for _ in range(copies * min(size, batch_for((dim, n)))):
                out.append(inputs.RequestSpec(rid, dim, n, (0,) * dim, 0.0))
                rid += 1
        return out

    def arm(prec, workers, batch_for):
        srv = serving.Server(device=dev, prec=prec, tol=tol, workers=workers, batch_for=batch_for,
                             check_exact=True)
        srv.sched.max_slots = args.serve_slots
        # plans of every power-of-two batch size, one per worker, resident before
        # the stream starts: no plan is created inside a request's latency
        size = 1
        while size <= max(batch_for(k) for k in mix):
            srv.sched.batch_for = lambda k, s=size: min(s, batch_for(k))  # batches of exactly this size
            srv.run(warm_specs(batch_for, size, workers, 10 ** 7 + 10000 * size), realtime=False)
            size *= 2
        srv.sched.batch_for = batch_for
        recs = srv.run(specs, realtime=True)
        srv.close()
        torch.cuda.empty_cache()
        return recs, serving.summarize(recs)

    # the batched servers take the tuner's batch sizes (and, in mixed, its launch shapes)
    cache = autotune.load(args.tune_cache)
    autotune.apply(cache)
    bfor = autotune.batch_for(cache, "mixed", serving.default_batch)
    ra, sa = arm("mixed", args.serve_workers, bfor)
    for k in cache:  # the FP64 arms run with the built-in shapes
        dim, n, _ = k.split(":")
        for kind in (ahoc.AHOC_TUNE_TRI_CHUNK, ahoc.AHOC_TUNE_DST_THREADS, ahoc.AHOC_TUNE_DST_RADIX):
            ahoc.lib().ahoc_tune_set(kind, int(dim), int(n), ahoc.AHOC_MIXED, 0)
    rb, sb = arm("fp64", args.serve_workers, bfor)
    rc, sc = arm("fp64", 1, lambda k: 1)
    ea = {r.rid: r.err_inf for r in ra}
    eb = {r.rid: r.err_inf for r in rb}
    ec = {r.rid: r.err_inf for r in rc}
    ratio = max(ea[i] / ec[i] for i in ea if ea[i] is not None and ec[i])
    return {
        "workload": "%d requests, Poisson arrivals (seed 5) at %.1f req/s = %d%% of the sequential FP64 capacity "
                    "%.1f req/s (sequential mixed capacity %.1f req/s); 2D N in %s (p=0.7), 3D N in %s; per-request "
                    "Fourier coefficient (M=6, K=4, A=0.5, seed = request id) and u = prod sin^2(pi x) cos(m pi x), "
                    "m in 0..4; Schur tol %g"
                    % (len(specs), rate, round(100 * SERVE_LOAD), cap["fp64"], cap["mixed"], list(inputs.SERVE_2D),
                       list(inputs.SERVE_3D), tol),
        "latency": "from the request's arrival with its data (alpha and f, synthesised from closed forms on a "
                   "feeder stream before the request enters the queue, as a client upload would be complete) to "
                   "its solution in device memory; parts: queue wait, copy of the data into the plan slot and "
                   "ahoc_plan_load, solve; the error check against the exact u runs after it.  Plans of shapes "
                   "up to 2^21 interior points run on high-priority streams",
        "batched_mixed": dict(sa, workers=args.serve_workers, plan_slots_per_shape=args.serve_slots,
                              batch="per shape from the autotuner: %s" % {k: v["batch"] for k, v in cache.items()}),
        "batched_fp64": dict(sb, workers=args.serve_workers, batch="as batched_mixed"),
        "sequential_fp64": dict(sc, workers=1, batch=1),
        "p99_speedup_mixed_over_batched_fp64": sb["p99_ms"] / sa["p99_ms"],
        "p99_speedup_mixed_over_sequential_fp64": sc["p99_ms"] / sa["p99_ms"],
        "dof_per_s_ratio_mixed_over_batched_fp64": sa["dof_per_s"] / sb["dof_per_s"],
        "max_err_ratio_mixed_over_fp64": ratio,
        "max_err_inf": max(max(v for v in e.values() if v is not None) for e in (ea, eb, ec)),
        "seq_ms_per_shape": {prec: {"%dD N=%d" % k: 1e3 * v for k, v in t.items()} for prec, t in t_seq.items()},
    }


HEADLINE = ("fourier3d_k32", 1024)   # 3D 1024^3, u = prod sin^2(pi x_a) sin(32 pi x_a), 6-mode coefficient in [0.5, 1.5]
VARIANT_2D = ("fourier2d", 4096)      # 2D 4096^2, 8-mode coefficient in [0.6, 1.4]


def _grid_str(N, dim):
    if isinstance(N, (list, tuple)):
        return "x".join(str(n) for n in N) if len(set(N)) > 1 else "%d^%d" % (N[0], dim)
    return "%d^%d" % (N, dim)


def _workload_name(name, N, dim):
    gs = _grid_str(N, dim)
    if name == "fourier3d_k32":
        return ("3D variable-coefficient clamped biharmonic, high wavenumber (u = prod sin^2(pi x_a) sin(32 pi x_a), "
                "coefficient 1 + 0.5 * 6 seeded Fourier modes) N=%s" % gs)
    if name == "fourier3d":
        return "3D variable-coefficient clamped biharmonic (Fourier coefficient, 6 modes) N=%s" % gs
    return "2D variable-coefficient clamped biharmonic (Fourier coefficient, 8 modes) N=%s" % gs


def _interior(N, dim):
    if isinstance(N, (list, tuple)):
        out = 1
        for n in N:
            out *= n - 1
        return out
    return (N - 1) ** dim


def _kernel_pass(data, dev, stream, prec, args):
    """One solve on an event-timed plan (every launch bracketed by CUDA events
    on the plan's stream, plain launches); the plan is closed on return."""
    import torch

    from paper_2609_16478_b300 import ahoc

    f = data["f"].reshape(-1).contiguous()
    p = ahoc.plan_for(data, device=dev, timing=True, restart=args.restart, max_iters=args.max_iters,
                      levels=args.levels if prec == "fp64" else -1, prec=prec, stream=stream)
    u = torch.empty_like(f)
    _, ti = p.solve(f, u, tol=args.tol)
    p.close()
    del u
    torch.cuda.empty_cache()
    return ti


def _dst_rates(ti, N, dim, itemsize):
    """Per DST class of the finest grid: average event-timed launch time and
    the algorithmic HBM rate (one read and one write of every interior point
    per launch)."""
    out = {}
    nbytes = 2 * itemsize * _interior(N, dim)
    for k in ("dst_x", "dst_y"):
        n = ti["kernel_launches_top"][k]
        if n == 0:
            continue
        ms = ti["kernel_ms_top"][k] / n
        out[k] = {"launches": n, "avg_launch_ms": ms, "algorithmic_bytes_per_launch": nbytes,
                  "hbm_GBs": nbytes / (ms / 1e3) / 1e9}
    return out


def _timed_solves(plan, f, u, steps, args, clk=None):
    import torch

    st = plan.stream
    infos = []
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        _, info = plan.solve(f, u, tol=args.tol)
        infos.append(info)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), infos


def _mixed_variant(data, dev, stream, args, u_ref):
    """The same workload through the mixed path (FP32 inner solves, FP64 refinement)."""
    import torch

    from paper_2609_16478_b300 import ahoc

    N = list(data["N"])
    dim = data["dim"]
    f = data["f"].reshape(-1).contiguous()
    pm = ahoc.plan_for(data, device=dev, restart=args.restart, max_iters=args.max_iters, prec="mixed",
                       stream=stream)
    um = torch.empty_like(f)
    for _ in range(args.mixed_warmup):
        pm.solve(f, um, tol=args.tol)
    steps = args.mixed_steps
    mms, ims = _timed_solves(pm, f, um, steps, args)
    pm.close()
    torch.cuda.empty_cache()
    err = float((um.reshape(data["u_exact"].shape) - data["u_exact"]).abs().max())
    rel = float(torch.linalg.norm(um - u_ref) / torch.linalg.norm(u_ref))
    del um
    torch.cuda.empty_cache()
    tm = _kernel_pass(data, dev, stream, "mixed", args)
    im = ims[-1]
    return {
        "value": steps * _interior(N, dim) / (mms / 1e3), "unit": UNIT, "ms_per_step": mms / steps, "steps": steps,
        "dtype": "f32 inner solves, f64 refinement", "refine_steps": im["refine_steps"],
        "gmres_iters_total": im["iters"], "err_inf_vs_exact": err, "rel_l2_vs_fp64": rel,
        "launches_per_step": sum(i["launches"] for i in ims) // steps,
        "kernel_ms_per_step": tm["kernel_ms"], "kernel_launches_per_step": tm["kernel_launches"],
        "dst_hbm_f32": _dst_rates(tm, N, dim, 4)}


def _variant_2d(args, dev, stream):
    """2D 4096^2, FP64 and mixed: K solves each, device-resident."""
    import torch

    from paper_2609_16478_b300 import ahoc, inputs

    name, N = VARIANT_2D
    data = inputs.sample(inputs.config_problem(name), [N, N], backend="torch", device=dev)
    f = data["f"].reshape(-1).contiguous()
    out = {"workload": _workload_name(name, N, 2)}
    u64 = None
    for prec in ("fp64", "mixed"):
        p = ahoc.plan_for(data, device=dev, restart=300, max_iters=args.max_iters, prec=prec, stream=stream)
        u = torch.empty_like(f)
        for _ in range(args.warmup):
            p.solve(f, u, tol=args.tol)
        ms, infos = _timed_solves(p, f, u, args.steps, args)
        p.close()
        err = float((u.reshape(N + 1, N + 1) - data["u_exact"]).abs().max())
        rec = {"value": args.steps * _interior(N, 2) / (ms / 1e3), "ms_per_step": ms / args.steps,
               "err_inf_vs_exact": err, "gmres_iters": infos[-1]["iters"],
               "coarse_gmres_iters": infos[-1]["coarse_iters"], "refine_steps": infos[-1]["refine_steps"],
               "launches_per_step": infos[-1]["launches"]}
        if prec == "fp64":
            u64 = u
        else:
            rec["rel_l2_vs_fp64"] = float(torch.linalg.norm(u - u64) / torch.linalg.norm(u64))
            rec["err_ratio_vs_fp64"] = err / max(out["fp64"]["err_inf_vs_exact"], 1e-300)
        out[prec] = rec
        torch.cuda.empty_cache()
    del data, f, u64
    torch.cuda.empty_cache()
    return out


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2609_16478_b300 import ahoc, inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    name = args.workload
    prob = inputs.config_problem(name)
    dim = prob.dim
    N = [int(v) for v in args.shape.split("x")] if args.shape else [args.n] * dim
    data = inputs.sample(prob, N, backend="torch", device=dev)
    data.pop("v_exact", None)
    # the plans' own stream: GMRES iterations are replayed as CUDA graphs (not
    # possible on the legacy default stream); kernel timing uses separate,
    # event-timed plans, so that the timed solves run exactly as a user's
    solve_stream = torch.cuda.Stream(device=dev)
    plan = ahoc.plan_for(data, device=dev, restart=args.restart, max_iters=args.max_iters,
                         levels=args.levels, stream=solve_stream, prec=args.prec)
    f = data["f"].reshape(-1).contiguous()
    u = torch.empty_like(f)
    dof = _interior(N, dim)

    for _ in range(args.warmup):
        _, info = plan.solve(f, u, tol=args.tol)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.cuda.synchronize()
            host_barrier(world, args.barrier_timeout)

    # device-resident timed region: inputs in HBM, exactly `steps` solves
    with ClockSampler(local) as clk:
        barrier()
        ms, infos = _timed_solves(plan, f, u, args.steps, args)
        barrier()
    clocks = clk.summary()
    err = float((u.reshape(data["u_exact"].shape) - data["u_exact"]).abs().max())

    # end to end through the C ABI with host buffers (ahoc_solve_host: pinned f
    # in, u out, the copies inside the timed region)
    f_host = f.cpu().pin_memory()
    u_host = torch.empty(f.numel(), dtype=torch.float64).pin_memory()
    e2e_steps = min(args.steps, args.e2e_steps)
    plan.solve_host(f_host, u_host, tol=args.tol)  # first call allocates the staging grids
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.solve_host(f_host, u_host, tol=args.tol)
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_err = float((u_host.reshape(data["u_exact"].shape) - data["u_exact"].cpu()).abs().max())
    plan.close()
    del plan, f_host, u_host
    torch.cuda.empty_cache()

    ms, e2e_ms = max_over_ranks([ms, 1e3 * e2e_s * args.steps / e2e_steps], world, dev)
    if rank != 0:
        return

    # kernel breakdown: one solve on an event-timed plan
    ti = _kernel_pass(data, dev, solve_stream, args.prec, args)
    value = whole_job_rate(world, args.steps, dof, ms)
    e2e_value = whole_job_rate(world, args.steps, dof, e2e_ms)
    launches = sum(i["launches"] for i in infos)
    kms, kn = ti["kernel_ms"], ti["kernel_launches"]
    kms_top, kn_top = ti["kernel_ms_top"], ti["kernel_launches_top"]
    # the roofline is taken on the finest grid's dominant DST class (coarse levels have other N)
    dk = max(("dst_x", "dst_y"), key=lambda k: kms_top[k])
    avg_ms = kms_top[dk] / max(1, kn_top[dk])
    ax = 0 if dk == "dst_x" else 1
    Nl = N[ax]                                      # line length along the transform axis
    lines = _interior(N, dim) // (Nl - 1)
    flops = dst_flops_per_line(Nl) * lines         # one launch transforms every line of the field along one axis
    achieved = flops / (avg_ms / 1e3) / 1e12
    peak = FP64_PEAK_TFLOPS_DERIVED
    roof = {"kernel": "k_%s<double> (DST-I along %s, FP64)" % (dk, dk[-1]), "bound": "alu", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": "derived, of the FP64 pipe: 148 SMs x 2 FP64 FMA lanes per clock (ncu's FP64 pipe "
                           "peak) x 2 flop x 2.032 GHz; MEASURED_PEAKS.json has no FP64 figure",
            "traffic": PROFILED_TRAFFIC.get((name, tuple(N), dk)), "avg_launch_ms": avg_ms, "launches": kn_top[dk],
            "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": 16 * Nl * lines,
            "hbm_achieved_GBs": 16 * Nl * lines / (avg_ms / 1e3) / 1e9, "hbm_peak_GBs": _peaks().get("hbm_gbs"),
            "share_of_step": kms[dk] / sum(kms.values()),
            "top_kernel_class_by_time": max(kms, key=lambda k: kms[k]),
            "flop_count": "algorithmic flops of the N/2-point complex FFT with DST-I pre- and post-processing "
                          "(complex product = 6 flops), independent of the kernel's FMA fusion"}
    variants = {}
    if not args.no_mixed and args.prec == "fp64":
        variants["mixed"] = _mixed_variant(data, dev, solve_stream, args, u)
        # a DOF/s figure counts at an error within 1.05x of the FP64 path's
        variants["mixed"]["err_ratio_vs_fp64"] = variants["mixed"]["err_inf_vs_exact"] / max(err, 1e-300)
    del data, f, u
    torch.cuda.empty_cache()
    if not args.no_2d:
        variants["2d_4096"] = _variant_2d(args, dev, solve_stream)
    if not args.no_serve and world == 1:
        variants["serving"] = serving_variant(args, dev)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        reps, tot, t_asm, t_lu = 0, 0.0, 0.0, 0.0
        while reps < 1 or (tot < 10.0 and reps < 5):  # about 10-30 s of CPU work
            v, dt, _, ta, tl = cpu_oracle_sample(name, args.cpu_n)
            reps += 1
            tot += dt
            t_asm += ta
            t_lu += tl
        v = reps * (args.cpu_n - 1) ** dim / tot
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d direct solves (assembly + SuperLU) of the same workload at N=%d, %.1f s in all; "
                         "single-threaded, %d host cores visible" % (reps, args.cpu_n, tot, _cores()),
               "split_s": {"assembly": t_asm, "superlu": t_lu}}
    f_numel = 1
    for n in N:
        f_numel *= n + 1
    nbytes = 8 * f_numel
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "f32 inner solves, f64 refinement",
        "data": "synthetic",
        "config": {"workload": _workload_name(name, N, dim) + ", %s, GMRES tol %g"
                               % ("FP64" if args.prec == "fp64" else "mixed FP32/FP64", args.tol),
                   "dim": dim, "N": N[0] if len(set(N)) == 1 else N, "dof_per_solve": dof, "tol": args.tol,
                   "gmres_iters": infos[-1]["iters"], "coarse_levels": infos[-1]["levels"],
                   "coarse_gmres_iters": infos[-1]["coarse_iters"], "err_inf_vs_exact": err,
                   "rel_resid": infos[-1]["rel_resid"], "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (one FP64 field of this grid is %.2f GB); no flush"
                         % (8 * f_numel / 1e9),
                   "cuda_graphs": "GMRES iterations replayed as CUDA graphs on the plan's own stream",
                   "kernel_timing": "kernel_ms_per_step and roofline from one more solve on a plan with every "
                                    "launch bracketed by CUDA events (plain launches)"},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "steps": e2e_steps, "err_inf_vs_exact": e2e_err,
                "how": "ahoc_solve_host through the C ABI: f from pinned host memory to the device, the solve, "
                       "u back to pinned host memory, host clock around each call"},
        "gpu_launches": launches,
        "kernel_ms_per_step": kms,
        "kernel_ms_per_step_finest_level": kms_top,
        "kernel_launches_per_step": kn,
        "roofline": roof,
        "dst_hbm_" + ("f64" if args.prec == "fp64" else "f32"): _dst_rates(ti, N, dim, 8 if args.prec == "fp64" else 4),
        "cpu_baseline": cpu,
        "variants": variants,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=HEADLINE[0])
    ap.add_argument("--n", type=int, default=HEADLINE[1])
    ap.add_argument("--shape", default=None, help="grid as N0xN1[xN2] (profiling cases); overrides --n")
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--prec", choices=["fp64", "mixed"], default="fp64", help="precision of the headline solves")
    ap.add_argument("--restart", type=int, default=100)
    ap.add_argument("--max-iters", type=int, default=2000)
    ap.add_argument("--cpu-n", type=int, default=20, help="grid of the oracle's timing sample")
    ap.add_argument("--levels", type=int, default=-1, help="coarse levels of the nested initial guess (-1 auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision variant")
    ap.add_argument("--mixed-steps", type=int, default=3, help="timed solves of the mixed variant")
    ap.add_argument("--mixed-warmup", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=3, help="timed solves through ahoc_solve_host (at most --steps)")
    ap.add_argument("--no-2d", action="store_true", help="skip the 2D 4096^2 variant")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving workload")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-tol", type=float, default=1e-12)
    ap.add_argument("--serve-slots", type=int, default=24, help="plans per shape in the serving pool")
    ap.add_argument("--suite", choices=["bench", "paper", "serving"], default="bench",
                    help="paper: the paper's printed workloads at their largest sizes, one JSON line each; "
                         "serving: the serving workload alone")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache (default: the shipped B300 choices)")
    ap.add_argument("--barrier-timeout", type=float, default=600.0,
                    help="seconds a rank waits at a host barrier for the others before it raises (N > 1)")
    ap.add_argument("--dst-radix", type=int, default=0, choices=[0, 4, 8],
                    help="FFT radix of the line DSTs for every shape and precision (0: built-in)")
    ap.add_argument("--dst-cta", type=int, default=0, choices=[0, 128, 256, 512, 1024],
                    help="CTA size of the line DSTs for every shape and precision (0: built-in)")
    args = ap.parse_args()
    if args.dst_radix or args.dst_cta:
        from paper_2609_16478_b300 import ahoc
        for dim in (2, 3):
            for lg in range(3, 13):
                for prec in (ahoc.AHOC_FP64, ahoc.AHOC_MIXED):
                    if args.dst_radix:
                        ahoc._check(ahoc.lib().ahoc_tune_set(ahoc.AHOC_TUNE_DST_RADIX, dim, 1 << lg, prec,
                                                             args.dst_radix), "ahoc_tune_set")
                    if args.dst_cta:
                        ahoc._check(ahoc.lib().ahoc_tune_set(ahoc.AHOC_TUNE_DST_THREADS, dim, 1 << lg, prec,
                                                             args.dst_cta), "ahoc_tune_set")
    if args.tune_cache is None:
        from paper_2609_16478_b300 import autotune
        args.tune_cache = autotune.SHIPPED_MIXED
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.suite == "paper":
        import torch
        torch.cuda.set_device(local)
        paper_suite(args, torch.device("cuda", local))
        return
    if args.suite == "serving":
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"suite": "serving", **serving_variant(args, torch.device("cuda", local))}), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        global _HOST_GROUP
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        _HOST_GROUP = dist.new_group(backend="gloo")
    run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
