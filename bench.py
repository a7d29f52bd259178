"""Benchmark: biharmonic DOF/s to a fixed error on one or more B300s.

A step is one whole solve (Algorithm 1: Schur right-hand side, GMRES on the
Schur system to relative residual 1e-12, recovery of V and U) of the 2D
variable-coefficient clamped problem on a 4096 x 4096 grid (coefficient
1 + 0.4 * 8 seeded Fourier modes, u = sin^2(pi x) sin^2(pi y) cos(pi x)),
FP64 throughout.  DOF = interior unknowns (N-1)^2 per solve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs (torchrun) solve independent replicas, one per rank (the
solve does not shard on this pool: every box has one GPU); value is the sum
over ranks.  The reference arm times the CPU oracle (assembled coupled
system + SuperLU) on a bounded sample of the same workload.
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
FP64_PEAK_TFLOPS = 1.25     # nominal dense FP64 rate of a B300 (no FP64 tensor path is used)


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


def whole_job_rate(world: int, steps: int, units_per_step: float, ms: float) -> float:
    """Units all ranks processed per second: each rank runs `steps` steps of
    `units_per_step` units, the job takes the slowest rank's `ms`."""
    return world * steps * units_per_step / (ms / 1e3)


_SAMPLES = {}


def cpu_oracle_sample(N_cpu: int):
    """Time the CPU oracle (assembly + SuperLU) on the 2D Fourier-coefficient workload at N_cpu; returns (DOF/s, seconds, err).

    The synthetic inputs are generated once, outside the timed region."""
    import numpy as np

    from oracle import coupled
    from paper_2609_16478_b300 import inputs

    if N_cpu not in _SAMPLES:
        _SAMPLES[N_cpu] = inputs.sample(inputs.config_problem("fourier2d"), [N_cpu, N_cpu])
    d = _SAMPLES[N_cpu]
    t0 = time.perf_counter()
    sol = coupled.solve_direct(coupled.assemble(d), d)
    dt = time.perf_counter() - t0
    err = float(np.max(np.abs(sol.U - d["u_exact"])))
    return (N_cpu - 1) ** 2 / dt, dt, err


def run_reference(args, rank, world):
    """The oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    N_cpu = args.cpu_n
    for _ in range(args.warmup):
        cpu_oracle_sample(N_cpu)
    t0 = time.perf_counter()
    errs = []
    for _ in range(args.steps):
        _, _, e = cpu_oracle_sample(N_cpu)
        errs.append(e)
    dt = time.perf_counter() - t0
    value = args.steps * (N_cpu - 1) ** 2 / dt
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "2D variable-coefficient clamped biharmonic (Fourier coefficient, 8 modes), oracle sample N=%d" % N_cpu,
                   "dim": 2, "N": N_cpu, "err_inf_vs_exact": max(errs)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "direct solve of the assembled coupled system at N=%d per step "
                                   "(SuperLU, single-threaded; %d host cores visible)" % (N_cpu, cores)},
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
    dimension, size, coefficient and right-hand side, at 80% of the measured
    sequential mixed-path capacity; the batched mixed-precision server
    against one-at-a-time plain FP64 solves of the same stream."""
    import numpy as np
    import torch

    from paper_2609_16478_b300 import ahoc, autotune, inputs, serving

    tol = args.serve_tol
    p3 = 0.3
    mix = {(2, n): (1 - p3) / len(inputs.SERVE_2D) for n in inputs.SERVE_2D}
    mix.update({(3, n): p3 / len(inputs.SERVE_3D) for n in inputs.SERVE_3D})
    # sequential capacity of the mixed path, one warm solve per shape
    t_seq = {}
    for (dim, n) in mix:
        d = inputs.sample_request(inputs.RequestSpec(10 ** 6, dim, n, (1,) * dim, 0.0), device=dev)
        p = ahoc.Plan(dim, [n] * dim, d["alpha"], prec="mixed", restart=60, max_iters=2000)
        p.solve(d["f"], tol=tol)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.solve(d["f"], tol=tol)
        t_seq[(dim, n)] = time.perf_counter() - t0
        p.close()
    cap = 1.0 / sum(mix[k] * t_seq[k] for k in mix)
    rate = 0.8 * cap
    specs = inputs.request_stream(args.serve_requests, rate, seed=5)

    def warm_specs(batch_for, size, rid0):
        # `size` requests of every shape at once (at most the shape's batch):
        # the pool then holds a plan of that size per shape
        out, rid = [], rid0
        for (dim, n) in mix:
            for _ in range(min(size, batch_for((dim, n)))):
                out.append(inputs.RequestSpec(rid, dim, n, (0,) * dim, 0.0))
                rid += 1
        return out

    def arm(prec, workers, batch_for):
        srv = serving.Server(device=dev, prec=prec, tol=tol, workers=workers, batch_for=batch_for,
                             check_exact=True)
        srv.sched.max_slots = args.serve_slots
        size = 1
        while size <= max(batch_for(k) for k in mix):  # plans of every power-of-two size resident
            srv.run(warm_specs(batch_for, size, 10 ** 7 + 1000 * size), realtime=False)
            size *= 2
        recs = srv.run(specs, realtime=True)
        srv.close()
        torch.cuda.empty_cache()
        return recs, serving.summarize(recs)

    # the mixed server takes the tuner's batch sizes and launch shapes
    cache = autotune.load(args.tune_cache)
    autotune.apply(cache)
    ra, sa = arm("mixed", args.serve_workers, autotune.batch_for(cache, "mixed", serving.default_batch))
    for k in cache:  # the FP64 arm runs with the built-in shapes
        dim, n, _ = k.split(":")
        for kind in (ahoc.AHOC_TUNE_TRI_CHUNK, ahoc.AHOC_TUNE_DST_THREADS):
            ahoc.lib().ahoc_tune_set(kind, int(dim), int(n), ahoc.AHOC_MIXED, 0)
    rb, sb = arm("fp64", 1, lambda k: 1)
    ea = {r.rid: r.err_inf for r in ra}
    eb = {r.rid: r.err_inf for r in rb}
    ratio = max(ea[i] / eb[i] for i in ea if eb[i] > 0)
    return {
        "workload": "%d requests, Poisson arrivals (seed 5) at %.1f req/s = 80%% of the sequential mixed-path "
                    "capacity %.1f req/s; 2D N in %s (p=0.7), 3D N in %s; per-request Fourier coefficient "
                    "(M=6, K=4, A=0.5, seed = request id) and u = prod sin^2(pi x) cos(m pi x), m in 0..4; "
                    "Schur tol %g" % (len(specs), rate, cap, list(inputs.SERVE_2D), list(inputs.SERVE_3D), tol),
        "batched_mixed": dict(sa, workers=args.serve_workers, plan_slots_per_shape=args.serve_slots,
                              batch="per shape from the autotuner: %s" % {k: v["batch"] for k, v in cache.items()}),
        "sequential_fp64": dict(sb, workers=1, batch=1),
        "p99_speedup": sb["p99_ms"] / sa["p99_ms"], "dof_per_s_ratio": sa["dof_per_s"] / sb["dof_per_s"],
        "max_err_ratio_mixed_over_fp64": ratio,
        "max_err_inf": max(max(ea.values()), max(eb.values())),
        "seq_mixed_ms_per_shape": {"%dD N=%d" % k: 1e3 * v for k, v in t_seq.items()},
    }


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2609_16478_b300 import ahoc, inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    N = args.n
    dim = 2
    prob = inputs.config_problem("fourier2d")
    data = inputs.sample(prob, [N, N], backend="torch", device=dev)
    # the plan's own stream: GMRES iterations are replayed as CUDA graphs (not
    # possible on the legacy default stream); kernel timing uses a second,
    # event-timed plan below, so that the timed solves run exactly as a user's
    solve_stream = torch.cuda.Stream(device=dev)
    plan = ahoc.plan_for(data, device=dev, restart=args.restart, max_iters=args.max_iters,
                         levels=args.levels, stream=solve_stream)
    f = data["f"].reshape(-1).contiguous()
    u = torch.empty_like(f)
    st = plan.stream
    dof = (N - 1) ** dim

    for _ in range(args.warmup):
        _, info = plan.solve(f, u, tol=args.tol)
    torch.cuda.synchronize()
    err = float((u.reshape(N + 1, N + 1) - data["u_exact"]).abs().max())

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # device-resident timed region
    infos = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            _, info = plan.solve(f, u, tol=args.tol)
            infos.append(info)
        e1.record(st)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    clocks = clk.summary()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    f_host = f.cpu().pin_memory()
    u_host = torch.empty(f.numel(), dtype=torch.float64).pin_memory()
    f_dev = torch.empty_like(f)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(st):
            f_dev.copy_(f_host, non_blocking=True)
        plan.solve(f_dev, u, tol=args.tol)
        with torch.cuda.stream(st):
            u_host.copy_(u, non_blocking=True)
        st.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()

    # kernel breakdown: the same solves on an event-timed plan (every launch
    # bracketed by CUDA events on the plan's stream, plain launches)
    plan_t = ahoc.plan_for(data, device=dev, timing=True, restart=args.restart, max_iters=args.max_iters,
                           levels=args.levels, stream=solve_stream)
    u_t = torch.empty_like(f)
    plan_t.solve(f, u_t, tol=args.tol)
    tinfos = []
    for _ in range(args.steps):
        _, ti = plan_t.solve(f, u_t, tol=args.tol)
        tinfos.append(ti)
    plan_t.close()

    ms, e2e_ms = max_over_ranks([ms, e2e_s * 1e3], world, dev)
    if rank != 0:
        return

    value = whole_job_rate(world, args.steps, dof, ms)
    e2e_value = whole_job_rate(world, args.steps, dof, e2e_ms)
    launches = sum(i["launches"] for i in infos)
    kms = {k: sum(i["kernel_ms"][k] for i in tinfos) for k in ahoc.KERNEL_NAMES}
    kn = {k: sum(i["kernel_launches"][k] for i in tinfos) for k in ahoc.KERNEL_NAMES}
    top = max(kms, key=lambda k: kms[k])
    # the roofline uses the N = 4096 grid's own launches (coarse levels have other N)
    kms_top = {k: sum(i["kernel_ms_top"][k] for i in tinfos) for k in ahoc.KERNEL_NAMES}
    kn_top = {k: sum(i["kernel_launches_top"][k] for i in tinfos) for k in ahoc.KERNEL_NAMES}
    avg_ms = kms_top["dst_x"] / max(1, kn_top["dst_x"])
    flops = dst_flops_per_line(N) * (N - 1)          # one launch transforms N-1 lines of N
    achieved = flops / (avg_ms / 1e3) / 1e12
    roof = {"kernel": "k_dst_x<double> (DST-I along x, FP64)", "bound": "alu", "achieved": achieved,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
            "peak_source": "nominal B300 FP64 rate (no measured FP64 peak in MEASURED_PEAKS.json)",
            # DRAM bytes per launch of k_dst_x<double,1,0> (forward transform with the fused M load, the
            # kernel's most frequent form in GMRES) from the ncu capture summarised in
            # profiles/k_dst_x_fp64_2d4096.md: 134.5 MB read + 94.5 MB written
            "traffic": 229.0e6, "avg_launch_ms": avg_ms, "launches": kn_top["dst_x"],
            "algorithmic_bytes_per_launch": 16 * N * (N - 1), "flops_per_launch": flops,
            "hbm_achieved_GBs": 16 * N * (N - 1) / (avg_ms / 1e3) / 1e9,
            "hbm_peak_GBs": _peaks().get("hbm_gbs"),
            "share_of_step": kms["dst_x"] / sum(kms.values()), "top_kernel_by_time": top,
            "fp64_instr_note": "FP64 pipe 90-92% busy under ncu (profiles/); the FFT's additions cannot all be "
                               "FMAs, so flops per FP64 operation stay below 2",
            "fp64_probe_ops_per_s": 0.463e12}
    # the same workload through the mixed-precision path (FP32 inner solves, FP64 refinement)
    variants = {}
    if not args.no_mixed:
        pm = ahoc.plan_for(data, device=dev, restart=args.restart, max_iters=args.max_iters,
                           prec="mixed", stream=solve_stream)
        um = torch.empty_like(f)
        for _ in range(args.warmup):
            pm.solve(f, um, tol=args.tol)
        torch.cuda.synchronize()
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        m0.record(pm.stream)
        ims = []
        for _ in range(args.steps):
            _, im = pm.solve(f, um, tol=args.tol)
            ims.append(im)
        m1.record(pm.stream)
        torch.cuda.synchronize()
        mms = m0.elapsed_time(m1)
        pm_t = ahoc.plan_for(data, device=dev, timing=True, restart=args.restart, max_iters=args.max_iters,
                             prec="mixed", stream=solve_stream)
        pm_t.solve(f, um, tol=args.tol)
        _, tm = pm_t.solve(f, um, tol=args.tol)
        pm_t.close()
        variants["mixed"] = {
            "value": args.steps * dof / (mms / 1e3), "unit": UNIT, "ms_per_step": mms / args.steps,
            "dtype": "f32 inner solves, f64 refinement", "refine_steps": im["refine_steps"],
            "gmres_iters_total": im["iters"],
            "err_inf_vs_exact": float((um.reshape(N + 1, N + 1) - data["u_exact"]).abs().max()),
            "rel_l2_vs_fp64": float(torch.linalg.norm(um - u) / torch.linalg.norm(u)),
            "launches_per_step": sum(i["launches"] for i in ims) // args.steps,
            "kernel_ms_per_step": tm["kernel_ms"], "kernel_launches_per_step": tm["kernel_launches"]}
        pm.close()
    if not args.no_serve and world == 1:
        del plan
        torch.cuda.empty_cache()
        variants["serving"] = serving_variant(args, dev)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, dt, _ = cpu_oracle_sample(args.cpu_n)
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "direct solve (assembly + SuperLU) of the same workload at N=%d, %.1f s; "
                         "single-threaded, %d host cores visible" % (args.cpu_n, dt, cores)}
    nbytes = f.numel() * 8
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "2D variable-coefficient clamped biharmonic (Fourier coefficient, 8 modes) N=%d, FP64, GMRES tol %g"
                               % (N, args.tol),
                   "dim": dim, "N": N, "dof_per_solve": dof, "tol": args.tol,
                   "gmres_iters": infos[-1]["iters"], "coarse_levels": infos[-1]["levels"],
                   "coarse_gmres_iters": infos[-1]["coarse_iters"], "err_inf_vs_exact": err,
                   "rel_resid": infos[-1]["rel_resid"], "parallelism": "replicas" if world > 1 else "single",
                   "l2": "working set (two 134 MB fields + coefficient/data arrays) larger than L2; no flush",
                   "cuda_graphs": "GMRES iterations replayed as CUDA graphs on the plan's own stream",
                   "kernel_timing": "kernel_ms_per_step and roofline from a second pass of the same solves with "
                                    "every launch bracketed by CUDA events (plain launches)"},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "kernel_ms_per_step": {k: v / args.steps for k, v in kms.items()},
        "kernel_ms_per_step_finest_level": {k: v / args.steps for k, v in kms_top.items()},
        "roofline": roof,
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
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--restart", type=int, default=300)
    ap.add_argument("--max-iters", type=int, default=2000)
    ap.add_argument("--cpu-n", type=int, default=256)
    ap.add_argument("--levels", type=int, default=-1, help="coarse levels of the nested initial guess (-1 auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision variant")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving workload")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-tol", type=float, default=1e-12)
    ap.add_argument("--serve-slots", type=int, default=8, help="plans per shape in the serving pool")
    ap.add_argument("--suite", choices=["bench", "paper"], default="bench",
                    help="paper: the paper's printed workloads at their largest sizes, one JSON line each")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache (default: the shipped B300 choices)")
    args = ap.parse_args()
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
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
