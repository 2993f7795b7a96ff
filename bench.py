"""Benchmark: KSVD-preconditioned matrix-free GMRES for 2D DG advection on GB300.

One step = one pass of the whole hot path over the 64 x 64 workload: the
Kronecker-SVD factor build of every element (Alg. 2d-form) followed by a
restarted right-preconditioned GMRES(30) solve of (M + dt A) x = b to a
1e-8 relative residual (Kronecker apply, sum-factorised operator, CGS2
Arnoldi).  The flux-Jacobian precomputation runs once per context, as in
Alg. matrix-free-matvec.

Default: one GPU, n = 16 (p = 15), 64 x 64 periodic unit-square quads,
divergence-free random-Fourier velocity (seed 1705), dt = 0.05, b ~ N(0, 1)
(seed 1706).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 16|31] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import ctypes
import contextlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "GMRES time to 1e-8 rel. residual (factor build + solve), 1 GB300"
FP64_PEAK_NOTE = ("FP64 peak = 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz = 1258.6 GFLOP/s "
                  "(FP64 pipe unit count and max clock; 1.19 TFLOP/s measured by a DFMA loop)")
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
# DRAM bytes (read + write) of one FP64 one-sided apply launch at n = 16 on the 64 x 64 mesh,
# from one ncu capture of the current kernel (dram__bytes_read.sum + dram__bytes_write.sum)
TRAFFIC_APPLY_FP64_N16 = 305.2e6 + 3.39e6


def bf16_peak_tflops():
    """Dense BF16 tensor peak for a kernel timed alone: the measured burst figure of
    MEASURED_PEAKS.json when present, else the machine's fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (MEASURED_PEAKS.json, burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s (no MEASURED_PEAKS.json)"


def workload(n: int, h: float = 1.0, solenoidal: bool = True):
    return dict(dim=2, n=n, nel=(64, 64), h=h, dt=0.05,
                velocity=synthetic.fourier_velocity(1705, 2, solenoidal=solenoidal),
                rhs_seed=1706)


def workload_3d(n: int = 11):
    return dict(dim=3, n=n, nel=(16, 16, 16), h=1.0, dt=0.05,
                velocity=synthetic.fourier_velocity(1707, 3), rhs_seed=1708)


def time_each(fn, reps, stream, flush):
    """Mean device time (ms) of fn() over reps launches, with the L2 flushed
    (a write of a buffer larger than L2) before each one, outside the events."""
    import torch
    tot = 0.0
    for _ in range(reps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / reps


def form_bits(args) -> int:
    from paper_1704_04549_gb300 import TPP_FEAT_TWO_SIDED
    return TPP_FEAT_TWO_SIDED if args.form == "two-sided" else 0


def max_over_ranks(value: float, device) -> float:
    """The largest value over the ranks of the default process group (the slowest
    replica's time); the value itself when the run is not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_oracle(n: int, gmres_iters: int, budget_s: float = 20.0):
    """The oracle, as it stands, on a bounded sample of the same workload.

    Sample: the first k elements of the 64 x 64 mesh.  Per element the oracle
    assembles the exact block, takes the dense SVD of its rearrangement,
    LU-factors P (the factor build) and then, per GMRES iteration, applies
    P^-1 (LU solve) and one block row of the assembled operator; the MGS
    Arnoldi work on full-length vectors is timed on vectors of the full size
    for the average basis length.  Extrapolated linearly to 4096 elements
    and to the GPU run's iteration count."""
    import scipy.linalg as sla

    from oracle.dg import AdvectionDG, PeriodicMesh
    from oracle.ksvd import ksvd_2d, kron_sum
    w = workload(n)
    dg = AdvectionDG(PeriodicMesh(w["nel"], w["h"]), n, w["dt"], w["velocity"])
    nl, E = dg.nloc, dg.mesh.num_elem
    rng = np.random.default_rng(0)
    t_build, t_iter, k = 0.0, 0.0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s and k < E:
        e = k
        tb = time.perf_counter()
        S = dg.element_block(e)
        _, As, Bs = ksvd_2d(S, n)
        lu = sla.lu_factor(kron_sum(As, Bs))
        t_build += time.perf_counter() - tb
        Fd, nbrs = dg.face_blocks(e)
        v = rng.standard_normal(nl)
        ti = time.perf_counter()
        z = sla.lu_solve(lu, v)
        y = S @ z
        for _, (nb, F) in nbrs.items():
            y += dg.dt * F @ z
        t_iter += time.perf_counter() - ti
        k += 1
    N = dg.ndof
    V = rng.standard_normal((16, N))
    wv = rng.standard_normal(N)
    ta = time.perf_counter()
    for i in range(16):                         # MGS at the average basis length
        h = np.dot(V[i], wv)
        wv -= h * V[i]
    t_arnoldi = time.perf_counter() - ta
    total_s = (t_build / k) * E + gmres_iters * ((t_iter / k) * E + t_arnoldi)
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count()
    return {"value": total_s * 1e3, "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": (f"{k} of {E} elements (exact block, dense SVD of the rearrangement, LU of P; "
                       f"per iteration LU solve + block-row matvec) and full-length MGS at basis "
                       f"length 16, extrapolated to {E} elements x {gmres_iters} iterations"),
            "sample_seconds": round(time.perf_counter() - t0, 2)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    iters = args.ref_iters
    vals = []
    for _ in range(args.warmup):
        cpu_baseline_oracle(args.n, iters, budget_s=2.0)
    t0 = time.time()
    last = None
    for _ in range(args.steps):
        last = cpu_baseline_oracle(args.n, iters, budget_s=args.ref_budget)
        vals.append(last["value"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"adv2d-fourier-64x64-n{args.n}", "n": args.n,
                       "nel": [64, 64], "h": 1.0, "dt": 0.05, "rtol": 1e-8, "restart": 30},
            "cpu_baseline": {**last, "value": value},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": round(time.time() - t0, 1)}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if torch.cuda.is_available() else 0)
    torch.cuda.set_device(dev)
    from paper_1704_04549_gb300 import TPP_FEAT_MIXED, TPP_FP32, TPP_FP64, TPP_PC_KRON, Context
    from paper_1704_04549_gb300 import _lib

    lib = _lib.load()
    w = workload(args.n, 1.0 / 64 if args.h_reading == "domain" else 1.0,
                 args.field == "solenoidal")
    ctx = Context(2, args.n, w["nel"], w["h"], w["dt"], w["velocity"], max_restart=30,
                  features=TPP_FEAT_MIXED | form_bits(args), device=str(dev))
    # the mixed-precision solver on its own context whose shifted inverses are formed in
    # FP32 only (the FP32 apply is all it needs; one-sided form, n <= 16)
    f32s = args.form == "one-sided" and args.n <= 16
    ctx32 = Context(2, args.n, w["nel"], w["h"], w["dt"], w["velocity"], max_restart=30,
                    features=TPP_FEAT_MIXED | _lib.TPP_FEAT_F32_SHIFTS, device=str(dev)) \
        if f32s else ctx
    N, E, n = ctx.num_dofs, ctx.num_elem, args.n
    b_host = synthetic.rhs(w["rhs_seed"], N)
    b = torch.as_tensor(b_host, device=dev)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream(dev)
    inner = TPP_FP32 if args.prec == "mixed" else TPP_FP64

    kin = args.inner if inner != TPP_FP64 else 0

    def step(prec=inner, k_in=kin, rtol=1e-8):
        cx = ctx if prec == TPP_FP64 else ctx32
        cx.tpp_build_factors()
        x.zero_()
        _, res = cx.gmres_solve(b, x, restart=30, rtol=rtol, max_iters=args.max_iters,
                                pc=TPP_PC_KRON, inner_prec=prec, flexible=(prec != TPP_FP64),
                                check=False, inner_iters=k_in, use_graph=args.graph)
        return res

    for _ in range(args.warmup):
        res = step()
    # timed region: K full steps, barrier + synchronize on both sides
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = lib.tpp_kernel_launch_count()
    with ClockSampler(local) as clk:
        e0.record(stream)
        results = [step() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
    launches = lib.tpp_kernel_launch_count() - l0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    res = results[-1]
    converged = all(r["converged"] for r in results)

    # the other precision mode on the same workload and clock rules (FP64 <-> mixed)
    o_prec = TPP_FP64 if inner != TPP_FP64 else TPP_FP32
    o_kin = args.inner if o_prec != TPP_FP64 else 0
    for _ in range(args.warmup):
        step(o_prec, o_kin)
    torch.cuda.synchronize(dev)
    o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    o0.record(stream)
    o_res = [step(o_prec, o_kin) for _ in range(args.steps)]
    o1.record(stream)
    torch.cuda.synchronize(dev)
    cxo = ctx if o_prec == TPP_FP64 else ctx32
    torch.cuda.synchronize(dev)
    ob0, ob1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ob0.record(stream)
    cxo.tpp_build_factors()
    ob1.record(stream)
    torch.cuda.synchronize(dev)
    other = {"mode": "fp64" if o_prec == TPP_FP64 else "mixed", "inner_iters_per_outer": o_kin,
             "build_ms": ob0.elapsed_time(ob1),
             "f32_shift_inverses": bool(o_prec != TPP_FP64 and f32s),
             "ms_per_step": o0.elapsed_time(o1) / args.steps, "iters": o_res[-1]["iters"],
             "inner_iters": o_res[-1]["inner_iters"],
             "converged": all(r["converged"] for r in o_res),
             "true_rel_res": o_res[-1]["true_rel_res"]}
    # iteration count at the paper's tolerance 1e-5 (shape comparison; untimed)
    iters_1e5 = step(rtol=1e-5)["iters"]

    # split of one step: build vs solve (CUDA events)
    torch.cuda.synchronize(dev)
    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eb0.record(stream)
    (ctx if inner == TPP_FP64 else ctx32).tpp_build_factors()
    eb1.record(stream)
    torch.cuda.synchronize(dev)
    build_ms = eb0.elapsed_time(eb1)
    ctx.tpp_build_factors()

    # preconditioner apply throughput, FP64 and FP32 (dominant kernel), on the bench stream
    z = torch.empty_like(b)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)     # 256 MB > L2
    apply = {}
    for name, prec in (("fp64", TPP_FP64), ("fp32", TPP_FP32)):
        for _ in range(3):
            ctx.tpp_apply_inverse(b, z, prec=prec)
        t_ms = time_each(lambda: ctx.tpp_apply_inverse(b, z, prec=prec), 20, stream, flush)
        apply[name] = {"ms": t_ms, "gdofs": N / (t_ms * 1e-3) / 1e9}
    # algorithmic work of the apply: 4 dense n x n x n products (8 n^3) + the
    # quasi-triangular Sylvester solve (2 n^3) per element; bytes: b, x and the
    # six n x n factors
    flops = 10.0 * n ** 3 * E
    achieved = flops / (apply["fp64"]["ms"] * 1e-3) / 1e9
    roofline = {"kernel": "k_apply_2d_g<double,16,double>", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS,
                "traffic": (TRAFFIC_APPLY_FP64_N16 if (n == 16 and args.form == "one-sided")
                            else None),
                "traffic_unit": "bytes per launch", "peak_note": FP64_PEAK_NOTE,
                "algorithmic": "10 n^3 flop per element (8 n^3 GEMM stages + 2 n^3 Sylvester)"}

    # end to end through the public API with host buffers (pinned), copies inside
    b_pin = torch.from_numpy(b_host).pin_memory()
    x_pin = torch.empty(N, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    t_e2e = []
    for it in range(max(1, min(args.steps, 3)) + 1):
        t0 = time.perf_counter()
        bd = b_pin.to(dev, non_blocking=True)
        ce = ctx if inner == TPP_FP64 else ctx32
        ce.tpp_build_factors()
        xd = torch.zeros_like(bd)
        ce.gmres_solve(bd, xd, restart=30, rtol=1e-8, max_iters=args.max_iters, pc=TPP_PC_KRON,
                       inner_prec=inner, flexible=(inner != TPP_FP64), check=False,
                       inner_iters=kin, use_graph=args.graph)
        x_pin.copy_(xd, non_blocking=True)
        torch.cuda.synchronize(dev)
        if it > 0:
            t_e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = statistics.median(t_e2e)

    # arithmetic peaks measured live by the DFMA / FFMA chain probe
    probe = {}
    for name, prec, iters in (("fp64", TPP_FP64, 12000), ("fp32", TPP_FP32, 400000)):
        rate = ctypes.c_double(0.0)
        if lib.tpp_probe_fma_rate(prec, iters, ctypes.byref(rate),
                                  ctypes.c_void_p(stream.cuda_stream)) == 0:
            probe[name] = rate.value / 1e9
    roofline["peak_probe_gflops"] = probe
    extra = {} if args.no_extra else other_configs(args, dev)

    if rank != 0:
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_oracle(n, res["iters"], budget_s=args.cpu_budget)
    line = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if inner == TPP_FP64 else "f64+f32",
        "data": "synthetic",
        "config": {"workload": f"adv2d-fourier-64x64-n{n} (p={n - 1}), "
                               f"{'unit-square quads' if w['h'] == 1.0 else 'h=1/64'}, "
                               f"dt=0.05, {args.field} random-Fourier velocity seed 1705, "
                               f"b~N(0,1) seed 1706",
                   "n": n, "nel": [64, 64], "h": w["h"], "dt": 0.05, "dofs": N, "rtol": 1e-8,
                   "restart": 30, "preconditioner": "KSVD rank-2 (Alg. 2d-form / 2d-apply)",
                   "inner_prec": args.prec, "apply_form": args.form,
                   "cuda_graphs": bool(args.graph),
                   "solver": ("FP64 flexible GMRES(30) around inner FP32 GMRES(%d) solves "
                              "(FP32 operator + FP32 Kronecker apply)" % kin) if kin > 0 else
                             ("flexible GMRES(30), FP32 Kronecker apply" if inner != TPP_FP64
                              else "GMRES(30), FP64"),
                   "l2": "step: inputs larger than L2 (Krylov basis %.0f MB + factors %.0f MB); "
                         "precond_apply: L2 flushed (256 MB write) before each timed launch"
                         % (31 * N * 8 / 1e6, 6 * N * 8 / 1e6),
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "other_mode": other,
        "gmres": {"iters": res["iters"], "inner_iters": res["inner_iters"], "iters_at_1e-5": iters_1e5,
                  "cycles": res["cycles"], "converged": converged,
                  "true_rel_res": res["true_rel_res"], "build_ms": build_ms,
                  "solve_ms": ms - build_ms},
        "precond_apply": {"fp64_gdofs": apply["fp64"]["gdofs"], "fp64_ms": apply["fp64"]["ms"],
                          "fp32_gdofs": apply["fp32"]["gdofs"], "fp32_ms": apply["fp32"]["ms"]},
        "roofline": roofline,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": N * 8,
                "d2h_bytes_per_step": N * 8},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "other_configs": extra,
    }
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def other_configs(args, dev):
    """Compact untimed-region records of the other configurations (each measured with
    CUDA events, L2 flushed before apply launches): the 64 x 64 mesh at n = 31 and the
    16^3 hex mesh at n = 11.  Apply GDOF/s in FP64 and FP32, the factor build, and the
    mixed solver (FP64 FGMRES(30) around FP32 GMRES(12)) to 1e-8 within a step cap."""
    import torch
    from paper_1704_04549_gb300 import TPP_FEAT_MIXED, TPP_FP32, TPP_FP64, TPP_PC_KRON, Context
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    out = {}
    for key, w, cap in (("adv2d_64x64_n31", workload(31), 300), ("adv3d_16cubed_n11", workload_3d(11), 400)):
        ctx = Context(w["dim"], w["n"], w["nel"], w["h"], w["dt"], w["velocity"], max_restart=30,
                      features=TPP_FEAT_MIXED, device=str(dev))
        N = ctx.num_dofs
        b = torch.as_tensor(synthetic.rhs(w["rhs_seed"], N), device=dev)
        z = torch.empty_like(b)
        ctx.tpp_build_factors()
        build_ms = time_each(lambda: ctx.tpp_build_factors(), 3, stream, flush)
        rec = {"dofs": N, "build_ms": build_ms}
        for name, prec in (("fp64", TPP_FP64), ("fp32", TPP_FP32)):
            for _ in range(3):
                ctx.tpp_apply_inverse(b, z, prec=prec)
            t = time_each(lambda: ctx.tpp_apply_inverse(b, z, prec=prec), 10, stream, flush)
            rec[f"apply_{name}_gdofs"] = N / (t * 1e-3) / 1e9
        x = torch.zeros_like(b)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, r = ctx.gmres_solve(b, x, restart=30, rtol=1e-8, max_iters=cap, pc=TPP_PC_KRON,
                               inner_prec=TPP_FP32, flexible=True, inner_iters=args.inner,
                               check=False, use_graph=args.graph)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        rec["mixed"] = {"solve_ms": e0.elapsed_time(e1), "outer_iters": r["iters"],
                        "inner_iters": r["inner_iters"], "converged": bool(r["converged"]),
                        "true_rel_res": r["true_rel_res"], "outer_cap": cap}
        out[key] = rec
        del ctx
        torch.cuda.empty_cache()
    # the mixed-degree batch at 10 % (per-system batched GMRES, autotuned shapes)
    res, tuned, groups, dofs, _, _ = batch_measure(args, 0.1, 2, 1, sample_clocks=False)
    out["batch_10pct"] = {"dof_rhs": dofs, "groups": len(groups),
                          "fp64": {k: res["fp64"][k] for k in ("ms", "solve_ms", "launch_ms",
                                                               "iters_mean", "iters_max",
                                                               "unconverged")},
                          "mixed": {k: res["mixed"][k] for k in ("ms", "solve_ms", "launch_ms",
                                                                 "iters_mean", "iters_max",
                                                                 "unconverged", "max_outer")},
                          "shapes": {m: {k: t[k] for k in ("warps", "reg_budget")}
                                     for m, t in tuned.items()}}
    torch.cuda.empty_cache()
    out["euler_vortex_16x12_n8"] = euler_record(dev)
    out["euler3d_periodic_6cubed"] = euler3d_record(dev)
    out["curved_64x64_n16"] = curved_record(dev, flush)
    return out


def euler3d_record(dev):
    """3D Euler equations linearised around the periodic case of Sec. 5.6 (rho = 1 + 0.2
    sin(pi (x + y + z)), v = (1, -1/2, 1), p = 1 on [0, 2]^3), its 6 x 6 x 6 mesh and
    dt = 2.5e-3, n = 4 and 6 (p = 3, 5): one backward Euler system from b ~ N(0, 1),
    GMRES(30) to 1e-8 with the Kronecker (K) and exact block Jacobi (J) preconditioners on
    the small and the full blocks.  Times (CUDA events) include the preconditioner build."""
    import numpy as np
    import torch
    from paper_1704_04549_gb300 import (TPP_FEAT_BLOCK_JACOBI, TPP_FEAT_FULL_BLOCKS,
                                        TPP_PC_BLOCK_JACOBI, TPP_PC_KRON, Context)
    L, N, dt = 2.0, 6, 2.5e-3
    h = L / N
    stream = torch.cuda.current_stream(dev)
    out = {}
    for n in (4, 6):
        xg = 0.5 * (np.polynomial.legendre.leggauss(n)[0] + 1.0)
        gz, gy, gx = np.meshgrid(xg, xg, xg, indexing="ij")
        E = N ** 3
        state = np.empty((E, 5, n ** 3))
        for e in range(E):
            cx, cy, cz = e % N, (e // N) % N, e // (N * N)
            X = np.stack([(cx + gx) * h, (cy + gy) * h, (cz + gz) * h], -1).reshape(-1, 3)
            state[e] = synthetic.euler3d_wave_state(X, L).T
        rec = {"dofs": E * 5 * n ** 3}
        for blocks, extra in (("small", 0), ("full", TPP_FEAT_FULL_BLOCKS)):
            ctx = Context.euler_system(n, (N, N, N), h, dt, state,
                                       features=TPP_FEAT_BLOCK_JACOBI | extra, device=str(dev))
            b = torch.as_tensor(synthetic.rhs(1714, ctx.num_dofs), device=dev)
            for kind, pc, build in (("K", TPP_PC_KRON, ctx.tpp_build_factors),
                                    ("J", TPP_PC_BLOCK_JACOBI, ctx.tpp_build_block_jacobi)):
                build()
                x = torch.zeros_like(b)
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                build()
                _, r = ctx.gmres_solve(b, x, restart=30, rtol=1e-8, max_iters=2000, pc=pc,
                                       check=False)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                rec[f"{kind}_{blocks}"] = {"iters": r["iters"], "converged": bool(r["converged"]),
                                           "true_rel_res": r["true_rel_res"],
                                           "build_solve_ms": e0.elapsed_time(e1)}
            del ctx
            torch.cuda.empty_cache()
        out[f"n={n}"] = rec
    return out


def curved_record(dev, flush):
    """Curved elements: the 64 x 64 mesh of the 2D configuration mapped by the periodic
    warp Phi(X) = X + 0.05 L sin(2 pi X / L) sin(2 pi Y / L) (1, 1) (L = 64, h = 1), n = 16,
    field 1705, dt = 0.05: operator and FP64 apply throughput, factor build, and the FP64
    GMRES(30) solve to 1e-8 (metric terms from mesh.warped_metric_terms)."""
    import torch
    from paper_1704_04549_gb300 import TPP_FP64, TPP_PC_KRON, Context, mesh
    n, N, h = 16, 64, 1.0
    vel = synthetic.fourier_velocity(1705, 2)
    ctx = Context(2, n, (N, N), h, 0.05, vel, max_restart=30, device=str(dev))
    warp = lambda X: synthetic.periodic_warp(X, N * h, 0.05)
    jd, fl, ff = mesh.warped_metric_terms((N, N), h, ctx.gauss_legendre()[0], vel, warp)
    ctx.tpp_set_metric_terms(jd, fl, ff, 0.05)
    stream = torch.cuda.current_stream(dev)
    Nd = ctx.num_dofs
    b = torch.as_tensor(synthetic.rhs(1706, Nd), device=dev)
    z = torch.empty_like(b)
    ctx.tpp_build_factors()
    rec = {"dofs": Nd, "build_ms": time_each(lambda: ctx.tpp_build_factors(), 3, stream, flush)}
    for _ in range(3):
        ctx.dg_apply_sumfact(b, z)
        ctx.tpp_apply_inverse(b, z, prec=TPP_FP64)
    rec["operator_gdofs"] = Nd / (time_each(lambda: ctx.dg_apply_sumfact(b, z), 10, stream,
                                            flush) * 1e-3) / 1e9
    rec["apply_fp64_gdofs"] = Nd / (time_each(lambda: ctx.tpp_apply_inverse(b, z, prec=TPP_FP64),
                                              10, stream, flush) * 1e-3) / 1e9
    x = torch.zeros_like(b)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, r = ctx.gmres_solve(b, x, restart=30, rtol=1e-8, max_iters=1000, pc=TPP_PC_KRON,
                           check=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    rec["gmres"] = {"solve_ms": e0.elapsed_time(e1), "iters": r["iters"],
                    "converged": bool(r["converged"]), "true_rel_res": r["true_rel_res"]}
    del ctx
    torch.cuda.empty_cache()
    return rec


def run_euler(args):
    """The Euler vortex systems (euler_record) as their own JSON line: value = factor build +
    GMRES solve of the dt = 0.1 system with the small-block Kronecker preconditioner."""
    import torch
    dev = torch.device("cuda:0")
    with ClockSampler(0) as clk:
        rec = euler_record(dev)
        rec["3d_periodic_6cubed"] = euler3d_record(dev)
    line = {"metric": "2D Euler vortex, linearised LLF system: build + GMRES(30) to 1e-8 with "
                      "the small-block Kronecker preconditioner, 1 GB300",
            "value": rec["dt=0.1"]["K_small"]["build_solve_ms"], "unit": "ms", "n_gpus": 1,
            "steps": 1, "warmup": 1, "higher_is_better": False, "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "16 x 12 periodic mesh of the 20 x 15 domain, n = 8, vortex "
                                   "of Sec. 5.3 at t = 0, dt = 0.1 and 0.01; 3D periodic case "
                                   "of Sec. 5.6 on 6 x 6 x 6, n = 4 and 6, dt = 2.5e-3"},
            "records": rec, "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def euler_record(dev):
    """2D Euler equations linearised around the vortex of Sec. 5.3 at t = 0: 16 x 12
    periodic mesh of the 20 x 15 domain (h = 1.25), n = 8 (p = 7), one backward Euler
    system per dt; GMRES(30) to 1e-8 with the Kronecker (K) and exact block Jacobi (J)
    preconditioners on the small (per-component) blocks and on the full n_c n^2 blocks.
    Times with CUDA events."""
    import numpy as np
    import torch
    from paper_1704_04549_gb300 import (TPP_FEAT_BLOCK_JACOBI, TPP_FEAT_FULL_BLOCKS,
                                        TPP_PC_BLOCK_JACOBI, TPP_PC_KRON, Context)
    nel, h, n = (16, 12), 1.25, 8
    xg = 0.5 * (np.polynomial.legendre.leggauss(n)[0] + 1.0)
    E = nel[0] * nel[1]
    state = np.empty((E, 4, n * n))
    for e in range(E):
        cx, cy = e % nel[0], e // nel[0]
        X = np.stack(np.meshgrid((cx + xg) * h, (cy + xg) * h, indexing="xy"), -1)
        state[e] = synthetic.euler_vortex_state(X.reshape(-1, 2)).T
    stream = torch.cuda.current_stream(dev)
    out = {"dofs": E * 4 * n * n}
    for dt in (0.1, 0.01):
        rec = {}
        for blocks, extra in (("small", 0), ("full", TPP_FEAT_FULL_BLOCKS)):
            ctx = Context.euler_system(n, nel, h, dt, state,
                                       features=TPP_FEAT_BLOCK_JACOBI | extra, device=str(dev))
            b = torch.as_tensor(synthetic.rhs(1713, ctx.num_dofs), device=dev)
            for kind, pc, build in (("K", TPP_PC_KRON, ctx.tpp_build_factors),
                                    ("J", TPP_PC_BLOCK_JACOBI, ctx.tpp_build_block_jacobi)):
                build()
                x = torch.zeros_like(b)
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                build()
                _, r = ctx.gmres_solve(b, x, restart=30, rtol=1e-8, max_iters=3000, pc=pc,
                                       check=False)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                rec[f"{kind}_{blocks}"] = {"iters": r["iters"], "converged": bool(r["converged"]),
                                           "true_rel_res": r["true_rel_res"],
                                           "build_solve_ms": e0.elapsed_time(e1)}
            del ctx
        out[f"dt={dt}"] = rec
    return out


def run_3d(args):
    """The 3D configuration (16^3 periodic hexes, n = 11, 5.45M DOFs, dt = 0.05):
    nested factor build (Alg. 3d-form), preconditioner apply (Alg. 3d-apply) in
    FP64 and FP32, the sum-factorised operator, and GMRES(30) with the nested
    preconditioner from b ~ N(0, 1), run for at most --max-iters iterations.
    value = FP64 preconditioner-apply throughput (GDOF/s)."""
    import torch
    from paper_1704_04549_gb300 import TPP_FEAT_MIXED, TPP_FP32, TPP_FP64, TPP_PC_KRON, Context
    from paper_1704_04549_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    w = workload_3d(args.n if args.n != 16 else 11)
    n = w["n"]
    ctx = Context(3, n, w["nel"], w["h"], w["dt"], w["velocity"], max_restart=30,
                  features=TPP_FEAT_MIXED | form_bits(args), device=str(dev))
    N, E = ctx.num_dofs, ctx.num_elem
    b = torch.as_tensor(synthetic.rhs(w["rhs_seed"], N), device=dev)
    z = torch.empty_like(b)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.tpp_build_factors()
    l0 = lib.tpp_kernel_launch_count()
    with ClockSampler(0) as clk:
        build_ms = time_each(lambda: ctx.tpp_build_factors(), args.steps, stream, flush)
        apply = {}
        for name, prec in (("fp64", TPP_FP64), ("fp32", TPP_FP32)):
            for _ in range(args.warmup):
                ctx.tpp_apply_inverse(b, z, prec=prec)
            t_ms = time_each(lambda: ctx.tpp_apply_inverse(b, z, prec=prec), 10 * args.steps,
                             stream, flush)
            apply[name] = {"ms": t_ms, "gdofs": N / (t_ms * 1e-3) / 1e9}
        for _ in range(args.warmup):
            ctx.dg_apply_sumfact(b, z)
        op_ms = time_each(lambda: ctx.dg_apply_sumfact(b, z), 10 * args.steps, stream, flush)
    launches = lib.tpp_kernel_launch_count() - l0
    gm = {}
    for name, prec, kin in (("fp64", TPP_FP64, 0), ("mixed", TPP_FP32, args.inner)):
        x = torch.zeros_like(b)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, r = ctx.gmres_solve(b, x, restart=30, rtol=1e-8, max_iters=args.max_iters,
                               pc=TPP_PC_KRON, inner_prec=prec, flexible=(prec != TPP_FP64),
                               check=False, inner_iters=kin)
        gm[name] = {"iters": r["iters"], "inner_iters": r["inner_iters"],
                    "converged": bool(r["converged"]), "true_rel_res": r["true_rel_res"],
                    "wall_ms": (time.perf_counter() - t0) * 1e3}
    flops = 12.0 * n ** 4 * E         # z transform 2 n^4 + n slice applies of 10 n^3
    achieved = flops / (apply["fp64"]["ms"] * 1e-3) / 1e9
    line = {
        "metric": "precond-apply GDOF/s, 3D nested Kronecker preconditioner, 1 GB300",
        "value": apply["fp64"]["gdofs"], "unit": "GDOF/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"adv3d-fourier-16x16x16-n{n} (p={n - 1}), unit hexes, dt=0.05, "
                               f"solenoidal random-Fourier velocity seed 1707, b~N(0,1) seed 1708",
                   "n": n, "nel": [16, 16, 16], "h": 1.0, "dt": 0.05, "dofs": N,
                   "apply_form": args.form,
                   "l2": "L2 flushed (256 MB write) before each timed launch"},
        "build_ms": build_ms,
        "precond_apply": {"fp64_gdofs": apply["fp64"]["gdofs"], "fp64_ms": apply["fp64"]["ms"],
                          "fp32_gdofs": apply["fp32"]["gdofs"], "fp32_ms": apply["fp32"]["ms"]},
        "operator": {"ms": op_ms, "gdofs": N / (op_ms * 1e-3) / 1e9},
        "gmres": gm,
        "roofline": {"kernel": "3D apply (k_apply_z + %s on z slices)"
                               % ("k_apply_2d_w<double>" if args.form == "two-sided"
                                  else "k_apply_2d_g<double>"),
                     "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS,
                     "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS, "traffic": None,
                     "peak_note": FP64_PEAK_NOTE, "algorithmic": "12 n^4 flop per element"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    return 0


def batch_measure(args, scale: float, steps: int, warmup: int, sample_clocks: bool = True):
    """Per-system batched GMRES on the mixed-degree batch scaled by `scale`: contexts and
    right-hand sides, autotuned launch shapes (5 % sample), then `warmup` untimed and
    `steps` timed steps (factor build of every group + solve) in FP64 and mixed precision.
    Returns (results per mode, autotune, groups, dof_rhs, clocks, kernel launches)."""
    import torch
    from paper_1704_04549_gb300 import Context
    from paper_1704_04549_gb300 import _lib
    from paper_1704_04549_gb300.batch import BatchGmres
    lib = _lib.load()
    dev = torch.device("cuda:0")
    groups = synthetic.mixed_degree_batch(e2d=int(round(20000 * scale)),
                                          e3d=int(round(2000 * scale)))
    vel = {2: synthetic.fourier_velocity(1709, 2), 3: synthetic.fourier_velocity(1709, 3)}
    h_el = 1.0 / 64 if args.h_reading == "domain" else 1.0
    R = 64
    feats = _lib.TPP_FEAT_TWO_SIDED | _lib.TPP_FEAT_MIXED

    def make(grps):
        cs, b_, x_ = [], [], []
        for g in grps:
            c = Context(g.dim, g.n, (len(g.ids),), h_el, 0.05, vel[g.dim], max_restart=1,
                        features=feats, device=str(dev), batch_rhs=R, centres=g.centres,
                        batch_span=1.0 / 64)
            c.tpp_build_factors()
            cs.append(c)
            b_.append(torch.as_tensor(synthetic.rhs(g.rhs_seed, c.num_dofs), device=dev))
            x_.append(torch.zeros(c.num_dofs, dtype=torch.float64, device=dev))
        return cs, b_, x_

    # launch shapes per lane-group width from the autotuner, on a 5 % sample of the batch
    # (same degree groups; JSON cache keyed by GPU, precision, restart and groups)
    from paper_1704_04549_gb300.autotune import tune_batch_gmres
    sample = synthetic.mixed_degree_batch(e2d=max(1, int(round(1000 * scale))),
                                          e3d=max(1, int(round(100 * scale))))
    sc, sb, sx = make(sample)
    common = dict(restart=args.batch_restart, rtol=1e-8, max_iters=args.max_iters,
                  inner_rtol=args.batch_inner_rtol, max_outer=8)
    tuned = {m: tune_batch_gmres(sc, sb, sx, mixed=(m == "mixed"), **common)
             for m in ("fp64", "mixed")}
    del sc, sb, sx
    ctxs, bs, xs = make(groups)
    dofs = sum(c.num_dofs for c in ctxs)
    solvers = {m: BatchGmres(ctxs, mixed=(m == "mixed"), warps=tuned[m]["warps"],
                             ctas_per_sm=tuned[m]["ctas_per_sm"],
                             reg_budget=tuned[m]["reg_budget"], per_system=True, **common)
               for m in ("fp64", "mixed")}
    stream = torch.cuda.current_stream(dev)

    def build():
        for c in ctxs:
            c.tpp_build_factors()

    def timed(fn, steps):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = [fn() for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps, out[-1]

    res = {}
    l0 = lib.tpp_kernel_launch_count()
    clk = ClockSampler(0) if sample_clocks else contextlib.nullcontext()
    with clk:
        for mode, sv in solvers.items():
            for _ in range(warmup):
                build()
                sv.solve(bs, xs)
            ms, rep = timed(lambda: (build(), sv.solve(bs, xs))[1], steps)
            ms_solve, _ = timed(lambda: sv.solve(bs, xs), steps)
            its = torch.cat([t.double() for t in sv.iters])
            res[mode] = {"ms": ms, "solve_ms": ms_solve, "build_ms": ms - ms_solve,
                         "launch_ms": rep["launch_ms"],
                         "unconverged": rep["unconverged"], "max_relres": rep["max_relres"],
                         "iters_mean": float(its.mean()), "iters_max": rep["max_iters"],
                         "iters_total": rep["total_iters"], "max_outer": rep["max_outer"],
                         "launches_per_solve": rep["launches"]}
    launches = lib.tpp_kernel_launch_count() - l0
    return res, tuned, groups, dofs, (clk.summary() if sample_clocks else None), launches


def run_batch(args):
    """The mixed-degree batch (20,000 2D elements, p ~ U{4..30}, and 2,000 3D elements,
    p ~ U{3..12}; isolated unit elements (h = 1; --h-reading domain: h = 1/64) covering 1/64
    of the velocity field's unit domain, centres uniform, random-Fourier velocity, dt = 0.05,
    64 right-hand sides ~ N(0, 1) per element), every (element, right-hand side) system
    solved to 1e-8 by its own GMRES (tpp_batch_gmres: persistent launches grouped by n).
    One context per degree group holds the factors; a step = the factor build of every
    group + the batched solve; value = device time of one FP64 step, the mixed-precision
    step as a sub-record.  Inputs (3.9 + 0.8 GB per vector set) exceed L2."""
    import torch
    if args.batch_solver == "group":
        return run_batch_groups(args)
    h_el = 1.0 / 64 if args.h_reading == "domain" else 1.0
    res, tuned, groups, dofs, clocks, launches = batch_measure(args, args.batch_scale,
                                                               args.steps, args.warmup)
    e2d = sum(len(g.ids) for g in groups if g.dim == 2)
    e3d = sum(len(g.ids) for g in groups if g.dim == 3)
    line = {
        "metric": "mixed-degree batch: time to solve every (element, rhs) system to 1e-8 "
                  "(factor build + per-system batched GMRES), 1 GB300",
        "value": res["fp64"]["ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": False, "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "mixed-degree batch, %d 2D elements p~U{4..30} + %d 3D elements "
                               "p~U{3..12}, h=%g, span 1/64, dt=0.05, 64 RHS each, seed 1709, "
                               "GMRES(%d) per system" % (e2d, e3d, h_el, args.batch_restart),
                   "groups": len(groups), "dof_rhs": dofs, "scale": args.batch_scale,
                   "l2": "inputs larger than L2"},
        "fp64": res["fp64"], "mixed": res["mixed"],
        "autotune": {m: {k: t[k] for k in ("warps", "ctas_per_sm", "reg_budget", "cached",
                                            "table")} for m, t in tuned.items()},
        "all_converged": all(r["unconverged"] == 0 for r in res.values()),
        "dof_rhs_per_s": {m: dofs / (r["ms"] * 1e-3) for m, r in res.items()},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(line))
    return 0


def run_batch_groups(args):
    """The mixed-degree batch (20,000 2D elements, p ~ U{4..30}, and 2,000 3D elements,
    p ~ U{3..12}; isolated unit elements (h = 1; --h-reading domain: h = 1/64) covering 1/64 of
    the velocity field's unit domain, centres uniform, random-Fourier velocity, dt = 0.05, 64
    right-hand sides ~ N(0, 1) per element; each
    element's block-diagonal system solved to 1e-8).  One context per degree group, groups
    in sequence, each group's systems as one Krylov solve (gmres_solve); value = the sum
    over groups of the device time of one step (factor build + solve)."""
    import torch
    from paper_1704_04549_gb300 import batch as B
    from paper_1704_04549_gb300 import _lib
    lib = _lib.load()
    groups = synthetic.mixed_degree_batch(e2d=int(round(20000 * args.batch_scale)),
                                          e3d=int(round(2000 * args.batch_scale)))
    vel = {2: synthetic.fourier_velocity(1709, 2), 3: synthetic.fourier_velocity(1709, 3)}
    h_el = 1.0 / 64 if args.h_reading == "domain" else 1.0   # element width (scales the block)
    out = {}
    l0 = lib.tpp_kernel_launch_count()
    with ClockSampler(0) as clk:
        for mode, kin in (("fp64", 0), ("mixed", args.inner)):
            rows = [B.solve_group(g, 64, h_el, 0.05, vel[g.dim], span=1.0 / 64,
                                  inner_iters=kin, max_iters=args.max_iters, steps=args.steps,
                                  warmup=args.warmup, use_graph=args.graph) for g in groups]
            out[mode] = rows
    launches = lib.tpp_kernel_launch_count() - l0
    tot = {m: sum(r["ms_per_step"] for r in rows) for m, rows in out.items()}
    dofs = sum(r["dofs"] for r in out["fp64"])
    line = {
        "metric": "mixed-degree batch: time to solve every block system to 1e-8 "
                  "(factor build + solve), 1 GB300",
        "value": tot["fp64"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": False, "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "mixed-degree batch, %d 2D elements p~U{4..30} + %d 3D elements "
                               "p~U{3..12}, h=%g, span 1/64, dt=0.05, 64 RHS each, seed 1709"
                               % (sum(len(g.ids) for g in groups if g.dim == 2),
                                  sum(len(g.ids) for g in groups if g.dim == 3), h_el),
                   "groups": len(groups), "dof_rhs": dofs,
                   "scale": args.batch_scale},
        "mixed": {"ms": tot["mixed"], "inner_iters_per_outer": args.inner,
                  "all_converged": all(r["converged"] for r in out["mixed"])},
        "all_converged": all(r["converged"] for r in out["fp64"]),
        "dof_rhs_per_s": {m: dofs / (t * 1e-3) for m, t in tot.items()},
        "groups": {m: [{k: r[k] for k in ("dim", "n", "elements", "ms_per_step", "iters",
                                          "inner_iters", "converged")} for r in rows]
                   for m, rows in out.items()},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    return 0


def run_learned(args):
    """Learned factors, n = 16 (p = 15).  Training: 50,000 isolated unit elements from
    10 random-Fourier fields (seeds 1801-1810, span 1/64, dt = 0.05), loss = the
    gauge-invariant relative rank-2 error on each exact rearranged block, Adam with
    a cosine learning rate, all in libtpp's kernels.  Held out: 10,000 elements from
    2 other fields (1811, 1812).  Then the 64 x 64 mesh of the default workload
    (field 1705, never seen in training): one step = learned build (inputs, network
    forward, error check, exact KSVD for the elements above 0.05, inverses and
    Schur forms) + GMRES(30) to 1e-8 with the iteration fallback, against one step
    of the exact build + the same GMRES."""
    import torch
    from paper_1704_04549_gb300 import TPP_FEAT_LEARNED, TPP_FEAT_MIXED, TPP_PC_KRON, Context
    from paper_1704_04549_gb300 import _lib
    from paper_1704_04549_gb300 import learned as LN
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    n = 16
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    l0 = lib.tpp_kernel_launch_count()
    with ClockSampler(0) as clk:
        Xt, Mt, _, basis = LN.element_samples(n, args.train_elems, range(1801, 1811), seed=1800)
        Xh, Mh, _, _ = LN.element_samples(n, args.eval_elems, (1811, 1812), seed=1799)
        net = LN.Mlp(n, max_batch=16384, params=LN.default_params(n, 1800))
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        hist = LN.train(net, basis, Xt, Mt, args.epochs, batch=args.mlp_batch, lr=args.lr,
                        lr_min=args.lr * 1e-2)
        t1.record(stream)
        torch.cuda.synchronize()
        train_s = t0.elapsed_time(t1) * 1e-3
        err_tr = LN.element_errors(net, basis, Xt[:10000], Mt[:10000]).cpu().numpy()
        err_ho = LN.element_errors(net, basis, Xh, Mh).cpu().numpy()

        w = workload(n)
        ctx = Context(2, n, w["nel"], w["h"], w["dt"], w["velocity"], max_restart=30,
                      features=TPP_FEAT_LEARNED | TPP_FEAT_MIXED, device=str(dev))
        b = torch.as_tensor(synthetic.rhs(w["rhs_seed"], ctx.num_dofs), device=dev)
        x = torch.zeros_like(b)
        Xm, Mm, _ = ctx.tpp_learned_inputs()
        err_mesh = LN.element_errors(net, basis, Xm, Mm).cpu().numpy()
        info = {}

        def exact_step():
            ctx.tpp_build_factors()
            x.zero_()
            _, info["exact"] = ctx.gmres_solve(b, x, restart=30, rtol=1e-8,
                                               max_iters=args.max_iters, pc=TPP_PC_KRON,
                                               check=False)

        def learned_step():
            x.zero_()
            _, info["learned"] = ctx.tpp_solve_learned(net, b, x, threshold=0.05,
                                                       iter_limit=args.iter_limit,
                                                       max_iters=args.max_iters, check=False)

        def exact_build():
            ctx.tpp_build_factors()

        def learned_build():
            info["build"] = ctx.tpp_build_factors_learned(net, 0.05)

        X16 = Xm.repeat(4, 1).contiguous()       # 16,384 rows: the roofline batch

        def forward():
            net.forward(X16)

        for fn in (exact_step, learned_step, exact_build, learned_build, forward):
            for _ in range(args.warmup):
                fn()
        ms = {nm: time_each(fn, args.steps, stream, flush)
              for nm, fn in (("exact_step", exact_step), ("learned_step", learned_step),
                             ("exact_build", exact_build), ("learned_build", learned_build),
                             ("forward", forward))}
    launches = lib.tpp_kernel_launch_count() - l0
    E = ctx.num_elem
    flop_fwd = 2.0 * sum(a * c for a, c in zip(net.widths[:-1], net.widths[1:])) * X16.shape[0]
    bf16_peak, peak_src = bf16_peak_tflops()
    lr_, ex = info["learned"], info["exact"]

    def stats(e):
        return {"accept_frac_0.05": float(np.mean(e <= 0.05)), "median_err": float(np.median(e)),
                "p90_err": float(np.quantile(e, 0.9)), "max_err": float(np.max(e))}

    line = {
        "metric": "learned factors, 64x64 mesh n=16: time to 1e-8 rel. residual (learned build "
                  "with KSVD fallback + GMRES), 1 GB300",
        "value": ms["learned_step"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms["learned_step"], "higher_is_better": False,
        "vs_baseline": None, "dtype": "f64 (network: bf16 weights, f32 accumulation)",
        "data": "synthetic",
        "config": {"workload": "learned factors n=16: train %d isolated elements (fields "
                               "1801-1810), hold out %d (fields 1811-1812), evaluate on the "
                               "adv2d-fourier-64x64-n16 mesh (field 1705)"
                               % (args.train_elems, args.eval_elems),
                   "epochs": args.epochs, "mlp_batch": args.mlp_batch, "lr": args.lr,
                   "threshold": 0.05, "iter_limit": args.iter_limit,
                   "l2": "flushed (256 MB write) before every timed step"},
        "exact": {"ms_per_step": ms["exact_step"], "iters": ex["iters"],
                  "converged": bool(ex["converged"]), "build_ms": ms["exact_build"]},
        "learned": {"ms_per_step": ms["learned_step"], "iters": lr_["iters"],
                    "converged": bool(lr_["converged"]), "rebuilt": lr_["rebuilt"],
                    "true_rel_res": lr_["true_rel_res"], "build_ms": ms["learned_build"],
                    "fallback_elems": info["build"]["num_fallback"], "elements": E},
        "errors": {"train_sample": stats(err_tr), "held_out": stats(err_ho),
                   "mesh": stats(err_mesh)},
        "training": {"seconds": train_s, "epoch_loss_first": hist[0], "epoch_loss_last": hist[-1],
                     "elements_per_s": args.epochs * args.train_elems / train_s},
        "roofline": {"kernel": "k_gemm_tc (tcgen05 BF16, network forward: pair split + 4 "
                               "GEMM launches over 16,384 rows)", "bound": "tensor",
                     "achieved": flop_fwd / (ms["forward"] * 1e-3) / 1e12,
                     "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": flop_fwd / (ms["forward"] * 1e-3) / 1e12 / bf16_peak,
                     "peak_note": peak_src + "; algorithmic flops 2 B sum_l K_l N_l (the BF16 "
                                  "pairs execute 2x that on the tensor pipe)",
                     "traffic": None},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    return 0


def run_timestep(args):
    """Implicit vs explicit time integration to t = 0.05 on the 64 x 64 mesh (n = 16,
    unit quads, field 1705, u^0 ~ N(0, 1) seed 1706), the comparison of Sec. 5.2: one
    step of Alexander's L-stable DIRK3 (dt = 0.05; the Kronecker factors rebuilt for the
    step, three KSVD-preconditioned GMRES(30) stage solves to 1e-10, FP64) against the
    classical RK4 method at 0.9 of its stability limit on the imaginary axis
    (2 sqrt 2 / rho(M^-1 J), rho from 40 power iterations).  value = DIRK3 ms."""
    import torch
    from paper_1704_04549_gb300 import TPP_FEAT_TIME, TPP_TS_DIRK3, TPP_TS_RK4, Context
    from paper_1704_04549_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    w = workload(args.n)
    n, t_end = args.n, 0.05
    ctx = Context(2, n, w["nel"], w["h"], w["dt"], w["velocity"], max_restart=30,
                  features=TPP_FEAT_TIME, device=str(dev))
    N = ctx.num_dofs
    u0 = torch.as_tensor(synthetic.rhs(w["rhs_seed"], N), device=dev)
    # spectral radius of M^-1 J (untimed): J v = (M v - S v) / dt, M the collocated mass
    x, wq = ctx.gauss_legendre()
    mdiag = torch.as_tensor(np.tile(np.kron(wq, wq) * w["h"] ** 2, ctx.num_elem), device=dev)
    v = torch.as_tensor(synthetic.rhs(7, N), device=dev)
    rho = 0.0
    for _ in range(40):
        Jv = (mdiag * v - ctx.dg_apply_sumfact(v)) / w["dt"]
        v2 = Jv / mdiag
        rho = float(torch.linalg.vector_norm(v2) / torch.linalg.vector_norm(v))
        v = v2 / torch.linalg.vector_norm(v2)
    dt_rk = 0.9 * 2.0 * 2.0 ** 0.5 / rho
    steps_rk = int(np.ceil(t_end / dt_rk))
    dt_rk = t_end / steps_rk
    stream = torch.cuda.current_stream(dev)
    res = {}
    l0 = lib.tpp_kernel_launch_count()
    with ClockSampler(0) as clk:
        for name, scheme, dt, steps in (("dirk3", TPP_TS_DIRK3, t_end, 1),
                                        ("rk4", TPP_TS_RK4, dt_rk, steps_rk)):
            times = []
            for it in range(args.warmup + args.steps):
                u = u0.clone()
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rep = ctx.tpp_time_integrate(u, scheme, dt, steps, rebuild_each_step=True,
                                             rtol=1e-10, use_graph=True)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if it >= args.warmup:
                    times.append(e0.elapsed_time(e1))
            res[name] = {"ms": statistics.median(times), "dt": dt, "steps": steps,
                         "gmres_iters": rep["gmres_iters"], "builds": rep["builds"],
                         "max_true_rel_res": rep["max_true_rel_res"],
                         "norm_ratio": float(torch.linalg.vector_norm(u) /
                                             torch.linalg.vector_norm(u0))}
    launches = lib.tpp_kernel_launch_count() - l0
    line = {"metric": "time to t = 0.05: one DIRK3 step (KSVD GMRES stages, factors rebuilt) "
                      "vs explicit RK4, 1 GB300",
            "value": res["dirk3"]["ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"adv2d-fourier-64x64-n{n}, unit quads, u0~N(0,1) seed 1706, "
                                   f"t_end=0.05", "rho_Minv_J": rho},
            "dirk3": res["dirk3"], "rk4": res["rk4"],
            "rk4_over_dirk3": res["rk4"]["ms"] / res["dirk3"]["ms"],
            "gpu_launches": int(launches), "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def run_mrhs(args):
    """Preconditioner apply with 64 right-hand sides per element (the dense case of the
    batch workload): 4096 isolated unit elements of the random-Fourier field 1705 sampled
    over 1/64 of the unit domain at centres uniform (seed 1709), n = 16, dt = 0.05,
    b ~ N(0, 1) (seed 1711).  FP64, FP32 (SIMT) and BF16 (tensor cores, FP32 accumulation)
    applies on the same float64 vectors, L2 flushed before each launch.
    value = BF16 apply GDOF/s."""
    import torch
    from paper_1704_04549_gb300 import (TPP_BF16, TPP_FEAT_BF16, TPP_FEAT_MIXED, TPP_FP32,
                                        TPP_FP64, Context)
    from paper_1704_04549_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    n, E, R = 16, 4096, 64
    rng = np.random.Generator(np.random.PCG64(1709))
    ctx = Context(2, n, (E,), 1.0, 0.05, synthetic.fourier_velocity(1705, 2), max_restart=1,
                  features=TPP_FEAT_MIXED | TPP_FEAT_BF16, device=str(dev), batch_rhs=R,
                  centres=rng.random((E, 2)), batch_span=1.0 / 64)
    ctx.tpp_build_factors()
    N = ctx.num_dofs
    b = torch.as_tensor(synthetic.rhs(1711, N), device=dev)
    z = torch.empty_like(b)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    out = {}
    l0 = lib.tpp_kernel_launch_count()
    with ClockSampler(0) as clk:
        for name, prec in (("fp64", TPP_FP64), ("fp32", TPP_FP32), ("bf16", TPP_BF16)):
            for _ in range(args.warmup):
                ctx.tpp_apply_inverse(b, z, prec=prec)
            t_ms = time_each(lambda: ctx.tpp_apply_inverse(b, z, prec=prec), 10 * args.steps,
                             stream, flush)
            out[name] = {"ms": t_ms, "gdofs": N / (t_ms * 1e-3) / 1e9}
    launches = lib.tpp_kernel_launch_count() - l0
    # algorithmic bytes of the BF16 apply: b and x in float64 plus the element's BF16 factors
    # (S_A, L_B^-1, Q1: 3 n^2; shifted inverses 2 n^3) and T1 in float (n^2)
    fbytes = E * (3 * n * n * 2 + n * n * 4 + 2 * n ** 3 * 2)
    vbytes = 2 * 8 * N
    achieved = (fbytes + vbytes) / (out["bf16"]["ms"] * 1e-3) / 1e9
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    line = {"metric": "preconditioner apply GDOF/s with 64 right-hand sides per element, "
                      "BF16 tensor cores vs FP32 / FP64, 1 GB300",
            "value": out["bf16"]["gdofs"], "unit": "GDOF/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "vs_baseline": None,
            "dtype": "bf16 operands, f32 accumulation (vectors f64)", "data": "synthetic",
            "config": {"workload": "4096 isolated elements n=16, 64 rhs each, field 1705 span "
                                   "1/64, centres seed 1709, b seed 1711",
                       "l2": "flushed (256 MB write) before each timed launch"},
            "apply": out,
            "roofline": {"kernel": "k_apply_2d_tc<double> (mma.sync BF16)", "bound": "hbm",
                         "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None,
                         "algorithmic": "2 x 8 B per DOF (b, x) + per element 3 n^2 BF16 "
                                        "factors, n^2 float T1, 2 n^3 BF16 shifted inverses"},
            "gpu_launches": int(launches), "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def run_kernels(args):
    """Kernel-only pass for profilers: one factor build, then a few launches of
    each hot-path kernel on the same workload (no GMRES loop)."""
    import torch
    if args.workload == "learned":         # network forward (4096 elements), loss, one train
        from paper_1704_04549_gb300 import TPP_FEAT_LEARNED, Context   # step, learned build
        from paper_1704_04549_gb300 import learned as LN
        w = workload(16)
        ctx = Context(2, 16, w["nel"], w["h"], w["dt"], w["velocity"], max_restart=30,
                      features=TPP_FEAT_LEARNED)
        net = LN.Mlp(16, max_batch=4096, params=LN.default_params(16, 1800))
        X, Mn, _ = ctx.tpp_learned_inputs()
        net.forward(X)
        net.element_loss(ctx, X, Mn)
        net.train_step(ctx, X[:512], Mn[:512], 1e-3)
        ctx.tpp_build_factors_learned(net, 0.05)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "kernels", "workload": "learned", "n": 16,
                          "elements": ctx.num_elem}))
        return 0
    if args.workload == "batch":           # per-system batched GMRES, one width class:
        import numpy as np                  # 2D n = 31, 152 isolated elements x 64 rhs
        from paper_1704_04549_gb300 import TPP_FEAT_TWO_SIDED, Context
        from paper_1704_04549_gb300.batch import BatchGmres
        rng = np.random.Generator(np.random.PCG64(7))
        c = Context(2, 31, (152,), 1.0, 0.05, synthetic.fourier_velocity(1709, 2), max_restart=1,
                    features=TPP_FEAT_TWO_SIDED, device="cuda:0", batch_rhs=64,
                    centres=rng.random((152, 2)), batch_span=1.0 / 64)
        c.tpp_build_factors()
        b = torch.as_tensor(synthetic.rhs(3, c.num_dofs), device="cuda:0")
        x = torch.zeros_like(b)
        sv = BatchGmres([c], restart=20, rtol=1e-8)
        sv.solve([b], [x])
        rep = sv.solve([b], [x])
        print(json.dumps({"mode": "kernels", "workload": "batch", "n": 31, "systems": rep["systems"],
                          "launch_ms": rep["launch_ms"], "total_iters": rep["total_iters"]}))
        return 0
    if args.workload == "euler":           # coupled Euler operator, 64 x 64 elements, n = 16
        import numpy as np
        from paper_1704_04549_gb300 import Context
        n, N, h = 16, 64, 20.0 / 64
        xg = 0.5 * (np.polynomial.legendre.leggauss(n)[0] + 1.0)
        cx, cy = np.arange(N * N) % N, np.arange(N * N) // N
        X = np.stack(np.meshgrid(xg, xg, indexing="xy"), -1).reshape(-1, 2)
        pts = np.stack([(cx[:, None] + X[None, :, 0]) * h, (cy[:, None] + X[None, :, 1]) * h], -1)
        state = synthetic.euler_vortex_state(pts).transpose(0, 2, 1)
        ctx = Context.euler_system(n, (N, N), h, 0.05, state, device="cuda:0")
        v = torch.as_tensor(synthetic.rhs(5, ctx.num_dofs), device="cuda:0")
        y = torch.empty_like(v)
        for _ in range(4):
            ctx.dg_apply_sumfact(v, y)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "kernels", "workload": "euler", "n": n, "dofs": ctx.num_dofs}))
        return 0
    if args.workload == "euler_full":      # 2D full blocks: vortex, 32 x 32 elements, n = 8
        import numpy as np
        from paper_1704_04549_gb300 import TPP_FEAT_FULL_BLOCKS, Context
        n, N, h = 8, 32, 20.0 / 32
        xg = 0.5 * (np.polynomial.legendre.leggauss(n)[0] + 1.0)
        cx, cy = np.arange(N * N) % N, np.arange(N * N) // N
        X = np.stack(np.meshgrid(xg, xg, indexing="xy"), -1).reshape(-1, 2)
        pts = np.stack([(cx[:, None] + X[None, :, 0]) * h, (cy[:, None] + X[None, :, 1]) * h], -1)
        state = synthetic.euler_vortex_state(pts).transpose(0, 2, 1)
        ctx = Context.euler_system(n, (N, N), h, 0.1, state, features=TPP_FEAT_FULL_BLOCKS,
                                   device="cuda:0")
        ctx.tpp_build_factors()
        v = torch.as_tensor(synthetic.rhs(5, ctx.num_dofs), device="cuda:0")
        y = torch.empty_like(v)
        for _ in range(4):
            ctx.tpp_apply_inverse(v, y)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "kernels", "workload": "euler_full", "n": n,
                          "dofs": ctx.num_dofs}))
        return 0
    if args.workload == "euler3d":         # 3D periodic case, 8^3 elements, n = 6, full blocks
        import numpy as np
        from paper_1704_04549_gb300 import TPP_FEAT_FULL_BLOCKS, Context
        n, N, L = 6, 8, 2.0
        h = L / N
        xg = 0.5 * (np.polynomial.legendre.leggauss(n)[0] + 1.0)
        gz, gy, gx = np.meshgrid(xg, xg, xg, indexing="ij")
        e = np.arange(N ** 3)
        cx, cy, cz = e % N, (e // N) % N, e // (N * N)
        pts = np.stack([(cx[:, None] + gx.reshape(-1)[None, :]) * h,
                        (cy[:, None] + gy.reshape(-1)[None, :]) * h,
                        (cz[:, None] + gz.reshape(-1)[None, :]) * h], -1)
        state = synthetic.euler3d_wave_state(pts, L).transpose(0, 2, 1)
        ctx = Context.euler_system(n, (N, N, N), h, 2.5e-3, state,
                                   features=TPP_FEAT_FULL_BLOCKS, device="cuda:0")
        ctx.tpp_build_factors()
        v = torch.as_tensor(synthetic.rhs(5, ctx.num_dofs), device="cuda:0")
        y = torch.empty_like(v)
        for _ in range(4):
            ctx.tpp_apply_inverse(v, y)
            ctx.dg_apply_sumfact(v, y)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "kernels", "workload": "euler3d", "n": n, "dofs": ctx.num_dofs}))
        return 0
    from paper_1704_04549_gb300 import TPP_FEAT_MIXED, TPP_FP32, TPP_FP64, Context
    w = workload_3d(args.n if args.n != 16 else 11) if args.workload == "adv3d" else workload(args.n)
    ctx = Context(w["dim"], w["n"], w["nel"], w["h"], w["dt"], w["velocity"], max_restart=30,
                  features=TPP_FEAT_MIXED | form_bits(args))
    b = torch.as_tensor(synthetic.rhs(w["rhs_seed"], ctx.num_dofs), device="cuda:0")
    z = torch.empty_like(b)
    ctx.tpp_build_factors()
    for _ in range(3):
        ctx.tpp_apply_inverse(b, z, prec=TPP_FP64)
    for _ in range(3):
        ctx.tpp_apply_inverse(b, z, prec=TPP_FP32)
    for _ in range(3):
        ctx.dg_apply_sumfact(b, z)
    if args.workload == "adv2d":           # one solve: the Arnoldi kernels in their share
        from paper_1704_04549_gb300 import TPP_PC_KRON
        x = torch.zeros_like(b)
        mixed = args.prec == "mixed"
        ctx.gmres_solve(b, x, restart=30, rtol=1e-8, max_iters=args.max_iters, pc=TPP_PC_KRON,
                        check=False, inner_prec=TPP_FP32 if mixed else TPP_FP64,
                        flexible=mixed, inner_iters=args.inner if mixed else 0)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "kernels", "workload": args.workload, "n": w["n"],
                      "dofs": ctx.num_dofs}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--prec", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["bench", "kernels"], default="bench",
                    help="kernels: one build and a few launches of each kernel (for ncu)")
    ap.add_argument("--max-iters", type=int, default=1000)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the n = 31 and 3D sub-records of the default line")
    ap.add_argument("--ref-iters", type=int, default=34,
                    help="GMRES iterations the reference arm extrapolates to")
    ap.add_argument("--ref-budget", type=float, default=15.0)
    ap.add_argument("--h-reading", choices=["unit", "domain"], default="unit",
                    help="unit: unit-square elements (h = 1); domain: the unit square tiled, "
                         "h = 1/64")
    ap.add_argument("--field", choices=["solenoidal", "components"], default="solenoidal",
                    help="random-Fourier velocity: divergence-free modes, or independent "
                         "modes per component")
    ap.add_argument("--inner", type=int, default=12,
                    help="mixed precision: inner FP32 GMRES steps per outer step (0: one FP32 "
                         "Kronecker apply per outer step)")
    ap.add_argument("--form", choices=["one-sided", "two-sided"], default="one-sided",
                    help="apply form: one-sided (shifted inverses, default) or the paper's "
                         "two-sided Schur / quasi-triangular Sylvester form")
    ap.add_argument("--batch-solver", choices=["system", "group"], default="system",
                    help="batch workload: per-system batched GMRES or one Krylov solve per "
                         "degree group")
    ap.add_argument("--batch-restart", type=int, default=20)
    ap.add_argument("--batch-inner-rtol", type=float, default=1e-4)
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="batch workload: fraction of the 20,000 + 2,000 elements")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="plain kernel launches instead of one captured CUDA graph per group "
                         "of Arnoldi steps (the default)")
    ap.add_argument("--train-elems", type=int, default=50000)
    ap.add_argument("--eval-elems", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--mlp-batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--iter-limit", type=int, default=50,
                    help="learned workload: GMRES iterations before the exact rebuild")
    ap.add_argument("--workload", choices=["adv2d", "adv3d", "batch", "learned", "timestep", "euler",
                                           "mrhs", "euler_full", "euler3d"],
                    default="adv2d",
                    help="adv3d: the 16^3 hex configuration (apply/operator/build throughput)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "kernels":
        return run_kernels(args)
    if args.workload == "adv3d":
        return run_3d(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "timestep":
        return run_timestep(args)
    if args.workload == "mrhs":
        return run_mrhs(args)
    if args.workload in ("euler", "euler_full", "euler3d"):
        return run_euler(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
