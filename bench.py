"""Benchmark of the IFGF apply (u = A sigma, Eq. field1) on GB300.

Metric: IFGF apply time t and equivalent interactions per second N^2 * nrhs / t
(the exact sum of Eq. field1 would touch N^2 pairs per right-hand side).

A step is one full apply (density permutation, leaf analytic factors, upward
interpolation of every level, target evaluation = near field + cousin
interpolation of every level, output permutation) on densities already resident
in HBM.  The plan (octree and relevant cones) is built once before timing, as the
paper's T_acc excludes T_pre; its build time is reported as t_plan_ms.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ifgf|reference]

With N > 1 (one process per GPU under torchrun) the job is a batch of N * nrhs
right-hand sides split over the ranks (rhs_shard): each rank builds its own plan of the
same geometry and applies its rows; no data crosses ranks while they evaluate.

--impl reference times the CPU oracle (the direct sum of Eq. field1 on a bounded
sample of targets, all host cores) on the same workload and metric.

The default workload is the largest one that fits one GPU: the 256-wavelength sphere
(N = 25,165,824, 8 right-hand sides, mixed precision).  The line reports the accuracy
of what it timed (rel_err_sampled: the largest relative l2 error over the right-hand
sides at sampled targets, against the oracle's FP64 direct sum, which the cpu_baseline
leg computes and times) and the roofline of the dominant kernel against FMA rates
measured on the device (ifgf_device_peak).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ifgf_inputs as wi  # noqa: E402

DEFAULT_WORKLOAD = "sphere_256lambda"
METRIC = "IFGF apply time and equivalent interactions/s (N^2/t) at rel.err<=1e-3 vs FP64 direct"
UNIT = "interactions/s"

# Algorithmic work of one upward evaluation (one parent interpolation point
# interpolated from one child cone and re-centred), for P = P_s * P_ang^2 nodes: the
# sum-factorised contraction over the azimuthal, polar and radial node indices,
# 2 * (P + P_s * P_ang + P_s) real FMAs (186 FMAs = 372 flops at (3, 5)), plus the
# complex multiply-accumulate by the re-centring factor, 8 flops.  The geometry (child
# cone, Lagrange weights, factor) is box-independent and tabulated per level where that
# pays, so it is not counted.
def upward_flops_per_eval(ps: int, pa: int) -> int:
    return 4 * (ps * pa * pa + ps * pa + ps) + 8


# Adjoint: every cousin or upward evaluation, transposed, is a rank-1 update of the P
# values of its cone's adjoint by the Lagrange weight product times the conjugated factor
# times the reader's value: P real-by-complex multiply-adds (4 P flops) plus the complex
# product of factor and value (8 flops) per RHS.
def adjoint_flops_per_eval(ps: int, pa: int) -> int:
    return 4 * ps * pa * pa + 8


NUM_SMS = 152

# DRAM bytes (read + write) per launch of the dominant kernels, from an ncu capture of
# them, keyed by (workload, precision): the mean over the launches whose time the
# roofline's "achieved" averages (for FP32 plans the upward stage: k_upward_runs on the
# tabled levels and k_upward_staged on the level computed on the fly, one chunk of
# right-hand sides).  Each entry records the SHA-256 of the kernel source it was captured
# on; when the source has changed since, the bench reports null instead of a stale figure.
KERNEL_SOURCE = os.path.join(ROOT, "paper_2010_02857_gb300", "csrc", "ifgf_apply_impl.cuh")
TRAFFIC_BYTES_PER_LAUNCH = {
    # 6 upward launches of one 4-RHS chunk: 963.9 GB read + 377.3 GB written
    ("sphere_256lambda", "mixed"): {"bytes": 223.5e9, "sha": "fe99ecd807d4632d"},
}


def _source_sha(path: str) -> str:
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_per_launch(workload: str, precision: str):
    ent = TRAFFIC_BYTES_PER_LAUNCH.get((workload, precision))
    if not ent or ent["sha"] != _source_sha(KERNEL_SOURCE):
        return None
    return ent["bytes"]


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest x over the ranks of the process group (the slowest rank sets the
    job's time); x itself when no group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def run_reference_ifgf(args, wl: wi.Workload):
    """The oracle's serial CPU IFGF on the whole workload (first right-hand side): the
    plan build (T_pre) once, then warm-up and timed applies (T_acc), on the host cores."""
    import oracle
    oracle.build()
    pts = wl.points()
    sig = wl.densities()[:1]
    t0 = time.perf_counter()
    o = oracle.Plan(pts, wl.kappa, wl.levels, wl.p_radial, wl.p_angular, wl.leaf_ns, wl.leaf_nc)
    t_pre = time.perf_counter() - t0
    run = o.apply if args.op == "apply" else o.apply_adjoint
    for _ in range(args.warmup):
        run(sig)
    times = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        run(sig)
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = wl.n * wl.n / t
    sample = (f"serial CPU IFGF (Algorithm 1), whole workload, first right-hand side; "
              f"T_pre {t_pre:.3f} s, T_acc {t:.3f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": max(1, args.steps), "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "op": args.op, "n": wl.n, "nrhs": 1, "kappa": wl.kappa,
                       "reference": "oracle IFGF"},
            "t_pre_ms": t_pre * 1e3,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_reference(args, wl: wi.Workload):
    """The oracle's direct sum on a bounded sample of targets, on the host cores."""
    import oracle
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    if args.ref_kind == "ifgf":
        run_reference_ifgf(args, wl)
        return
    oracle.build()
    direct = oracle.direct if args.op == "apply" else oracle.direct_adjoint
    pts = wl.points()
    sig = wl.densities()
    tg = wl.target_indices()
    # each step is a bounded sample: at most --ref-targets targets, fewer when one step
    # would take more than about --ref-step-s seconds (the run stays within minutes)
    m0 = min(len(tg), max(1, oracle.num_threads()))  # one target per host core
    t0 = time.perf_counter()
    direct(pts, wl.kappa, sig, tg[:m0])  # warms the library and sizes the sample
    per_target = (time.perf_counter() - t0) / m0
    m = int(min(len(tg), max(m0, int(args.ref_targets)), max(m0, args.ref_step_s / max(per_target, 1e-9))))
    tg = tg[:m]
    times = []
    for _ in range(args.warmup):
        direct(pts, wl.kappa, sig, tg)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        direct(pts, wl.kappa, sig, tg)
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = m * wl.n * wl.nrhs / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "op": args.op, "n": wl.n, "nrhs": wl.nrhs, "kappa": wl.kappa},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"FP64 direct sum of Eq. (field1) at {m} sampled targets x {wl.n} sources"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_baseline(wl: wi.Workload, op: str = "apply", seconds: float = 15.0, u=None) -> tuple[dict, dict]:
    """The oracle's FP64 direct sum (or its conjugate transpose) at sampled targets, timed
    on the host cores, on a bounded sample: the first m of the workload's sampled targets,
    m sized to about `seconds` of CPU work.  The same exact values give the accuracy of
    the GPU result u [nrhs, N] at those targets: the largest relative l2 error over the
    right-hand sides."""
    import oracle
    oracle.build()
    direct = oracle.direct if op == "apply" else oracle.direct_adjoint
    pts = wl.points()
    sig = wl.densities()
    tg = wl.target_indices()
    # the oracle runs its targets in parallel over the host cores: size the sample from
    # a first call with one target per core
    m0 = min(len(tg), max(1, oracle.num_threads()))
    t0 = time.perf_counter()
    direct(pts, wl.kappa, sig, tg[:m0])
    per_target = (time.perf_counter() - t0) / m0
    m = int(min(len(tg), max(m0, seconds / max(per_target, 1e-9))))
    t0 = time.perf_counter()
    ex = direct(pts, wl.kappa, sig, tg[:m])
    t = time.perf_counter() - t0
    value = m * wl.n * wl.nrhs / t
    base = {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 direct sum of Eq. (field1){'' if op == 'apply' else ', conjugate transpose,'} "
                      f"at {m} sampled targets x {wl.n} sources x {wl.nrhs} RHS, {t:.1f} s"}
    acc = None
    if u is not None:
        got = u[:, tg[:m]].astype(np.complex128)
        errs = [float(np.linalg.norm(got[r] - ex[r]) / np.linalg.norm(ex[r])) for r in range(wl.nrhs)]
        acc = {"rel_err_sampled": max(errs), "targets": m,
               "reference": "oracle FP64 direct sum (the cpu_baseline sample)"}
    return base, acc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(wi.WORKLOADS))
    ap.add_argument("--impl", default="ifgf", choices=["ifgf", "reference"])
    ap.add_argument("--ref-targets", type=int, default=256)
    ap.add_argument("--ref-step-s", type=float, default=4.0,
                    help="reference arm: bound of one step's CPU time (sizes the target sample)")
    ap.add_argument("--ref-kind", default="direct", choices=["direct", "ifgf"],
                    help="reference arm: the FP64 direct sum on sampled targets (default), or the "
                         "oracle's serial IFGF (Algorithm 1): plan build and full applies, one "
                         "right-hand side (OMP_NUM_THREADS sets its threads)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed", "batched", "batched_fp16"],
                    help="override the workload's precision")
    ap.add_argument("--nrhs", type=int, default=None,
                    help="override the workload's number of right-hand sides (same generator)")
    ap.add_argument("--op", default="apply", choices=["apply", "adjoint"],
                    help="time ifgf_apply (default) or ifgf_apply_adjoint")
    ap.add_argument("--plan-flags", type=int, default=0,
                    help="ifgf_options.flags of the plan (e.g. 32: no evaluation caches, as in plans too large for them)")
    ap.add_argument("--tune-cache", default=None,
                    help="tune-cache file of batched plans: reuse a stored tile-shape choice, else time and store one")
    args = ap.parse_args()
    wl = wi.WORKLOADS[args.workload]
    if args.nrhs is not None:
        wl = dataclasses.replace(wl, nrhs=args.nrhs)
    if args.impl == "reference":
        run_reference(args, wl)
        return

    import torch
    import paper_2010_02857_gb300 as pkg

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    precision = args.precision or wl.precision
    pts = torch.from_numpy(wl.points()).to(dev)
    t0 = time.perf_counter()
    plan = pkg.Plan(pts, wl.kappa, wl.levels, wl.p_radial, wl.p_angular, wl.leaf_ns, wl.leaf_nc,
                    max_nrhs=wl.nrhs, precision=precision, leaf_max=wl.leaf_max, flags=args.plan_flags)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    stats = plan.stats()
    # right-hand sides sharded over the ranks: the job is a batch of world * nrhs
    # right-hand sides of the workload's kind, and rank r applies rows
    # [r nrhs, (r + 1) nrhs) of it on its own plan (weak scaling; no data crosses ranks)
    batch = world * wl.nrhs
    r0, r1 = pkg.rhs_shard(batch, rank, world)
    sig_np = wl.densities((r0, r1, batch)).astype(plan.numpy_dtype)
    sig = torch.from_numpy(sig_np).to(dev)
    u = torch.empty_like(sig)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # the operation timed: the forward apply or its adjoint (same plan, same buffers)
    evaluate = plan.apply if args.op == "apply" else plan.apply_adjoint
    # batched plans: the tile shapes come from the autotuner, timed on this plan
    tiles = None
    if precision.startswith("batched") and wl.nrhs % 2 == 0 and wl.nrhs <= (64 if wl.p_radial == 3 else 48):
        t0 = time.perf_counter()
        tiles = plan.autotune(wl.nrhs, cache=args.tune_cache)
        tiles["tune_s"] = time.perf_counter() - t0
    # every evaluation below replays a CUDA graph of the apply's launches; the graphs
    # (with and without the stage events) are captured during the warm-up
    plan.set_graphs(True)
    plan.set_profiling(True)
    for _ in range(max(3, args.warmup)):
        evaluate(sig, out=u)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    plan.set_profiling(True)  # clears the warm-up's stage totals
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between steps (256 MB > 129 MB L2)
        ev[k][0].record(stream)
        evaluate(sig, out=u)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    timings = plan.timings()
    plan.set_profiling(False)

    # end to end through the C ABI with pinned host buffers
    sig_h = torch.empty(sig.shape, dtype=sig.dtype, pin_memory=True)
    sig_h.copy_(torch.from_numpy(sig_np))
    u_h = torch.empty(sig.shape, dtype=sig.dtype, pin_memory=True)
    evaluate(sig_h, out=u_h)  # captures the graph of the host-pointer calls
    e2e_times = []
    for _ in range(max(2, min(args.steps, 3))):
        t0 = time.perf_counter()
        evaluate(sig_h, out=u_h)  # host pointers: H2D, evaluation, D2H, synchronise
        e2e_times.append(time.perf_counter() - t0)
    clk = clocks.stop()

    ms = max_over_ranks(float(np.mean(step_ms)), dev)
    n, nrhs = wl.n, wl.nrhs
    value = world * n * n * nrhs / (ms * 1e-3)
    e2e_s = max_over_ranks(float(np.median(e2e_times)), dev)
    eb = 16 if precision == "fp64" else 8

    # roofline of the dominant kernel, against FMA or tensor rates measured on this device
    st = timings["stages"]
    calls = max(1, timings["calls"])
    up_ms = st["upward"]["ms"] / calls
    up_launches = st["upward"]["launches"] / calls
    up_evals = sum(lv["upward_evals"] for lv in stats["level"])
    cousin_evals = sum(lv["cousin_evals"] for lv in stats["level"])
    fp64_peak = pkg.device_peak("fp64")
    fp32_peak = pkg.device_peak("fp32")
    pipe = "FP64" if precision == "fp64" else "FP32"
    peak_src = (f"measured {pipe} FMA rate of this device (ifgf_device_peak: independent FMA chains, "
                f"CUDA events)")
    if args.op == "adjoint":
        # k_adj_level: the transposed cousin-target and upward evaluations of every level
        ad_ms = st["adj_level"]["ms"] / calls
        ad_launches = st["adj_level"]["launches"] / calls
        adj_flops = adjoint_flops_per_eval(wl.p_radial, wl.p_angular)
        flops = (up_evals + cousin_evals) * adj_flops * nrhs
        peak = fp64_peak if precision == "fp64" else fp32_peak
        roofline = {"bound": "alu", "kernel": "k_adj_level", "peak_source": peak_src,
                    "work": f"{up_evals + cousin_evals} transposed evaluations x {adj_flops} flops "
                            f"per RHS, {ad_launches:.0f} launches, {ad_ms:.3f} ms"}
        up_ms = ad_ms
    elif precision.startswith("batched"):
        # tcgen05 cone kernels: every cousin and upward evaluation is one GEMM row of
        # P weights x 2 nrhs real columns (useful flops; the hi/lo operand split and
        # the padding of K to a multiple of 16 are not counted)
        rows = up_evals + cousin_evals
        npts = wl.p_radial * wl.p_angular ** 2
        flops = rows * 2 * npts * 2 * nrhs
        peak = float(measured_peaks().get("bf16_tflops", 1900.0))
        roofline = {"bound": "tensor", "kernel": "k_cone_mma", "peak_source": "measured bf16 dense (burst)",
                    "work": f"{rows} GEMM rows x {2 * npts * 2 * nrhs} flops per apply, "
                            f"{up_launches:.0f} launches, {up_ms:.3f} ms"}
    else:
        up_flops = upward_flops_per_eval(wl.p_radial, wl.p_angular)
        flops = up_evals * up_flops * nrhs
        peak = fp64_peak if precision == "fp64" else fp32_peak
        kname = "k_upward" if precision == "fp64" else "k_upward_runs + k_upward_staged"
        roofline = {"bound": "alu", "kernel": kname, "peak_source": peak_src,
                    "work": f"{up_evals} upward evaluations x {up_flops} {pipe} flops per RHS, "
                            f"{nrhs} RHS, {up_launches:.0f} launches, {up_ms:.3f} ms"}
    achieved = flops / (up_ms * 1e-3) / 1e12 if up_ms > 0 else None
    traffic = (traffic_per_launch(wl.name, precision)
               if nrhs == wi.WORKLOADS[wl.name].nrhs and args.op == "apply" else None)
    roofline.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic, "traffic_unit": "bytes per launch" if traffic else None,
                     "measured_fma_peaks_tflops": {"fp64": fp64_peak, "fp32": fp32_peak}})

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "mixed": "f32+f64", "batched": "bf16x3+f32+f64",
                          "batched_fp16": "f16x3+f32+f64"}[precision],
                "data": "synthetic",
                "config": {"workload": wl.name, "op": args.op, "n": n, "nrhs": nrhs, "kappa": wl.kappa, "levels": wl.levels,
                           "p_radial": wl.p_radial, "p_angular": wl.p_angular,
                           "leaf_cones": [wl.leaf_ns, wl.leaf_nc], "precision": precision,
                           "leaf_max": wl.leaf_max, "plan_flags": args.plan_flags,
                           "l2": "flushed between steps (256 MB write)", "launch": "CUDA graph replay",
                           "parallelism": f"rhs-sharded x{world}", "batch_nrhs": batch},
                "t_plan_ms": t_plan * 1e3, "tiles": tiles,
                "stage_ms": {k: v["ms"] / calls for k, v in st.items() if v["launches"] or v["ms"]},
                "e2e": {"value": world * n * n * nrhs / e2e_s, "unit": UNIT,
                        "h2d_bytes_per_step": n * nrhs * eb, "d2h_bytes_per_step": n * nrhs * eb,
                        "ms_per_step": e2e_s * 1e3},
                "gpu_launches": int(sum(v["launches"] for v in st.values()) / calls * args.steps),
                "roofline": roofline, "clocks": clk,
                "device_bytes": stats["device_bytes"]}
        if not args.no_cpu_baseline and world == 1:
            base, acc = cpu_baseline(wl, args.op, u=u.cpu().numpy())
            line["cpu_baseline"] = base
            line["rel_err_sampled"] = acc["rel_err_sampled"]
            line["accuracy"] = acc
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
