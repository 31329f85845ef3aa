#!/usr/bin/env python
"""Benchmark: MG-PCG solves/s of tensor-product spline smoothing on one GB300.

One step = sps_set_points (sort, work lists, diagonals, right-hand side,
coarse matrix, damping) + sps_solve to the workload's tolerance, i.e. the
whole solve path, with the inputs already resident in HBM.  Default workload:
P = 3 cubic splines on 64^3 intervals (K = 300,763), n = 1,000,000 clustered
points (3-component Gaussian mixture clipped to [0,1]^3), lambda = 1e-4,
6 levels, FP64, |r| <= 1e-8 |Phi'y|.

Launch: `python bench.py [--gpus N --steps K --warmup W]`; for N > 1 under
torchrun every rank solves its own replica (no collective on the data path)
and the job value is all solves / max rank time.
`--impl reference` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "MG-PCG solves/s & operator Gpoint-applies/s at rel.res 1e-8; p50/p99 vs plain FP64"


def make_problem(name: str, n: int | None):
    if name == "scale":
        return W.scale(n=n or 1_000_000)
    if name == "pr1":
        return W.pr1(n=n or 2000)
    if name == "mixed":
        return W.mixed(n=n or 4_000_000)
    raise ValueError(name)


def workload_desc(pr) -> str:
    return "%s: P=%d q=3 N=%s (K=%d) n=%d levels=%d lambda=%g tol=%g %s" % (
        pr.name, pr.P, "x".join(str(v) for v in pr.intervals), pr.K, pr.n, pr.levels, pr.lam, pr.tol,
        "FP32 x/y, mixed precision" if pr.precision == "mixed" else "FP64")


def _peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


HBM_GBS = float(_peaks().get("hbm_gbs", 6800.0))   # measured copy bandwidth (fallback 6.8 TB/s)


def point_traffic(kind: str, pr, shape) -> dict | None:
    """DRAM bytes (read + write) of one apply launch of the point operator,
    scaled by the number of points from the ncu capture recorded in
    profiles/traffic.json for this kernel, workload and launch shape; None when
    no capture matches."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None
    for c in rec.get("captures", []):
        if c["kernel"] == kind and c["workload"] == pr.name and c["P"] == pr.P and list(c["shape"]) == list(shape):
            return {"bytes": c["dram_bytes_per_launch"] * pr.n / c["points"],
                    "source": "%s (%s), scaled from %d to %d points" % (c["summary"], c["metric"], c["points"], pr.n)}
    return None


def golden_alpha(pr):
    """The oracle's converged coefficients of this workload (tests/golden), if
    recorded for exactly these inputs."""
    import hashlib
    path = os.path.join(GOLDEN_DIR, "%s_alpha.json" % pr.name)
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    sha = lambda a: hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()
    if rec.get("x_sha256") != sha(pr.x) or rec.get("y_sha256") != sha(pr.y):
        return None
    return np.load(os.path.join(GOLDEN_DIR, "%s_alpha.npy" % pr.name))


def coef_error(coef_dev, gold) -> dict:
    c = coef_dev.cpu().numpy()
    return {"max_rel": float(np.max(np.abs(c - gold)) / np.max(np.abs(gold))),
            "l2_rel": float(np.linalg.norm(c - gold) / np.linalg.norm(gold)),
            "oracle": "tier-2 MG-PCG converged to rel.res 1e-15 (tests/golden)"}


GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- reference arm (CPU oracle)

def host_cpu() -> dict:
    """CPU model and core count of this host (recorded beside every oracle timing)."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Vendor ID") and ":" in line:
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model, "host_cores": os.cpu_count(), "machine": platform.machine()}




def oracle_iterations(pr) -> tuple:
    """Outer iterations the oracle's own MG-PCG took to rel.res 1e-8 on this
    workload, measured by running it to convergence (tests/golden/*.json,
    written by tests/golden/make_scale_alpha.py), or (None, why)."""
    path = os.path.join(GOLDEN_DIR, "%s_alpha.json" % pr.name)
    if not os.path.exists(path):
        return None, "no recorded oracle solve for workload %s" % pr.name
    rec = json.load(open(path))
    return int(rec["iterations_to_1e-8"]), path


class OracleSolveTiming:
    """The oracle's solve of a workload, timed on this host's cores.

    PR1-sized problems (K <= 5e4): the tier-1 direct solve (assembly + banded
    Cholesky), timed whole.  The scale workload: the tier-2 MG-PCG (Algorithm 8
    on assembled matrices, Galerkin coarse operators).  Its set-up is timed once
    on the first n_sample points, the part proportional to n (assembly of Phi
    and Phi'Phi) scaled to all n; each `step` then times real MG-PCG iterations
    at the full K (their cost depends on K and the stencil, not on n), and a
    solve is priced as set-up + (the oracle's own iteration count to 1e-8) x
    (seconds per iteration)."""

    def __init__(self, pr, n_sample: int):
        from oracle import mgcg, spline
        self.pr = pr
        self.kind = "direct" if pr.K <= 50_000 else "tier2"
        self.info = host_cpu()
        self.iters = None
        if self.kind == "direct":
            return
        self.iters, self.iters_src = oracle_iterations(pr)
        ns = min(pr.n, n_sample)
        xs, ys = pr.x[:ns], pr.y[:ns]
        # assembly time a + b n from two sample sizes, extrapolated to all n
        t_sys = []
        for m in (ns // 2, ns):
            t0 = time.perf_counter()
            spline.system(xs[:m], ys[:m], pr.lo, pr.hi, pr.intervals, pr.q, pr.lam)
            t_sys.append(time.perf_counter() - t0)
        per_point = max(t_sys[1] - t_sys[0], 0.0) / (ns - ns // 2)
        t0 = time.perf_counter()
        self.H = mgcg.build_hierarchy(xs, ys, pr.lo, pr.hi, pr.intervals, pr.q, pr.lam, pr.levels, omega=0.5,
                                      galerkin=True)
        t_build = time.perf_counter() - t0
        t_sys = t_sys[1]
        self.setup_s = t_build + per_point * (pr.n - ns)
        self.sample = ns
        self.t_sys, self.t_build = t_sys, t_build

    def step(self, iters: int = 1) -> float:
        """Time one bounded sample; returns its seconds."""
        from oracle import mgcg, spline
        pr = self.pr
        t0 = time.perf_counter()
        if self.kind == "direct":
            A, b, _, _ = spline.system(pr.x, pr.y, pr.lo, pr.hi, pr.intervals, pr.q, pr.lam)
            mgcg.solve_direct(A, b)
            self.solve_s = time.perf_counter() - t0
            return self.solve_s
        mgcg.mgcg(self.H, 0.0, max_iter=iters)     # `iters` iterations (tol 0 never stops early)
        dt = time.perf_counter() - t0
        self.iter_s = dt / iters
        return dt

    def solve_seconds(self) -> float:
        if self.kind == "direct":
            return self.solve_s
        return self.setup_s + self.iters * self.iter_s

    def describe(self) -> str:
        if self.kind == "direct":
            return ("oracle tier-1 direct solve (sparse assembly + LAPACK banded Cholesky) of the whole workload, "
                    "timed whole; single-threaded assembly, LAPACK threads as the host's BLAS sets")
        return ("oracle tier-2 MG-PCG (assembled matrices, Galerkin coarse operators): set-up %.1f s (hierarchy on "
                "%d of %d points %.1f s; Phi/Phi'Phi assembly, %.1f s there, extrapolated linearly in n from two "
                "sample sizes to all points) + %d iterations "
                "(the oracle's own count to rel.res 1e-8, from %s) x %.3f s per iteration timed at the full K; "
                "single-threaded sparse products" % (self.setup_s, self.sample, self.pr.n, self.t_build, self.t_sys,
                                                     self.iters, os.path.relpath(self.iters_src, ROOT), self.iter_s))


def run_reference(args, pr):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if pr.K > 50_000 and oracle_iterations(pr)[0] is None:
        print(json.dumps({"impl": "reference", "unavailable": oracle_iterations(pr)[1]}), flush=True)
        return
    t_wall = time.perf_counter()
    ot = OracleSolveTiming(pr, args.ref_sample)
    for _ in range(args.warmup):
        ot.step(1)
    step_s = [ot.step(1) for _ in range(args.steps)]
    wall = time.perf_counter() - t_wall
    v = 1.0 / ot.solve_seconds()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(step_s),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(pr),
                       "step": ("one oracle MG-PCG iteration at the full K" if ot.kind == "tier2"
                                else "one oracle direct solve")},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": ot.describe(),
                             **ot.info},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm

def run_ours(args, pr):
    import torch
    import torch.distributed as dist

    from paper_1901_00654_gb300 import binding as B
    from paper_1901_00654_gb300 import build as libbuild
    from paper_1901_00654_gb300 import replicas

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    libbuild.build_library()
    B.lib()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    mixed = pr.precision == "mixed"
    xdt = torch.float32 if pr.x.dtype == np.float32 else torch.float64
    x_d = torch.from_numpy(np.ascontiguousarray(pr.x)).to(dev)
    y_d = torch.from_numpy(np.ascontiguousarray(pr.y)).to(dev)
    prec = B.SPS_PREC_MIXED if mixed else B.SPS_PREC_FP64
    plan = B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=prec, autotune=1)
    coef = torch.zeros(plan.K, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def step():
        plan.set_points(x_d, y_d)
        _, res = plan.solve(pr.tol, coef)
        return res

    for _ in range(max(args.warmup, 3)):
        res = step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed before each, CUDA events on the launch stream
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip().isdigit()]
    clocks = ClockSampler(int(ids[local]) if local < len(ids) else local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = B.sps_launch_count()
    B.sps_profile_begin()
    results = []
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        results.append(step())
        ends[k].record(stream)
    torch.cuda.synchronize()
    point_ms, point_launches = B.sps_profile_end()
    launches = B.sps_launch_count() - launches0
    barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    value, max_s = replicas.job_rate(args.steps, total_ms * 1e-3, world, dev)
    max_ms = max_s * 1e3
    res = results[-1]

    # ---- operator apply throughput on the finest level (FP64 and FP32 kernels)
    def time_apply(fn, reps=20):
        v = torch.randn(plan.K, dtype=torch.float64, device=dev)
        u = torch.zeros_like(v)
        for _ in range(3):
            fn(plan.h, pr.levels, v, u)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        total = 0.0
        for _ in range(reps):
            flush.fill_(1.0)
            e0.record(stream)
            fn(plan.h, pr.levels, v, u)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        return total / reps

    apply64 = time_apply(lambda h, g, v, u: B.sps_apply(h, g, B.SPS_PREC_FP64, v, u))
    point64 = time_apply(lambda h, g, v, u: B.sps_point_apply(h, g, B.SPS_PREC_FP64, v, u))

    # ---- FMA peaks of this GPU at run-time clocks (the library's probe) and their derivation
    props = torch.cuda.get_device_properties(dev)
    fma64 = B.sps_probe_fma_rate(fp64=True)
    fma32 = B.sps_probe_fma_rate(fp64=False)
    mhz = clk.get("sm_mhz") or 2070.0
    probe = {"sms": props.multi_processor_count, "sm_mhz_median": mhz,
             "fp64_fma_per_sm_per_clock": fma64 / (props.multi_processor_count * mhz * 1e6),
             "fp32_fma_per_sm_per_clock": fma32 / (props.multi_processor_count * mhz * 1e6),
             "how": "sps_probe_fma_rate: 8 independent FMA chains per thread, 256 threads x 8 CTAs per SM, "
                    "CUDA events; rate / (SMs x median SM clock during the timed steps)"}

    # ---- roofline of the dominant kernel (point operator, apply mode), timed inside the steps
    fma_pt = 2 * 4 ** pr.P                       # gather + scatter multiply-adds per point
    flops_launch = 2.0 * fma_pt * pr.n
    avg_ms = point_ms / max(point_launches, 1)
    fp64_kernel = not mixed
    achieved = flops_launch / (avg_ms * 1e-3) / 1e12
    peak = 2.0 * (fma64 if fp64_kernel else fma32) / 1e12
    tuning = [list(B.sps_get_tuning(plan.h, g)) for g in range(1, pr.levels + 1)]
    cap = point_traffic("fp64" if fp64_kernel else "fp32", pr, tuning[-1])
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": cap["bytes"] if cap else None, "kernel": "k_point (apply mode), %s" % (
                    "FP64" if fp64_kernel else "FP32"),
                "flops_per_launch": flops_launch, "avg_launch_ms": avg_ms, "launches": point_launches,
                "peak_source": "measured %s FMA probe x 2 flops at run-time clocks (not in MEASURED_PEAKS.json)"
                               % ("FP64" if fp64_kernel else "FP32"),
                "traffic_source": cap["source"] if cap else "no ncu capture of this kernel and launch shape"}

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
            "config": {"workload": workload_desc(pr), "step": "set_points (device inputs) + solve",
                       "l2": "flushed (256 MB write) before every timed step", "parallelism": "replicas"},
            "iterations": res.iterations, "rel_res_true": res.rel_res_true, "fp64_applies": res.fp64_applies,
            "operator_gpoint_applies_per_s": {"fp64_apply": pr.n / (apply64 * 1e-3) / 1e9,
                                              "fp64_point_only": pr.n / (point64 * 1e-3) / 1e9},
            "point_launch_shape": tuning, "roofline": roofline, "fma_probe": probe, "clocks": clk,
            "gpu_launches": launches, "step_ms": step_ms}
    gold = golden_alpha(pr)
    if gold is not None:
        line["coef_rel_err_vs_oracle"] = coef_error(coef, gold)

    if not mixed:
        point32 = time_apply(lambda h, g, v, u: B.sps_point_apply(h, g, B.SPS_PREC_MIXED, v, u))
        apply32 = time_apply(lambda h, g, v, u: B.sps_apply(h, g, B.SPS_PREC_MIXED, v, u))
        line["operator_gpoint_applies_per_s"]["fp32_apply_incl_casts"] = pr.n / (apply32 * 1e-3) / 1e9
        line["operator_gpoint_applies_per_s"]["fp32_point_incl_casts"] = pr.n / (point32 * 1e-3) / 1e9
        # the mixed-precision solve of the same workload, beside the plain FP64 one
        with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED,
                    autotune=1) as pm:
            cm = torch.zeros(plan.K, dtype=torch.float64, device=dev)
            pm.set_points(x_d, y_d)
            _, rm = pm.solve(pr.tol, cm)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tm = 0.0
            mixed_steps = max(1, min(args.steps, 3))
            B.sps_profile_begin()
            for _ in range(mixed_steps):
                flush.fill_(2.0)
                e0.record(stream)
                pm.set_points(x_d, y_d)
                _, rm = pm.solve(pr.tol, cm)
                e1.record(stream)
                e1.synchronize()
                tm += e0.elapsed_time(e1)
            p32_ms, p32_n = B.sps_profile_end()
            shape32 = list(B.sps_get_tuning(pm.h, pr.levels))
        mp = {"solves_per_s": mixed_steps / (tm * 1e-3), "iterations": rm.iterations,
              "fp64_applies": rm.fp64_applies, "rel_res_true": rm.rel_res_true,
              "coef_rel_err_vs_fp64_gpu": float((cm - coef).abs().max() / coef.abs().max())}
        if gold is not None:
            mp["coef_rel_err_vs_oracle"] = coef_error(cm, gold)
        line["mixed_precision"] = mp
        # FP32 point operator inside the mixed solves: the slower of streaming its algorithmic
        # bytes at the measured HBM copy bandwidth and its multiply-adds at the FP32 FMA peak
        avg32 = p32_ms / max(p32_n, 1)
        bytes32 = pr.n * pr.P * 4 + 2 * 4 * plan.K
        t_hbm = bytes32 / (HBM_GBS * 1e9)
        t_alu = flops_launch / (2.0 * fma32)
        cap32 = point_traffic("fp32", pr, shape32)
        line["roofline_fp32"] = {
            "bound": "alu" if t_alu >= t_hbm else "hbm", "achieved": flops_launch / (avg32 * 1e-3) / 1e12,
            "peak": 2.0 * fma32 / 1e12, "unit": "TFLOP/s", "frac": max(t_alu, t_hbm) / (avg32 * 1e-3),
            "hbm_achieved_gbs": bytes32 / (avg32 * 1e-3) / 1e9, "hbm_peak_gbs": HBM_GBS,
            "algorithmic_bytes_per_launch": bytes32, "traffic": cap32["bytes"] if cap32 else None,
            "kernel": "k_point (apply mode), FP32, in the mixed solves", "avg_launch_ms": avg32,
            "launches": p32_n, "launch_shape": shape32,
            "frac_definition": "max(t_alu, t_hbm) / measured time: t_alu = 2 (q+1)^P FMA per point at the "
                               "FP32 probe peak, t_hbm = P*4 B per point + 2*4 B per coefficient at the "
                               "measured HBM copy bandwidth"}

    # ---- end to end through the C ABI with pinned host buffers (copies inside the timed region)
    xh = torch.from_numpy(np.ascontiguousarray(pr.x)).pin_memory()
    yh = torch.from_numpy(np.ascontiguousarray(pr.y)).pin_memory()
    ch = torch.zeros(plan.K, dtype=torch.float64).pin_memory()
    xn, yn, cn = xh.numpy(), yh.numpy(), ch.numpy()
    torch.cuda.synchronize()
    barrier()
    e2e_steps = max(3, min(args.steps, 5))
    e2e_s = 0.0
    for _ in range(e2e_steps):
        flush.fill_(3.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.set_points(xn, yn)
        plan.solve(pr.tol, cn)
        e2e_s += time.perf_counter() - t0
    e2e_rate, _ = replicas.job_rate(e2e_steps, e2e_s, world, dev)
    line["e2e"] = {"value": e2e_rate, "unit": "solves/s", "steps": e2e_steps,
                   "h2d_bytes_per_step": int(xn.nbytes + yn.nbytes), "d2h_bytes_per_step": int(cn.nbytes),
                   "timing": "host clock around sps_set_points (host x, y) + sps_solve (host coef), "
                             "L2 flushed before each step"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline and pr.K > 50_000 and oracle_iterations(pr)[0] is None:
        # no recorded oracle solve: the tier-2 hierarchy of this workload is not built (at P = 4,
        # K = 1.5e6 its assembled matrix alone would hold 3.6e9 entries, beyond host memory)
        line["cpu_baseline"] = {"value": None, "unavailable": oracle_iterations(pr)[1]}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        ot = OracleSolveTiming(pr, args.cpu_sample)
        ot.step(3)
        line["cpu_baseline"] = {"value": 1.0 / ot.solve_seconds(), "unit": "solves/s", "cores": 1,
                                "kind": "oracle", "sample": ot.describe(), **ot.info}
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_apply_only(args, pr):
    """Set up the workload once and apply the finest-level point operator
    `--reps` times in FP64 and FP32 (the kernel that ncu captures); prints the
    event-timed average per launch."""
    import torch

    from paper_1901_00654_gb300 import binding as B
    from paper_1901_00654_gb300 import build as libbuild
    libbuild.build_library()
    x_d = torch.from_numpy(np.ascontiguousarray(pr.x)).cuda()
    y_d = torch.from_numpy(np.ascontiguousarray(pr.y)).cuda()
    out = {"workload": workload_desc(pr)}
    if args.sweep:
        # every launch shape of the finest level's point operator (tile side, FP32 lane layout)
        ts0 = {1: 256, 2: 32, 3: 8, 4: 4, 5: 2}[pr.P]
        rows = []
        for ts in (ts0 // 2, ts0, ts0 * 2):
            for lanes in ((2, 3) if pr.P in (3, 4) else (0,)):
                try:
                    with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, tile=ts, lanes_r=lanes) as plan:
                        plan.set_points(x_d, y_d)
                        v = torch.randn(plan.K, dtype=torch.float64, device="cuda")
                        u = torch.zeros_like(v)
                        row = {"tile": ts, "lanes_r": lanes}
                        for prec, name in ((B.SPS_PREC_FP64, "fp64"), (B.SPS_PREC_MIXED, "fp32")):
                            B.sps_point_apply(plan.h, pr.levels, prec, v, u)
                            torch.cuda.synchronize()
                            B.sps_profile_begin()
                            for _ in range(args.reps):
                                B.sps_point_apply(plan.h, pr.levels, prec, v, u)
                            torch.cuda.synchronize()
                            ms, cnt = B.sps_profile_end()
                            row[name + "_ms"] = ms / max(cnt, 1)
                        rows.append(row)
                except B.SpsError as e:
                    rows.append({"tile": ts, "lanes_r": lanes, "error": str(e)})
        out["sweep"] = rows
        print(json.dumps(out), flush=True)
        return
    # the plans of the bench's FP64 and mixed solves (autotuned launch shapes), FP64 first
    # --tile / --lanes-r fix the launch shape (no tuning) so that a profiler sees a known shape
    shape = dict(tile=args.tile, lanes_r=args.lanes_r, autotune=0) if args.tile else dict(autotune=1)
    for prec, name in ((B.SPS_PREC_FP64, "fp64"), (B.SPS_PREC_MIXED, "fp32")):
        with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=prec, **shape) as plan:
            plan.set_points(x_d, y_d)
            v = torch.randn(plan.K, dtype=torch.float64, device="cuda")
            u = torch.zeros_like(v)
            B.sps_point_apply(plan.h, pr.levels, prec, v, u)
            torch.cuda.synchronize()
            B.sps_profile_begin()
            torch.cuda.profiler.start()   # profiler capture range (ncu --profile-from-start off)
            for _ in range(args.reps):
                B.sps_point_apply(plan.h, pr.levels, prec, v, u)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
            ms, cnt = B.sps_profile_end()
            out[name + "_ms_per_launch"] = ms / max(cnt, 1)
            out[name + "_launch_shape"] = list(B.sps_get_tuning(plan.h, pr.levels))
    print(json.dumps(out), flush=True)


def run_launch_profile(args, pr):
    """One set-up and one solve of the bench workload, capped at --profile-iters
    outer iterations: a short run with the same kernel mix per iteration as a
    timed step, for an ncu launch list (ncu intercepts every launch, so a
    whole bench run is far too long under it)."""
    import torch

    from paper_1901_00654_gb300 import binding as B
    from paper_1901_00654_gb300 import build as libbuild
    libbuild.build_library()
    x_d = torch.from_numpy(np.ascontiguousarray(pr.x)).cuda()
    y_d = torch.from_numpy(np.ascontiguousarray(pr.y)).cuda()
    prec = B.SPS_PREC_MIXED if pr.precision == "mixed" else B.SPS_PREC_FP64
    with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=prec,
                max_iter=args.profile_iters, autotune=1) as plan:
        coef = torch.zeros(plan.K, dtype=torch.float64, device="cuda")
        l0 = B.sps_launch_count()
        B.sps_profile_begin()
        t0 = time.perf_counter()
        plan.set_points(x_d, y_d)
        _, res = plan.solve(pr.tol, coef, check=False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        pm, pn = B.sps_profile_end()
        print(json.dumps({"workload": workload_desc(pr), "iterations": res.iterations, "launches": B.sps_launch_count() - l0,
                          "point_launch_shape": [list(B.sps_get_tuning(plan.h, g)) for g in range(1, pr.levels + 1)],
                          "wall_ms": wall * 1e3, "point_apply_ms": pm, "point_apply_launches": pn,
                          "point_apply_share_of_wall": pm / (wall * 1e3)}), flush=True)


def run_paper(args):
    """Section 4 of the paper on the GPU: n = 1e5 sigmoid data, plain CG
    against MGCG -- P = 1..4 on G = 5 grids (Table 2) and P = 2 on
    G = 4..7 (Fig. 2).  lambda and the tolerance are not stated in the paper;
    lambda = 0.1 (at which kappa(A) for P = 2, G = 5 is close to the printed
    1933) and rel.res 1e-6 are used."""
    import torch

    from paper_1901_00654_gb300 import binding as B
    from paper_1901_00654_gb300 import build as libbuild
    libbuild.build_library()
    lam, tol = 0.1, 1e-6
    paper = {1: (22, 2), 2: (73, 4), 3: (367, 14), 4: (747, 19)}   # Table 2 iterations (CG, MGCG_JAC)

    def run(P, G):
        x, y = W.paper_sigmoid(5, 100_000, P)
        out = {}
        for name, pc in (("cg", 0), ("mgcg", 1)):
            with B.Plan(P, [2 ** G] * P, G, lam, precondition=pc, max_iter=50000) as pl:
                pl.set_points(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
                coef = torch.zeros(pl.K, dtype=torch.float64, device="cuda")
                pl.solve(tol, coef, check=False)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, res = pl.solve(tol, coef, check=False)
                torch.cuda.synchronize()
                out[name] = {"iterations": res.iterations, "solve_ms": (time.perf_counter() - t0) * 1e3,
                             "status": res.status}
        return out

    if args.paper_sweep:
        return run_paper_sweep(args, lam, tol, paper)
    table2 = {P: run(P, 5) for P in (1, 2, 3, 4)}
    fig2 = {G: run(2, G) for G in (4, 5, 6, 7)}
    # Table 3 / Fig. 3: condition numbers of A_G and C_MG A_G at P = 2, G = 5 (K = 1225)
    from paper_1901_00654_gb300 import analysis
    x, y = W.paper_sigmoid(5, 100_000, 2)
    with B.Plan(2, [32, 32], 5, lam) as pl:
        pl.set_points(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
        sp = analysis.spectra(*analysis.operator_matrices(pl, 5))
    table3 = {"kappa_A": sp["kappa_A"], "kappa_MG_JAC_A": sp["kappa_MA"],
              "eig_MG_JAC_A_min_max": [float(sp["eig_MA"][0]), float(sp["eig_MA"][-1])],
              "paper": {"kappa_A": 1933.27, "kappa_MG_JAC_A": 1.82}}
    line = {"workload": "paper Section 4: n=1e5 sigmoid data, lambda=%g, rel.res %g, FP64" % (lam, tol),
            "table2_gpu": table2, "fig2_gpu_P2": fig2,
            "table2_paper_iterations_cg_mgcg": paper, "table3_gpu": table3}
    print(json.dumps(line), flush=True)


def run_paper_sweep(args, lam, tol, paper):
    """Section 4 with the smoothing parameters the paper does not state: for
    nu1 = nu2 in {1, 2, 3} and the damping omega = f * 4 / (3 lambda_hat), lambda_hat
    the library's estimate of lambda_max(D^-1 A) (its default damping 1.8 / lambda_hat
    is f = 1.35), with f in {0.5, 0.75, 1, 1.25, 1.4}: the condition number of C_MG A_G at
    P = 2, G = 5 (Table 3, printed 1.82) and the MGCG iteration counts of
    Table 2 (P = 1..4, G = 5; printed 2 / 4 / 14 / 19), on the same data."""
    import torch

    from paper_1901_00654_gb300 import analysis
    from paper_1901_00654_gb300 import binding as B
    from paper_1901_00654_gb300 import build as libbuild
    libbuild.build_library()
    data = {P: W.paper_sigmoid(5, 100_000, P) for P in (1, 2, 3, 4)}
    rows = []
    for nu in (1, 2, 3):
        for f in (0.5, 0.75, 1.0, 1.25, 1.4):
            row = {"nu1": nu, "nu2": nu, "omega_factor": f, "iterations": {}}
            for P in (1, 2, 3, 4):
                x, y = data[P]
                with B.Plan(P, [32] * P, 5, lam, nu1=nu, nu2=nu, max_iter=50000) as pl:
                    pl.set_points(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
                    om = B.sps_get_omega(pl.h, 5)
                    # the library's default omega is 1.8 / lambda_hat
                    B.sps_set_omega(pl.h, [max(o * f * (4.0 / 3.0) / 1.8, 1e-12) if o > 0 else 1.0 for o in om])
                    coef = torch.zeros(pl.K, dtype=torch.float64, device="cuda")
                    _, res = pl.solve(tol, coef, check=False)
                    row["iterations"][P] = res.iterations
                    if P == 2:
                        sp = analysis.spectra(*analysis.operator_matrices(pl, 5))
                        row["kappa_MG_A_P2"] = sp["kappa_MA"]
                        row["eig_MG_A_min_max"] = [float(sp["eig_MA"][0]), float(sp["eig_MA"][-1])]
            rows.append(row)
            print(json.dumps(row), flush=True)
    print(json.dumps({"workload": "paper Section 4 sweep: n=1e5 sigmoid data, lambda=%g, rel.res %g" % (lam, tol),
                      "table3_paper_kappa_MG_JAC_A": 1.82, "table2_paper_iterations_cg_mgcg": paper,
                      "sweep": rows}), flush=True)


def run_batched(args):
    """The batched workload: 512 independent problems solved by one persistent
    graph-captured launch (plans resident), against the same problems solved
    one after the other by the plain FP64 solver."""
    import torch

    from paper_1901_00654_gb300 import binding as B
    from paper_1901_00654_gb300 import build as libbuild
    libbuild.build_library()
    probs = W.batched(count=args.batch_count)
    plans = []
    t0 = time.perf_counter()
    for pr in probs:
        pl = B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi, precision=B.SPS_PREC_MIXED)
        pl.set_points(torch.from_numpy(pr.x).cuda(), torch.from_numpy(pr.y).cuda())
        plans.append(pl)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    coefs = [torch.zeros(pl.K, dtype=torch.float64, device="cuda") for pl in plans]
    hs = [pl.h for pl in plans]
    tol = args.batch_tol
    # the default shape (clusters of 2 for the costliest problems), then the autotuner's pick
    default_s = []
    for _ in range(max(args.warmup, 1)):
        B.sps_solve_batch_shape(hs, coefs, tol, cluster=2, check=False)
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.sps_solve_batch_shape(hs, coefs, tol, cluster=2, check=False)
        torch.cuda.synchronize()
        default_s.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    tuned = B.sps_tune_batch(hs, coefs, tol)
    tune_s = time.perf_counter() - t0
    for _ in range(max(args.warmup, 1)):
        B.sps_solve_batch(hs, coefs, tol, check=False)
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = B.sps_solve_batch(hs, coefs, tol, check=False)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    bt = statistics.median(times)
    its = [r.iterations for r in res]
    cta_ms = sorted((r.solve_ms for r in res), reverse=True)
    ok = sum(r.status == B.SPS_OK for r in res)
    # sequential plain FP64 on a sample of the same problems (the full set takes minutes)
    seq_n = min(args.seq_sample, len(probs))
    seq_t = 0.0
    for pr in probs[:seq_n]:
        with B.Plan(pr.P, pr.intervals, pr.levels, pr.lam, pr.lo, pr.hi) as p64:
            p64.set_points(torch.from_numpy(pr.x).cuda(), torch.from_numpy(pr.y).cuda())
            c = torch.zeros(p64.K, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p64.solve(tol, c, check=False)
            torch.cuda.synchronize()
            seq_t += time.perf_counter() - t0
    for pl in plans:
        pl.close()
    line = {"metric": METRIC, "value": len(probs) / bt, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 1), "ms_per_step": bt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batched: %d problems P in {1,2,3}, K <= 40k, n log-uniform [1e3,1e5], "
                                   "lambda log-uniform [1e-5,1e-1], tol %g, plans resident" % (len(probs), tol)},
            "converged": ok, "iterations_median": statistics.median(its), "iterations_max": max(its),
            "cta_ms_per_problem": {"max": cta_ms[0], "top5": cta_ms[:5], "sum": sum(cta_ms),
                                   "median": statistics.median(cta_ms)},
            "setup_s_all_plans": setup_s,
            "autotuned_shape": {"cluster": tuned[0], "big": tuned[1], "simulated_ms": tuned[2],
                                "tuning_s": tune_s},
            "default_shape_cluster2_solves_per_s": len(probs) / statistics.median(default_s),
            "sequential_plain_fp64": {"solves_per_s": seq_n / seq_t, "sample": seq_n}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    """Poisson request trace through the continuous-batching server, then a
    sample of the same requests one at a time with the plain FP64 solver.

    Every request is solved to --serve-tol with at most --serve-max-iter outer
    iterations (requests that hit the cap are counted as not converged and
    reported).  The plain-FP64 comparison runs the first --serve-seq-sample
    requests of the trace (same arrival times) through the server, and then
    through a one-slot server with the plain FP64 solver; both report solves/s
    and p50/p99 latency on exactly those requests."""
    import torch  # noqa: F401

    from paper_1901_00654_gb300 import binding as B
    from paper_1901_00654_gb300 import build as libbuild
    from paper_1901_00654_gb300 import serving
    libbuild.build_library()
    trace = W.serving_trace(count=args.serve_count, n_hi=args.serve_n_hi)
    srv = serving.Server(slots=args.slots, tol=args.serve_tol, max_iter=args.serve_max_iter)
    try:
        warm = W.serving_trace(seed=99, count=4, n_hi=2e4, P_choices=(2, 3))
        srv.run(warm, time_scale=0.0)
        stats = srv.run(trace)
    finally:
        srv.close()
    mixed = stats.summary()
    by_p = {}
    for c, rq in zip(stats.completed, trace):
        d = by_p.setdefault(str(rq.problem.P), {"requests": 0, "converged": 0, "iterations": []})
        d["requests"] += 1
        d["converged"] += int(c.status == B.SPS_OK)
        d["iterations"].append(int(c.result.iterations))
    for d in by_p.values():
        d["iterations_median"] = float(np.median(d.pop("iterations")))
    # the same sub-trace (first requests, same arrival times) served, then one at a time in plain FP64
    sample = trace[:max(1, min(args.serve_seq_sample, len(trace)))]
    srv = serving.Server(slots=args.slots, tol=args.serve_tol, max_iter=args.serve_max_iter)
    try:
        served_sub = srv.run(sample).summary()
    finally:
        srv.close()
    seq = serving.Server(slots=1, precision=B.SPS_PREC_FP64, tol=args.serve_tol, max_iter=args.serve_max_iter)
    try:
        plain = seq.run(sample).summary()
    finally:
        seq.close()
    line = {"metric": METRIC, "value": mixed["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": len(trace), "warmup": 4, "ms_per_step": 1e3 / max(mixed["solves_per_s"], 1e-12),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "serving: %d Poisson requests at 200/s, P in {2,3,4,5}, n log-uniform [1e4,%g], "
                                   "tol %g, at most %d iterations, %d slots, 120 GB budget"
                                   % (len(trace), args.serve_n_hi, args.serve_tol, args.serve_max_iter, args.slots)},
            "served": mixed, "served_by_P": by_p,
            "same_requests": {"requests": len(sample), "what": "first %d requests of the trace, same arrivals"
                              % len(sample), "served": served_sub, "sequential_plain_fp64": plain}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="scale", choices=["scale", "pr1", "mixed", "batched", "serving", "paper"])
    ap.add_argument("--apply-only", action="store_true", help="time the finest-level point operator only")
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--launch-profile", action="store_true", help="one set-up + capped solve (ncu launch list)")
    ap.add_argument("--profile-iters", type=int, default=100)
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-tol", type=float, default=1e-8)
    ap.add_argument("--seq-sample", type=int, default=32)
    ap.add_argument("--serve-count", type=int, default=48)
    ap.add_argument("--serve-n-hi", type=float, default=2e6)
    ap.add_argument("--serve-tol", type=float, default=1e-6)
    ap.add_argument("--serve-max-iter", type=int, default=1500)
    ap.add_argument("--serve-seq-sample", type=int, default=6)
    ap.add_argument("--sweep", action="store_true", help="with --apply-only: every tile side and lane layout")
    ap.add_argument("--paper-sweep", action="store_true",
                    help="with --config paper: nu1 = nu2 in {1,2,3} x damping factors (Table 3 / Table 2)")
    ap.add_argument("--tile", type=int, default=0, help="with --apply-only: fixed tile side (no autotuning)")
    ap.add_argument("--lanes-r", type=int, default=0, help="with --apply-only --tile: fixed lane layout")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--n", type=int, default=None, help="override the number of points")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default=None,
                    help="override the workload's solver precision (--launch-profile, --apply-only)")
    ap.add_argument("--ref-sample", type=int, default=100_000,
                    help="points on which the reference arm times the oracle's set-up")
    ap.add_argument("--cpu-sample", type=int, default=50_000,
                    help="points on which cpu_baseline times the oracle's set-up")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.config == "batched":
        return run_batched(args)
    if args.config == "serving":
        return run_serving(args)
    if args.config == "paper":
        return run_paper(args)
    pr = make_problem(args.config, args.n)
    if args.precision:
        pr.precision = args.precision
    if args.apply_only:
        return run_apply_only(args, pr)
    if args.launch_profile:
        return run_launch_profile(args, pr)
    if args.impl == "reference":
        run_reference(args, pr)
    else:
        run_ours(args, pr)


if __name__ == "__main__":
    main()
