#!/usr/bin/env python
"""Benchmark of the twogrid-preconditioned FGMRES Helmholtz solver on GB300.

Workload: 2D P1 on the unit square, h = 1/512 (263,169 complex DoFs), k = 200
(kh ~ 0.39), Gaussian point source (sigma = 2h) at the centre with g = 0,
shift epsilon = 0.5 k^2, twogrid V(2,2) with damped Jacobi (omega = 0.6),
FGMRES(80), true relative residual 1e-8. Precision: complex64 V-cycle inside
complex128 FGMRES (the all-FP64 form is measured beside it).

One step = the whole hot path for one problem: helm_setup (stencil tables,
coarse matrix and its FP64 factorisation) + helm_solve (FGMRES to 1e-8) +
helm_destroy. `value` = steps per second over all GPUs (replicas: every rank
solves its own problem; no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import helm_inputs as hi  # noqa: E402

METRIC = "FGMRES solves/s & p99 latency at relres 1e-8, mixed vs FP64; stencil HBM GB/s"
WL = hi.GAUSS_P1
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
L2_FLUSH_BYTES = 512 << 20


def workload_config(prec_name):
    return {
        "workload": f"{WL.name}: 2D P1 Helmholtz, h=1/{WL.n} ({WL.num_dofs} complex DoFs), k={WL.k:g}, "
                    f"eps=0.5k^2, Gaussian source sigma=2h, impedance BC, V(2,2) omega=0.6, "
                    f"FGMRES({WL.restart}), relres {WL.tol:g}, {prec_name}",
        "step": "helm_setup + helm_solve + helm_destroy (all hot-path rows, setup included)",
        "l2": "flushed between timed steps (512 MB write); the step's working set (~0.9 GB) also exceeds L2",
        "parallelism": "replicas",
    }


# ---------------------------------------------------------------------------- helpers

def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out" if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else ".",
                                 f".clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    mx = float(c[2])
                except ValueError:
                    continue
                for n, v in zip(names, c[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            os.remove(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return world, rank, local, dist


def max_over_ranks(x, dist, device):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, torch):
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()


# ---------------------------------------------------------------------------- CPU oracle leg

def _oracle_sample(n_iters, q):
    """Bounded sample of the oracle on this workload (runs in a spawned process)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    from oracle import solver
    t0 = time.perf_counter()
    pb = solver.build_problem(WL)
    tg = pb.twogrid()
    t1 = time.perf_counter()
    r = solver.fgmres(pb.A0, pb.F, tg.apply, WL.restart, WL.tol, n_iters)
    t2 = time.perf_counter()
    q.put({"setup_s": t1 - t0, "iter_s": (t2 - t1) / max(r.iters, 1), "iters": r.iters})


def oracle_baseline(n_iters=30):
    """Oracle setup + n_iters FGMRES iterations, extrapolated to a full solve with the
    oracle's own iteration count (tests/golden/oracle_iterations.json)."""
    env_threads = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    old = {k: os.environ.get(k) for k in env_threads}
    os.environ.update(env_threads)
    try:
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        p = ctx.Process(target=_oracle_sample, args=(n_iters, q))
        p.start()
        res = q.get(timeout=900)
        p.join(timeout=60)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    with open(GOLDEN) as f:
        full_iters = json.load(f)[WL.name]["iters"]
    t_full = res["setup_s"] + res["iter_s"] * full_iters
    return {
        "value": 1.0 / t_full, "unit": "solves/s", "cores": 1, "kind": "oracle",
        "sample": f"oracle (numpy/scipy, 1 thread) assembly + sparse LU setup ({res['setup_s']:.1f} s) "
                  f"and the first {res['iters']} FGMRES iterations ({res['iter_s'] * 1e3:.0f} ms each), "
                  f"extrapolated to the oracle's full {full_iters} iterations",
        "seconds_per_solve": t_full,
    }


def run_reference(args):
    world, rank, local, dist = dist_setup()
    if rank != 0:
        return
    samples = []
    for i in range(args.warmup + args.steps):
        b = oracle_baseline(n_iters=20)
        if i >= args.warmup:
            samples.append(b)
    v = statistics.mean(s["value"] for s in samples)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config("FP64 oracle (CPU)"),
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": samples[-1]["sample"]},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU leg

def run_ours(args):
    import torch
    world, rank, local, dist = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2104_01439_gb300 as pkg

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sigma = 2.0 / WL.n

    def make(prec):
        return pkg.Solver(WL.k, WL.n, WL.order, WL.shift, restart=WL.restart, maxit=WL.maxit, tol=WL.tol,
                          omega=WL.omega, nu=WL.nu, precision=prec, stream=stream)

    # host input (the library's own load-vector builder), resident on the device before timing
    probe = make(pkg.HELM_MIXED)
    F_host = probe.rhs_gaussian(sigma).pin_memory()
    probe.close()
    F = F_host.to(dev)
    x = torch.empty_like(F)

    def step(prec, host=False, xh=None):
        s = make(prec)
        if host:
            r = s.solve_host(F_host, xh)
        else:
            _, r = s.solve(F, x)
        kern = s.setup_kernels + r.kernels
        s.close()
        return r, kern

    def timed(prec, K, W, host=False):
        xh = torch.empty_like(F_host).pin_memory() if host else None
        for _ in range(W):
            step(prec, host, xh)
        barrier(dist, torch)
        times, results, kernels = [], [], 0
        for _ in range(K):
            flush.fill_(1.0)                       # evict L2 (untimed)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r, kern = step(prec, host, xh)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            results.append(r)
            kernels += kern
        barrier(dist, torch)
        return times, results, kernels

    with ClockSampler(local) as clk:
        t_mixed, r_mixed, kern_mixed = timed(pkg.HELM_MIXED, args.steps, args.warmup)
    clocks = clk.summary()
    t_e2e, r_e2e, _ = timed(pkg.HELM_MIXED, max(1, args.steps // 2), 1, host=True)
    fp64_steps = max(1, args.steps // 2)
    t_fp64, r_fp64, _ = timed(pkg.HELM_FP64, fp64_steps, 1)

    total = max_over_ranks(sum(t_mixed), dist, dev)
    value = world * len(t_mixed) / total
    e2e_total = max_over_ranks(sum(t_e2e), dist, dev)
    fp64_total = max_over_ranks(sum(t_fp64), dist, dev)

    # solve-only rate (factor reused across right-hand sides) and the kernel profile
    s = make(pkg.HELM_MIXED)
    setup_ms_mixed = s.setup_ms
    s.solve(F, x)
    solve_ms = []
    for _ in range(max(3, args.steps)):
        flush.fill_(1.0)
        _, r = s.solve(F, x)
        solve_ms.append(r.solve_ms)
    s.set_profiling(True)
    _, rp = s.solve(F, x)
    prof = s.profile()
    s.set_profiling(False)
    s.close()
    s64 = make(pkg.HELM_FP64)
    setup_ms_fp64 = s64.setup_ms
    _, r64 = s64.solve(F, x)
    s64.close()

    if rank != 0:
        return

    # roofline of the dominant kernel (coarse triangular solves), from CUDA events inside the solve
    dom = max(prof, key=lambda k: prof[k][0])
    hbm, peak_kind = peaks()
    Wc = WL.n // 2 + 1
    bytes_coarse = (2 * Wc - 1) * Wc * Wc * 8           # complex64 inverse blocks streamed once per sweep
    phase_ms = {k: v[0] / max(v[1], 1) for k, v in prof.items()}
    achieved = bytes_coarse / (phase_ms["coarse_solve"] * 1e-3) / 1e9
    traffic = None
    try:
        import re
        with open(os.path.join(ROOT, "profiles", "coarse_solve_p1_n512.md")) as f:
            m = re.search(r"traffic_bytes_per_launch:\s*(\d+)", f.read())
        traffic = int(m.group(1)) if m else None
    except Exception:
        pass

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_baseline(n_iters=30)
        cpu.pop("seconds_per_solve", None)

    lat = sorted(t * 1e3 for t in t_mixed)
    p99 = lat[min(len(lat) - 1, math.ceil(0.99 * len(lat)) - 1)]
    n = WL.num_dofs
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(t_mixed),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": workload_config("complex64 V-cycle in complex128 FGMRES"),
        "p50_ms": statistics.median(lat),
        "p99_ms": p99,
        "iters": r_mixed[-1].iters,
        "relres_true": r_mixed[-1].relres_true,
        "setup_ms": setup_ms_mixed,
        "solve_only": {"solves_per_s": 1e3 / statistics.median(solve_ms), "solve_ms": statistics.median(solve_ms),
                       "note": "same operator, new right-hand side: factor reused"},
        "fp64": {"value": world * len(t_fp64) / fp64_total, "unit": "solves/s", "iters": r64.iters,
                 "relres_true": r64.relres_true, "setup_ms": setup_ms_fp64, "solve_ms": r64.solve_ms,
                 "mixed_speedup": value / (world * len(t_fp64) / fp64_total)},
        "phase_ms_per_iteration": phase_ms,
        "roofline": {"kernel": "k_coarse_solve<float> (" + dom + " dominant)", "bound": "hbm",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "peak_kind": peak_kind, "traffic": traffic,
                     "algorithmic_bytes": bytes_coarse},
        "cpu_baseline": cpu,
        "e2e": {"value": world * len(t_e2e) / e2e_total, "unit": "solves/s",
                "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 16 * n},
        "gpu_launches": kern_mixed,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_kernel(args):
    """Repeated launches of one hot-path step on the bench workload (for ncu captures)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2104_01439_gb300 as pkg
    prec = pkg.HELM_FP64 if args.fp64 else pkg.HELM_MIXED
    s = pkg.Solver(WL.k, WL.n, WL.order, WL.shift, restart=WL.restart, tol=WL.tol, precision=prec)
    g = torch.Generator().manual_seed(0)
    if args.kernel == "coarse":
        v = torch.randn(s.num_coarse_dofs, dtype=torch.complex128, generator=g).cuda()
        for _ in range(args.steps):
            s.coarse_solve(v)
    elif args.kernel == "vcycle":
        v = torch.randn(s.num_dofs, dtype=torch.complex128, generator=g).cuda()
        for _ in range(args.steps):
            s.vcycle(v)
    elif args.kernel == "apply":
        v = torch.randn(s.num_dofs, dtype=torch.complex128, generator=g).cuda()
        for _ in range(args.steps):
            s.apply(v, 0)
    else:   # a full solve
        F = s.rhs_gaussian(2.0 / WL.n).cuda()
        for _ in range(args.steps):
            s.solve(F)
    torch.cuda.synchronize()
    s.close()
    print(f"ran {args.steps} x {args.kernel}", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", choices=["coarse", "vcycle", "apply", "solve"],
                    help="only launch one hot-path step --steps times (profiling aid)")
    ap.add_argument("--fp64", action="store_true", help="with --kernel: the all-FP64 form")
    args = ap.parse_args()
    if args.kernel:
        run_kernel(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
