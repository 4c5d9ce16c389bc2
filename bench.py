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
import tempfile
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

COARSE_TRAFFIC_BYTES = 235.9e6   # ncu DRAM bytes of one coarse solve (the coarse-solve summary under profiles/)

# stencil kernels at a size above L2: 2D P1, h = 1/4096 (16.8 M DoFs; one complex128
# vector is 268 MB, twice the 129 MB L2), same kh and shift exponent as the solve workload
STENCIL_N = 4096
STENCIL_NU = 4


def stencil_bytes_per_dof(nu, mixed):
    """Algorithmic bytes per DoF of helm_apply and of nu smoothing sweeps from u = 0 (2D).

    apply: read x, write y (complex128): 32 B.
    smoother: the sweeps run fused on shared-memory tiles (one kernel), so the operation's own
    traffic is all it moves: read f (complex128, 16 B) and write u^nu (complex128, 16 B),
    32 B in both precisions (the complex64 form converts on the way in and out)."""
    return {"apply": 32, "smooth": 32, "kernels": 1}


def stencil_hbm(pkg, stream, dev, hbm, peak_kind, reps=20):
    """CUDA-event times of helm_apply (A0, complex128) and of STENCIL_NU smoothing sweeps on
    A_eps at h = 1/STENCIL_N, inputs resident and larger than L2 (no flush needed)."""
    import torch
    k = WL.k * STENCIL_N / WL.n
    shift = k ** (math.log(WL.shift) / math.log(WL.k))
    out = {"workload": f"2D P1, h=1/{STENCIL_N}, k={k:g}, eps=k^{math.log(WL.shift) / math.log(WL.k):.3f}",
           "peak": hbm, "peak_kind": peak_kind, "l2": "each vector 2x L2; no flush"}
    g = torch.Generator(device=dev).manual_seed(3)
    for prec, name in ((pkg.HELM_MIXED, "mixed"), (pkg.HELM_FP64, "fp64")):
        s = pkg.Solver(k, STENCIL_N, 1, shift, precision=prec, stream=stream, operator_only=True)
        N = s.num_dofs
        x = torch.randn(N, dtype=torch.complex128, device=dev, generator=g)
        y = torch.empty_like(x)
        bpd = stencil_bytes_per_dof(STENCIL_NU, prec == pkg.HELM_MIXED)
        for label, fn, b in (("apply_A0", lambda: s.apply(x, 0, y), bpd["apply"]),
                             (f"smooth_nu{STENCIL_NU}", lambda: s.smooth(x, STENCIL_NU, y), bpd["smooth"])):
            if prec == pkg.HELM_FP64 and label == "apply_A0":
                continue   # the outer apply is complex128 in both forms
            for _ in range(3):
                fn()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = b * N / (ms * 1e-3) / 1e9
            key = label if label == "apply_A0" else f"{label}_{name}"
            out[key] = {"ms": ms, "GBs": gbs, "frac": gbs / hbm, "bytes_per_dof": b, "dofs": N,
                        "kernels_per_call": 1 if label == "apply_A0" else bpd["kernels"]}
        s.close()
        del x, y
    return out

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
        self.path = os.path.join(tempfile.gettempdir(), f"helm_clocks_{os.getpid()}.csv")

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
        import torch
        import torch.distributed as dist
        # one process per GPU over NCCL; gloo where there is no GPU (CPU tests of this path)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local, dist


def max_over_ranks(x, dist, device):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, torch):
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def replica_rate(units_per_rank, seconds, dist, device):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest rank's time."""
    world = dist.get_world_size() if dist is not None else 1
    return world * units_per_rank / max_over_ranks(seconds, dist, device)


# ---------------------------------------------------------------------------- CPU oracle leg

_ONE_THREAD = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}


def _oracle_full_solve(want_x):
    """One full oracle solve of the workload (assembly, sparse LU of the coarse matrix, FGMRES
    to relres 1e-8: every iteration, nothing extrapolated), in a spawned worker process."""
    sys.path.insert(0, ROOT)
    from oracle import solver
    t0 = time.perf_counter()
    pb = solver.build_problem(WL)
    r = pb.solve()
    t1 = time.perf_counter()
    return {"seconds": t1 - t0, "iters": r.iters, "relres": r.relres_true, "x": r.x if want_x else None}


def host_info():
    """Host cores and CPU model (lscpu when present)."""
    ncpu = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Vendor ID") and ":" in line:
                model = (model + " / " if model else "") + line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return ncpu, model or platform.processor() or platform.machine()


def oracle_pool_run(n_solves, procs, warm=0, want_x=False):
    """n_solves full oracle solves on `procs` single-threaded processes (spawned; a process
    pool forked after GPU work could hang). Returns the wall time of the n_solves (after `warm`
    untimed ones on the same pool) and each solve's own record."""
    old = {k: os.environ.get(k) for k in _ONE_THREAD}
    os.environ.update(_ONE_THREAD)
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs) as pool:
            if warm:
                pool.map(_oracle_full_solve, [False] * warm, chunksize=1)
            t0 = time.perf_counter()
            recs = pool.map(_oracle_full_solve, [want_x and i == 0 for i in range(n_solves)], chunksize=1)
            wall = time.perf_counter() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return wall, recs


def oracle_baseline(want_x=False):
    """The oracle timed on the host cores: one full solve per process, one process per core
    (at most 16), all at once. value = solves / wall time; the one-core rate is 1 / the
    median solve's own time."""
    ncpu, model = host_info()
    procs = max(1, min(16, ncpu))
    wall, recs = oracle_pool_run(procs, procs, want_x=want_x)
    per = statistics.median(r["seconds"] for r in recs)
    out = {
        "value": len(recs) / wall, "unit": "solves/s", "cores": procs, "kind": "oracle",
        "sample": f"{len(recs)} full oracle solves of this workload at once (numpy/scipy, one thread each: "
                  f"assembly, sparse LU, all {recs[0]['iters']} FGMRES iterations; nothing extrapolated), "
                  f"{wall:.1f} s wall",
        "single_core": {"value": 1.0 / per, "unit": "solves/s", "seconds_per_solve": per},
        "nproc": ncpu, "cpu_model": model,
        "iters": recs[0]["iters"], "relres_true": recs[0]["relres"],
    }
    return out, recs[0]["x"]


def run_reference(args):
    world, rank, local, dist = dist_setup()
    if rank != 0:
        return
    ncpu, model = host_info()
    procs = max(1, min(16, ncpu, max(args.steps, args.warmup)))
    wall, recs = oracle_pool_run(args.steps, procs, warm=args.warmup)
    v = len(recs) / wall
    per = statistics.median(r["seconds"] for r in recs)
    cpu = {"value": v, "unit": "solves/s", "cores": min(procs, len(recs)), "kind": "oracle",
           "sample": f"{len(recs)} full oracle solves (numpy/scipy, one thread each, {procs} processes: assembly, "
                     f"sparse LU, all {recs[0]['iters']} FGMRES iterations; nothing extrapolated) after "
                     f"{args.warmup} untimed ones",
           "single_core": {"value": 1.0 / per, "unit": "solves/s", "seconds_per_solve": per},
           "nproc": ncpu, "cpu_model": model}
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / len(recs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config("FP64 oracle (CPU)"),
        "iters": recs[0]["iters"], "relres_true": recs[0]["relres"],
        "cpu_baseline": cpu,
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
    value = replica_rate(len(t_mixed), sum(t_mixed), dist, dev)
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
    x_mixed = x.cpu().numpy()
    s.set_profiling(True)
    _, rp = s.solve(F, x)
    prof = s.profile()
    s.set_profiling(False)
    reuse_mixed = (s.factored_blocks, s.reused_blocks)
    s.close()
    s64 = make(pkg.HELM_FP64)
    setup_ms_fp64 = s64.setup_ms
    _, r64 = s64.solve(F, x)
    x_fp64 = x.cpu().numpy()
    reuse_fp64 = (s64.factored_blocks, s64.reused_blocks)
    s64.close()

    if rank != 0:
        return
    hbm, peak_kind = peaks()
    stencil_large = stencil_hbm(pkg, stream, dev, hbm, peak_kind)

    # roofline of the dominant phase (the coarse solve: block pre-pass, segment chains, segment
    # fix-ups, middle block), from CUDA events inside the solve: algorithmic bytes = the banded
    # LU's two triangular factors read once, 2 b 8 B per coarse DoF (complex64, b = W_c + 1),
    # i.e. (2 W_c - 1) W_c^2 8 B for the 2D P1 coarse grid
    dom = max(prof, key=lambda k: prof[k][0])
    Wc = WL.n // 2 + 1
    bytes_coarse = (2 * Wc - 1) * Wc * Wc * 8
    phase_ms = {k: v[0] / max(v[1], 1) for k, v in prof.items()}
    achieved = bytes_coarse / (phase_ms["coarse_solve"] * 1e-3) / 1e9
    # DRAM bytes of one coarse solve at this workload (dram__bytes_read.sum + dram__bytes_write.sum
    # of k_block_gemv, the four k_seg_chain launches, the two k_seg_fixup launches and k_seg_middle,
    # one-pass ncu capture of `bench.py --kernel coarse`): the distinct inverses, couplings and
    # segment products read once each (repeated blocks of converged chains come from L2)
    traffic = COARSE_TRAFFIC_BYTES
    # stencil kernels: outer apply reads z and writes w (32 B/DoF, complex128); the fine level of
    # the V-cycle moves >= 52 B/DoF (read v_j 16, u 8 + 8, write z_j 16, transfers ~4)
    n_f = WL.num_dofs
    stencil = {
        "apply_A0_GBs": 32 * n_f / (phase_ms["apply_A0"] * 1e-3) / 1e9,
        "vcycle_fine_GBs": 52 * n_f / ((phase_ms["vcycle_pre_restrict"] + phase_ms["vcycle_prolong_post"]) * 1e-3)
        / 1e9,
        "peak_GBs": hbm,
        "note": "algorithmic bytes / CUDA-event phase time inside the solve; the vectors are L2-resident "
                "at this size and the phases include launch gaps",
        "above_l2": stencil_large,
    }

    cpu, x_orc = None, None
    if not args.no_cpu_baseline and world == 1:
        cpu, x_orc = oracle_baseline(want_x=True)

    def accuracy(xg, r):
        """This result against the FP64 oracle's solution of the same problem (Sec. 4 FGMRES)."""
        out = {"iters": r.iters, "relres_true": r.relres_true, "relres_givens": r.relres_est,
               # |Givens estimate - true residual| at the last cycle's end: zero when the Arnoldi
               # relation A0 Z = V Hbar holds with an orthonormal V, so it measures both at once
               "residual_gap": abs(r.relres_est - r.relres_true) / r.relres_true if r.relres_true else None}
        if x_orc is not None:
            import numpy as np
            out["x_rel_err_vs_oracle"] = float(np.linalg.norm(xg - x_orc) / np.linalg.norm(x_orc))
            out["iters_minus_oracle"] = r.iters - cpu["iters"]
        return out

    legs = {}
    if world == 1 and not args.no_legs:
        with ClockSampler(local) as ck:
            legs["sweep"] = sweep_leg(pkg, args.pairs, args.max_n, args.fp64_samples, args.max_active)
        legs["sweep"]["clocks"] = ck.summary()
        with ClockSampler(local) as ck:
            legs["serve"] = serve_leg(pkg, args.requests, args.rate, tuple(int(g) for g in args.grids.split(",")),
                                      args.max_active)
        legs["serve"]["clocks"] = ck.summary()
        with ClockSampler(local) as ck:
            legs["qp_wedge"] = qp_leg(pkg)
        legs["qp_wedge"]["clocks"] = ck.summary()

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
        "accuracy": {"mixed": accuracy(x_mixed, r), "fp64": accuracy(x_fp64, r64),
                     "note": "complex64 V-cycle with double-float (~48-bit) Arnoldi basis, second Gram-Schmidt "
                             "pass and coarse factor, first-pass projections in float (mixed); complex128 "
                             "throughout except the double-float Gram-Schmidt (fp64)"},
        "coarse_factor": {"mixed": {"factored_blocks": reuse_mixed[0], "reused_blocks": reuse_mixed[1]},
                          "fp64": {"factored_blocks": reuse_fp64[0], "reused_blocks": reuse_fp64[1]}},
        "phase_ms_per_iteration": phase_ms,
        "stencil": stencil,
        "roofline": {"kernel": "coarse solve phase: k_block_gemv + 4 k_seg_chain + 2 k_seg_fixup + k_seg_middle ("
                               + dom + " dominant)", "bound": "hbm",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "peak_kind": peak_kind, "traffic": traffic,
                     "algorithmic_bytes": bytes_coarse},
        "cpu_baseline": cpu,
        "e2e": {"value": world * len(t_e2e) / e2e_total, "unit": "solves/s",
                "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 16 * n},
        "gpu_launches": kern_mixed,
        "clocks": clocks,
    }
    line.update(legs)
    print(json.dumps(line), flush=True)


def _host_load(req, pkg, seed):
    import torch
    return torch.from_numpy(hi.random_load(pkg.num_dofs(req), seed))


def sweep_leg(pkg, n_pairs, max_n, fp64_samples, max_active):
    """Batched shift sweep: (k, kh) pairs x 16 shifts on a log grid in [0.05 k^2, 2 k^2], 2D P1,
    plane wave, restart 50, cap 500. Mixed precision through the request server (all samples
    in flight together) against the plain FP64 form solved one problem at a time."""
    import torch
    from paper_2104_01439_gb300 import sweep
    wls = [w for w in hi.shift_sweep(seed=4) if w.n <= max_n][: 16 * n_pairs]
    samples = [sweep.Sample(w.k, w.n, w.shift) for w in wls]
    pairs = len({(s.k, s.n) for s in samples})
    sweep.run_sweep(samples[:2], max_active=2)   # warm-up (library load, first-launch costs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = sweep.run_sweep(samples, theta=0.3, restart=50, maxit=500, precision=pkg.HELM_MIXED,
                          budget_bytes=150 << 30, max_active=max_active)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    # plain FP64 per-solve form on a bounded prefix of the same samples
    nf = min(len(samples), fp64_samples)
    t1 = time.perf_counter()
    it64 = []
    for smp in samples[:nf]:
        slv = pkg.Solver(smp.k, smp.n, 1, smp.shift, restart=50, maxit=500, tol=1e-8, precision=pkg.HELM_FP64)
        F = slv.rhs_planewave(0.3).cuda()
        _, r = slv.solve(F)
        it64.append(r.iters)
        slv.close()
    torch.cuda.synchronize()
    wall64 = time.perf_counter() - t1
    best = sweep.best_shifts(res)
    params, loss = sweep.fit_shift_map([b.sample.k for b in best], [b.sample.ell for b in best],
                                       [b.sample.sigma for b in best])
    v, v64 = len(samples) / wall, nf / wall64
    return {
        "workload": f"shift sweep: {pairs} (k, kh) pairs (k~U[10,300], kh~U[0.3,0.8], seed 4, n <= {max_n}) "
                    f"x 16 shifts log-spaced in [0.05k^2, 2k^2], 2D P1, plane wave theta=0.3, FGMRES(50) "
                    f"cap 500, relres 1e-8; all samples through the request server (complex64 V-cycle, "
                    f"max_active={max_active}, budget 150 GB), setup included",
        "value": v, "unit": "solves/s", "wall_s": wall, "solves": len(samples),
        "iters": {"min": min(r.iters for r in res), "max": max(r.iters for r in res),
                  "mean": statistics.mean(r.iters for r in res),
                  "capped": sum(r.status != "converged" for r in res)},
        "fp64_per_solve": {"value": v64, "unit": "solves/s", "samples": nf,
                           "iters_equal_to_mixed": sum(a == r.iters for a, r in zip(it64, res[:nf])),
                           "batched_mixed_speedup": v / v64},
        "best_shift_fit": {"params": [float(x) for x in params], "loss": loss, "points": len(best)},
    }


def wedge_k(k_max, n, dim=2):
    """k = k_max mu(x) of the wedge profile at the element centres of an n^dim tensor mesh, in
    the element order helm_setup_het takes (cells lexicographic, x fastest)."""
    import numpy as np
    c = (np.arange(n) + 0.5) / n
    xs = np.stack(np.meshgrid(*([c] * dim), indexing="ij")[::-1], axis=-1).reshape(-1, dim)
    return k_max * hi.wedge_profile(xs)


def qp_leg(pkg, k_max=100.0, steps=2):
    """The paper's own elements and smoother on its wedge-type problem (Sec. 6, Sec. 7): Q_p,
    p = 1, 2, 3 (helm_setup_het, HELM_TENSOR) with about 263k DoFs each, k(x) = k_max mu(x) on
    the synthetic wedge, V(3,3) with omega = 2/3, the shift eps = k_max^sigma from the paper's
    fitted map (Table tab:optweights at k_max and l = log2 n), the point source of Sec. 6,
    FGMRES(50) to relres 1e-8. setup + solve per step, mixed and FP64."""
    import math as _m
    import torch
    from paper_2104_01439_gb300 import sweep
    out = {"workload": f"2D Q_p wedge, k_max={k_max:g}, V(3,3) omega=2/3, eps from the fitted map, point "
                       f"source, FGMRES(50), relres 1e-8; setup + solve per step"}
    for p, n in ((1, 512), (2, 256), (3, 170)):
        eps = sweep.shift_of(sweep.PAPER_SHIFT_WEIGHTS[p], k_max, n)
        kf, kc = wedge_k(k_max, n), wedge_k(k_max, n // 2)
        row = {"n": n, "dofs": (p * n + 1) ** 2, "eps": eps}
        for prec, name in ((pkg.HELM_MIXED, "mixed"), (pkg.HELM_FP64, "fp64")):
            def step():
                s = pkg.Solver(k_max, n, p, eps, elements=pkg.HELM_TENSOR, k_fine=kf, k_coarse=kc, omega=2.0 / 3.0,
                               nu=3, restart=50, maxit=500, tol=1e-8, precision=prec)
                F = s.rhs_source().cuda()
                _, r = s.solve(F)
                setup = s.setup_ms
                s.close()
                return r, setup
            step()                                 # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                r, setup = step()
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / steps
            row[name] = {"solves_per_s": 1.0 / dt, "iters": r.iters, "relres_true": r.relres_true,
                         "status": r.status, "setup_ms": setup}
        out[f"q{p}"] = row
    return out


def run_sweep_bench(args):
    import __graft_entry__
    __graft_entry__.build()
    import paper_2104_01439_gb300 as pkg
    leg = sweep_leg(pkg, args.pairs, args.max_n, args.fp64_samples, args.max_active)
    line = {
        "metric": METRIC, "value": leg["value"], "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": 1e3 * leg["wall_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": leg["workload"], "step": "all samples of the sweep", "parallelism": "request server"},
        "sweep": leg,
    }
    print(json.dumps(line), flush=True)


def serve_leg(pkg, requests, rate, grids, max_active):
    """Serving loop: Poisson arrivals, P1/P2 50/50, n from the grid set, k~U[20,400],
    eps = k^sigma_p(k, log2 n) from the shift map (the paper's printed weights), random
    N(0,1) complex load vectors, 150 GB budget. p50/p99 latency and solves/s, mixed vs FP64."""
    from paper_2104_01439_gb300 import sweep
    arr = hi.poisson_arrivals(seed=5, rate=rate, count=requests)
    reqs = hi.serving_requests(seed=5, count=requests, grids=grids)
    out = {}
    for prec, name in ((pkg.HELM_MIXED, "mixed"), (pkg.HELM_FP64, "fp64")):
        rq = []
        for (order, n, k, seed) in reqs:
            eps = sweep.shift_of(sweep.PAPER_SHIFT_WEIGHTS[order], k, n)
            r = pkg.make_request(k, n, order, eps, restart=50, maxit=500, tol=1e-8, precision=prec)
            rq.append((r, _host_load(r, pkg, seed)))
        with pkg.Server(150 << 30, max_active) as srv:
            srv.submit(*rq[0])   # warm-up request (first-launch costs), not counted
            srv.drain()
            t0 = time.perf_counter()
            tickets = []
            for (r, F), ta in zip(rq, arr):
                dt = t0 + ta - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets.append(srv.submit(r, F))
            infos = [srv.wait(t) for t in tickets]
            wall = time.perf_counter() - t0
        lat = sorted(i.latency * 1e3 for i in infos)
        ok = [i for i in infos if i.rc == 0]
        out[name] = {"solves_per_s": len(ok) / wall, "p50_ms": statistics.median(lat),
                     "p99_ms": lat[min(len(lat) - 1, math.ceil(0.99 * len(lat)) - 1)], "makespan_s": wall,
                     "failed": len(infos) - len(ok), "capped": sum(i.result.status != "converged" for i in ok),
                     "mean_iters": statistics.mean(i.result.iters for i in ok) if ok else None}
    return {
        "workload": f"serving trace: {requests} requests, Poisson arrivals {rate:g}/s (seed 5), P1/P2 50/50, "
                    f"n in {list(grids)}, k~U[20,400], eps from the paper's shift map, random N(0,1) complex "
                    f"load, FGMRES(50) cap 500, relres 1e-8; request server (max_active={max_active}, "
                    f"budget 150 GB), setup included",
        "value": out["mixed"]["solves_per_s"], "unit": "solves/s",
        "p50_ms": out["mixed"]["p50_ms"], "p99_ms": out["mixed"]["p99_ms"],
        "mixed": out["mixed"], "fp64": out["fp64"],
        "mixed_vs_fp64": out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"],
    }


def run_serve_bench(args):
    import __graft_entry__
    __graft_entry__.build()
    import paper_2104_01439_gb300 as pkg
    leg = serve_leg(pkg, args.requests, args.rate, tuple(int(g) for g in args.grids.split(",")), args.max_active)
    line = {
        "metric": METRIC, "value": leg["value"], "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": 1e3 * leg["mixed"]["makespan_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": leg["workload"], "step": "whole trace", "parallelism": "request server"},
        "p50_ms": leg["p50_ms"], "p99_ms": leg["p99_ms"], "serve": leg,
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
    elif args.kernel == "stencil":   # apply and smoother at h = 1/STENCIL_N (above L2)
        s.close()
        k = WL.k * STENCIL_N / WL.n
        s = pkg.Solver(k, STENCIL_N, 1, k ** (math.log(WL.shift) / math.log(WL.k)), precision=prec,
                       operator_only=True)
        v = torch.randn(s.num_dofs, dtype=torch.complex128, generator=g).cuda()
        y = torch.empty_like(v)
        for _ in range(args.steps):
            s.apply(v, 0, y)
            s.smooth(v, STENCIL_NU, y)
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
    ap.add_argument("--no-legs", action="store_true", help="skip the sweep and serve legs of the default line")
    ap.add_argument("--kernel", choices=["coarse", "vcycle", "apply", "stencil", "solve"],
                    help="only launch one hot-path step --steps times (profiling aid)")
    ap.add_argument("--fp64", action="store_true", help="with --kernel: the all-FP64 form")
    ap.add_argument("--workload", default="solve", choices=["solve", "sweep", "serve", "qp"],
                    help="solve: the headline step (default); sweep: batched shift sweep; serve: serving trace; "
                         "qp: Q1-Q3 on the heterogeneous wedge")
    ap.add_argument("--pairs", type=int, default=8, help="sweep: (k, kh) pairs (x 16 shifts)")
    ap.add_argument("--max-n", type=int, default=256, help="sweep: keep pairs whose mesh has n <= this")
    ap.add_argument("--fp64-samples", type=int, default=32, help="sweep: samples of the FP64 per-solve form")
    ap.add_argument("--max-active", type=int, default=16, help="sweep/serve: requests in flight")
    ap.add_argument("--requests", type=int, default=120, help="serve: requests in the trace")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: mean arrival rate (1/s)")
    ap.add_argument("--grids", default="128,256,512", help="serve: mesh sizes n of the trace")
    args = ap.parse_args()
    if args.kernel:
        run_kernel(args)
    elif args.workload == "sweep":
        run_sweep_bench(args)
    elif args.workload == "serve":
        run_serve_bench(args)
    elif args.workload == "qp":
        import __graft_entry__
        __graft_entry__.build()
        import paper_2104_01439_gb300 as pkg
        print(json.dumps({"metric": METRIC, "qp_wedge": qp_leg(pkg)}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
