"""Benchmark: reproducible PBiCGStab iterations per second on one GB300.

Workload (one step = one full solve): 3D Poisson 7-point on a 256^3 grid
(n = 16,777,216, nnz = 117,047,296), CSR binary64, b = A*1, x0 = 0, Jacobi,
classic reproducible PBiCGStab (Fig. 2) with exact dots, stop at relative
residual 1e-10. Inputs are synthetic (seeded generator) and resident in HBM
when the timed region starts; the 1.8 GB matrix is larger than the 129 MB L2,
so no flush is needed between steps.

The JSON line also carries: `e2e` (the same solve through the C ABI from pinned
host buffers, copies inside the timed region), `roofline` for the dominant
kernel (SpMV + dot epilogue, CUDA events inside the library over the timed
steps), `cpu_baseline` (the CPU oracle on a bounded sample), the plain
non-reproducible comparator and the pipelined variant on the same workload,
and the standalone exact-dot and SpMV kernel throughputs.

`--impl reference` times the CPU oracle (this method has no other reference
implementation) on the same workload, a bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID = 256  # --grid changes it for profiling runs only; the headline is 256^3
TOL = 1e-10
MAXIT = 20000
METRIC = "reproducible PBiCGStab iters/s"
UNIT = "iters/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _workload_config(A):
    return {"workload": f"poisson3d_7pt_{GRID}^3 classic reproducible PBiCGStab, Jacobi, "
                        f"b=A*1, x0=0, tol={TOL:g}",
            "n": int(A.n), "nnz": int(A.nnz), "grid": GRID, "variant": "classic",
            "tol": TOL, "dots": "exact, rounded once",
            "l2": "inputs larger than L2 (1.8 GB CSR + vectors), no flush"}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""
        else:
            self.out = ""

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_model():
    import platform
    impl = part = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":", 1)[0].strip().lower()
            if key in ("model name", "cpu model"):
                return line.split(":", 1)[1].strip()
            if key == "cpu implementer":
                impl = line.split(":", 1)[1].strip()
            if key == "cpu part":
                part = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if part:
        return f"{platform.machine()} (CPU implementer {impl}, part {part})"
    return platform.machine()


def _cpu_baseline(A, b, iters=2):
    """The CPU oracle on a bounded sample of the benchmark solve (set-up and the
    first iterations): on all host cores (the threaded oracle: rows split over
    threads, exact dots merged as integers, bitwise the one-thread result) and
    on one thread."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    legs = {}
    for T, its in ((cores, 4 * iters), (1, iters)):
        oracle.set_threads(T)
        t = time.perf_counter()
        o = oracle.solve(A, b, tol=TOL, maxit=its, variant=0, history=False)
        legs[T] = (o["iters"], time.perf_counter() - t)
    oracle.set_threads(1)
    (ia, da), (i1, d1) = legs[cores], legs[1]
    return {"value": ia / da, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu": _cpu_model(),
            "sample": f"set-up + {ia} classic iterations of the same {GRID}^3 solve, threaded C oracle on "
                      f"{cores} threads ({da:.1f} s)",
            "single_thread": {"value": i1 / d1, "unit": UNIT, "cores": 1,
                              "sample": f"set-up + {i1} iterations, one thread ({d1:.1f} s)"}}


def run_reference(args):
    """The reference arm: the CPU oracle (this method has no other
    implementation to run) on the host cores, the same workload; each step a
    bounded sample of it (set-up and one iteration)."""
    world, rank, _ = _dist()
    if world > 1 and rank != 0:
        return 0
    from paper_2302_04180_gb300 import gen
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    A = gen.poisson3d(GRID)
    b = oracle.spmv(A, np.ones(A.n))
    per = 1
    for _ in range(args.warmup):
        oracle.solve(A, b, tol=TOL, maxit=per, variant=0, history=False)
    t = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        its += oracle.solve(A, b, tol=TOL, maxit=per, variant=0, history=False)["iters"]
    dt = time.perf_counter() - t
    v = its / dt
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _workload_config(A),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": _cpu_model(),
                             "sample": f"per step: set-up + {per} classic iteration of the "
                                       f"{GRID}^3 solve, threaded C oracle on {cores} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    import __graft_entry__ as ge
    ge.build()
    import paper_2302_04180_gb300 as rbs
    from paper_2302_04180_gb300 import gen

    A = gen.poisson3d(GRID)
    Ad = rbs.to_device(A, dev)
    ones = torch.ones(A.n, dtype=torch.float64, device=dev)
    b = rbs.rbs_spmv_csr(Ad, ones)
    x = torch.empty(A.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    loop_mode = 1 if args.loop == "host" else 0

    def solve(variant=0, dot_mode=0, profile=False, history=False):
        return rbs.rbs_solve(Ad, b, tol=TOL, maxit=MAXIT, variant=variant, x_out=x,
                             dot_mode=dot_mode, profile=profile, history=history,
                             loop_mode=loop_mode)

    for _ in range(args.warmup):
        r0 = solve()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    prof_tot = {}
    iters = 0
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            r = solve(profile=True)
            iters += r["iters"]
            for k, (nl, ms) in r["prof"].items():
                a = prof_tot.setdefault(k, [0, 0.0])
                a[0] += nl
                a[1] += ms
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0
    value = world * iters / (ms * 1e-3)
    clocks = clk.summary()

    roofline = _roofline(A, prof_tot)

    if not args.extras:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": _workload_config(A), "clocks": clocks,
                "roofline": roofline, "gpu_launches": sum(v[0] for v in prof_tot.values())}
        print(json.dumps(line), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # e2e: the same solve through the C ABI from pinned host buffers
    rp = torch.from_numpy(A.rowptr).pin_memory()
    cl = torch.from_numpy(A.col).pin_memory()
    vl = torch.from_numpy(A.val).pin_memory()
    bh = b.cpu().pin_memory()
    xh = torch.empty(A.n, dtype=torch.float64).pin_memory()
    Ah = rbs.DeviceCSR(A.n, rp, cl, vl)
    rbs.rbs_solve(Ah, bh, tol=TOL, maxit=MAXIT, variant=0, x_out=xh, history=False)
    e2e_steps = max(1, min(args.steps, 3))
    t = time.perf_counter()
    e_iters = 0
    for _ in range(e2e_steps):
        e_iters += rbs.rbs_solve(Ah, bh, tol=TOL, maxit=MAXIT, variant=0, x_out=xh, history=False)["iters"]
    e_dt = time.perf_counter() - t
    h2d = 8 * (A.n + 1) + 4 * A.nnz + 8 * A.nnz + 8 * A.n
    # the copies alone (same bytes, same pinned buffers, one stream): the share
    # of the end-to-end step that is host<->device traffic
    scratch = [torch.empty_like(t_, device=dev) for t_ in (rp, cl, vl, bh)]
    xd = torch.empty(A.n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        for src, dst in zip((rp, cl, vl, bh), scratch):
            dst.copy_(src, non_blocking=True)
        xh.copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
    c_dt = (time.perf_counter() - t) / e2e_steps
    del scratch, xd
    e2e = {"value": world * e_iters / e_dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": 8 * A.n + 4, "path": "rbs_solve on pinned host buffers",
           "s_per_step": e_dt / e2e_steps, "copy_s_per_step": c_dt,
           "copy_GB_per_s": (h2d + 8 * A.n) / c_dt / 1e9}

    # inputs of the exact-dot grid, generated on the host cores while the
    # GPU-bound sections run (the comparator, the pipelined and C3b solves use
    # the device-side graph loop); the sections that depend on host latency
    # (C1, the batch, serving) run after the generators have finished
    import tempfile
    from concurrent.futures import ProcessPoolExecutor
    import multiprocessing as mp
    tmp = tempfile.mkdtemp(prefix="rbs_exdot_")
    cases = [(lg, cond, seed) for lg in EXDOT_LOG2N for cond in EXDOT_CONDS
             for seed in (EXDOT_SEEDS if lg < 27 else (0,))]
    pool = ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4), mp_context=mp.get_context("spawn"))
    futs = {c: pool.submit(_gen_dot_case, c[0], c[1], c[2], tmp) for c in cases}

    plain = _comparator(rbs, Ad, b, x, dev)
    rq_ = solve(variant=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rq_ = solve(variant=1)
    torch.cuda.synchronize()
    pipelined = {"value": rq_["iters"] / (time.perf_counter() - t0), "iters": rq_["iters"],
                 "converged": rq_["converged"]}
    c3b = _c3b(rbs, gen, dev)
    c27 = _c27(rbs, gen, dev)
    kernels = _kernel_micro(rbs, gen, dev, futs)
    pool.shutdown()
    import shutil
    shutil.rmtree(tmp, ignore_errors=True)
    c1 = _c1(rbs, gen, dev)
    batched = _batched(rbs, gen, dev)
    serving = _serving(rbs, gen, dev, rates=(300.0, 600.0, 2000.0))
    gpu_launches = sum(v[0] for v in prof_tot.values())
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**_workload_config(A), "iters_per_solve": r["iters"],
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roofline,
            "plain_comparator": plain,
            "pipelined": pipelined, "c1_poisson16": c1, "c3b_convdiff192": c3b, "stencil27_159": c27,
            "kernels": kernels,
            "batched": batched, "serving": serving}
    if args.cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(A, b.cpu().numpy())
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


DRIFT_ITERS = (1, 10, 50, 100, 200, 400)


def _hex(v):
    return f"{int(np.array([v], dtype=np.float64).view(np.uint64)[0]):016x}"


def _runs(rbs, Ad, b, x, dot_mode, reps, variant=0, tol=TOL):
    """reps solves of one system (graph loop); per run: iterations, tau (hex)
    at DRIFT_ITERS, tau_final and a digest of x (hex), and the wall time."""
    import hashlib
    import torch
    out = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = rbs.rbs_solve(Ad, b, tol=tol, maxit=MAXIT, variant=variant, x_out=x, dot_mode=dot_mode)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        col = 7 if variant == 0 else 8
        taus = {j: _hex(r["hist"][j - 1, col]) for j in DRIFT_ITERS if j <= r["iters"]}
        xd = hashlib.sha256(x.cpu().numpy().tobytes()).hexdigest()[:16]
        out.append({"iters": r["iters"], "tau": taus, "tau_final": _hex(r["tau_final"]), "x": xd,
                    "s": dt, "converged": r["converged"]})
    return out


def _drift_summary(runs):
    pats = {(r["iters"], tuple(sorted(r["tau"].items())), r["tau_final"], r["x"]) for r in runs}
    return {"runs": len(runs), "distinct_results": len(pats),
            "distinct_iters": sorted({r["iters"] for r in runs}),
            "distinct_tau_at": {str(j): len({r["tau"].get(j) for r in runs if j in r["tau"]})
                                for j in DRIFT_ITERS},
            "distinct_x": len({r["x"] for r in runs})}


def _comparator(rbs, Ad, b, x, dev, reps=10):
    """The plain non-reproducible comparator (binary64 dots, atomic
    accumulation across blocks) against the reproducible solve on the same
    workload: both timed as the median of `reps` solves, and the run-to-run
    drift of each (Table 4 style: iteration counts, tau at fixed iterations,
    x). Also on a small system (Poisson 32^3), where the plain dots' block
    order changes more of the rounding."""
    plain = _runs(rbs, Ad, b, x, 1, reps)
    exact = _runs(rbs, Ad, b, x, 0, max(5, reps // 2))
    tp = statistics.median(r["s"] for r in plain)
    te = statistics.median(r["s"] for r in exact)
    ip = statistics.median(r["iters"] for r in plain)
    ie = statistics.median(r["iters"] for r in exact)
    out = {"value": ip / tp, "iters": int(ip), "converged": min(r["converged"] for r in plain),
           "what": "same loop, binary64 dots with atomic accumulation across blocks (non-reproducible)",
           "repro_iters_per_s": ie / te, "repro_over_plain_time": (te / ie) / (tp / ip),
           "repro_over_plain_time_range": [min(r["s"] / r["iters"] for r in exact) /
                                           max(r["s"] / r["iters"] for r in plain),
                                           max(r["s"] / r["iters"] for r in exact) /
                                           min(r["s"] / r["iters"] for r in plain)],
           "timing": f"median of {len(plain)} plain and {len(exact)} reproducible solves (graph loop)",
           "drift": {"plain": _drift_summary(plain), "reproducible": _drift_summary(exact)},
           "runs_plain": [{"iters": r["iters"], "tau": r["tau"], "tau_final": r["tau_final"]} for r in plain],
           "runs_reproducible": [{"iters": r["iters"], "tau": r["tau"], "tau_final": r["tau_final"]}
                                 for r in exact]}
    import torch
    from paper_2302_04180_gb300 import gen
    A32 = gen.poisson3d(32)
    A32d = rbs.to_device(A32, dev)
    b32 = rbs.rbs_spmv_csr(A32d, torch.ones(A32.n, dtype=torch.float64, device=dev))
    x32 = torch.empty(A32.n, dtype=torch.float64, device=dev)
    out["drift_poisson32"] = {"plain": _drift_summary(_runs(rbs, A32d, b32, x32, 1, 20)),
                              "reproducible": _drift_summary(_runs(rbs, A32d, b32, x32, 0, 20))}
    return out


def _roofline(A, prof_tot):
    """Roofline of the dominant kernel -- the SpMV with its exact-dot epilogue,
    classic K1 (<r0,s>) and K3 (<q,y>, <y,y>) -- from the library's CUDA events
    over the timed solves. Only launches that ran are counted (the library
    leaves out those that returned at once on the stop flag). Algorithmic bytes
    per launch: 12 nnz (col + val) + 8 (n+1) (rowptr) + 8 n (x, ideal reuse)
    + 8 n (the companion vector of the dot) + 8 n (output) = 12 nnz + 32 n + 8.
    K4 (x and r updates with <r0,r>, <r,r>) moves 64 n bytes per launch."""
    hbm, peak_kind = _peaks()
    alg = 12 * A.nnz + 32 * A.n + 8
    total_ms = max(sum(t[1] for t in prof_tot.values()), 1e-12)

    def stat(names, byt):
        nl = sum(prof_tot.get(k, [0, 0.0])[0] for k in names)
        ms = sum(prof_tot.get(k, [0, 0.0])[1] for k in names)
        if not nl:
            return None
        us = ms * 1e3 / nl
        gbs = byt / (us * 1e-6) / 1e9
        return {"launches": nl, "avg_launch_us": us, "achieved": gbs, "frac": gbs / hbm,
                "time_share": ms / total_ms, "alg_bytes_per_launch": byt}

    both = stat(["k1_spmv_dot", "k3_spmv_dot2"], alg)
    per = {"K1 SpMV + <r0,s>": stat(["k1_spmv_dot"], alg),
           "K3 SpMV + <q,y>, <y,y>": stat(["k3_spmv_dot2"], alg),
           "K4 x, r + <r0,r>, <r,r>": stat(["k4_vec_dot2"], 64 * A.n),
           "K2, K5 vector updates": stat(["vec"], 44 * A.n)}
    return {"bound": "hbm", "achieved": both["achieved"] if both else None, "peak": hbm, "unit": "GB/s",
            "frac": both["frac"] if both else None, "traffic": _traffic(),
            "kernel": "SpMV + exact-dot epilogue (classic K1 and K3 launches)",
            "alg_bytes_per_launch": alg, "launches": both["launches"] if both else 0,
            "avg_launch_us": both["avg_launch_us"] if both else None,
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
            "per_kernel": per,
            "time_share": {k: round(v[1] / total_ms, 4) for k, v in prof_tot.items() if v[0]}}


def _traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary (None when absent or stale)."""
    p = os.path.join(ROOT, "profiles", "spmv_dot_poisson256_traffic.txt")
    try:
        for line in open(p):
            if line.startswith("dram_bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null", "stale") else float(v)
    except Exception:
        pass
    return None


def _batched(rbs, gen, dev):
    """512 independent convection-diffusion systems (2D/3D, n 1k-300k, Pe 0-50,
    classic/pipelined mix, tol 1e-8) in one persistent cluster launch: timed
    under the default schedule, then autotuned (proxy solves weighted by the
    first solve's iteration counts) and timed under the tuned schedule."""
    import torch
    work = gen.batch_workload(512, seed=0)
    systems = []
    for A, v in work:
        Ad = rbs.to_device(A, dev)
        b = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
        systems.append({"A": Ad, "b": b, "x": torch.empty(A.n, dtype=torch.float64, device=dev),
                        "tol": 1e-8, "maxit": 5000, "variant": v})
    default = {"cluster": 8, "split": 0}

    def timed(schedule):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = rbs.rbs_solve_batched(systems, history=False, schedule=schedule)
        torch.cuda.synchronize()
        return res, time.perf_counter() - t

    first = rbs.rbs_solve_batched(systems, history=False, schedule=default)
    res0, dt0 = timed(default)
    x0s = [r["x"].clone() for r in res0]
    t = time.perf_counter()
    best = rbs.rbs_batch_tune(systems, prev=first, proxy_iters=24)
    tune_s = time.perf_counter() - t
    res, dt = timed({"cluster": best["cluster"], "split": best["split"]})
    same = all(a["iters"] == b["iters"] and bool(torch.equal(a["x"], x)) for a, b, x in zip(res, res0, x0s))
    its = sum(r["iters"] for r in res)
    # algorithmic bytes of the whole batch: per iteration 2 SpMV (12 nnz each)
    # plus the fused vector passes, 216 n bytes classic / 352 n pipelined
    alg = sum(r["iters"] * (24 * A.nnz + (352 if v else 216) * A.n) for r, (A, v) in zip(res, work))
    hbm, _ = _peaks()
    return {"systems": len(systems), "unknowns": int(sum(A.n for A, _ in work)),
            "alg_bytes": int(alg), "achieved_GB/s": alg / dt / 1e9, "frac_of_hbm": alg / dt / 1e9 / hbm,
            "seconds": dt, "systems_per_s": len(systems) / dt, "iters_per_s": its / dt,
            "total_iters": its, "converged": int(sum(r["converged"] for r in res)),
            "schedule": {"cluster": best["cluster"], "split": best["split"]},
            "tuning_seconds": tune_s, "default_schedule": default, "default_seconds": dt0,
            "default_frac_of_hbm": alg / dt0 / 1e9 / hbm,
            "tuned_schedule_differs": (best["cluster"], best["split"]) != (default["cluster"], default["split"]),
            "results_identical_to_default": same}


def _serving(rbs, gen, dev, rates=(100.0, 300.0, 1000.0), count=10000, seed=3):
    """Poisson-arrival solve requests against the per-iteration continuous-
    batching server: a pool of 48 systems (3D upwind convection-diffusion and
    3D Poisson up to 128^3, classic/pipelined mix, tol 1e-8), `count` requests
    per arrival rate. Per rate: p50/p99 latency (submission to completion),
    solves/s, the most systems in flight at once, the pool's peak reserved
    memory, and whether every answer is bitwise the system's solo solve."""
    import torch
    pool = []
    for A, v in gen.serving_pool(48, 0):
        Ad = rbs.to_device(A, dev)
        b = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
        alone = rbs.rbs_solve(Ad, b, tol=1e-8, maxit=3000, variant=v, history=False)
        pool.append((A, Ad, b, v, alone))
    torch.cuda.synchronize()
    out = []
    for rate in rates:
        arr = gen.poisson_arrivals(count, rate, seed)
        picks = (gen.splitmix64(seed + 11, count) % np.uint64(len(pool))).astype(int)
        xs = [torch.empty(pool[p][0].n, dtype=torch.float64, device=dev) for p in range(len(pool))]
        same = True
        lat = []
        with rbs.RbsServer(engines=1, max_active=128, budget_bytes=24 << 30) as srv:
            tk = []
            t0 = time.perf_counter()
            for k in range(count):
                while time.perf_counter() - t0 < arr[k]:
                    time.sleep(0.0001)
                A, Ad, b, v, _ = pool[picks[k]]
                # one output buffer per request in flight; answers are checked as they finish
                sd = {"A": Ad, "b": b, "x": torch.empty(A.n, dtype=torch.float64, device=dev),
                      "tol": 1e-8, "maxit": 3000, "variant": v}
                tk.append((srv.submit(sd), picks[k]))
                while len(tk) > 2048:
                    t, p = tk.pop(0)
                    r = srv.wait(t)
                    lat.append(r["latency_s"])
                    same = same and r["iters"] == pool[p][4]["iters"] and torch.equal(r["x"], pool[p][4]["x"])
            for t, p in tk:
                r = srv.wait(t)
                lat.append(r["latency_s"])
                same = same and r["iters"] == pool[p][4]["iters"] and torch.equal(r["x"], pool[p][4]["x"])
            t1 = time.perf_counter()
            st = srv.stats()
        lat = np.array(lat)
        out.append({"rate_per_s": rate, "requests": count, "solves_per_s": count / (t1 - t0),
                    "p50_ms": float(np.percentile(lat, 50) * 1e3),
                    "p99_ms": float(np.percentile(lat, 99) * 1e3), "identical_to_solo": bool(same),
                    "engine_steps": st["steps"], "peak_in_flight": st["peak_active"],
                    "pool_reserved_peak_MB": st["pool_reserved_peak"] / 2**20})
    return out


EXDOT_LOG2N = (16, 20, 24, 27)
EXDOT_CONDS = (1e0, 1e16, 1e32, 1e48)
EXDOT_SEEDS = (0, 1, 2)


def _gen_dot_case(lg, cond, seed, tmp):
    """(spawned worker) one ill-conditioned dot of the kernel microbenchmark,
    saved as .npy files; returns their paths and the exact value as a string."""
    sys.path.insert(0, ROOT)
    from paper_2302_04180_gb300 import gen
    x, y, exact = gen.ill_conditioned_dot(1 << lg, cond, seed)
    px = os.path.join(tmp, f"x_{lg}_{cond:g}_{seed}.npy")
    py = os.path.join(tmp, f"y_{lg}_{cond:g}_{seed}.npy")
    np.save(px, x)
    np.save(py, y)
    return px, py, None if exact is None else str(exact)


def _kernel_micro(rbs, gen, dev, futs):
    """Standalone exact dot over the n x cond grid (C2a: n = 2^16..2^27, cond
    1 .. 1e48, three seeds below 2^27) with its GB/s and whether each result is
    the exact value rounded once; SpMV on Poisson 128^3 (C2b) and on the
    27-point e-type stencil at 159^3."""
    import torch
    from fractions import Fraction
    out = {}

    def timeit(f, reps=10):
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            f()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    hbm, _ = _peaks()
    grid = []
    o = torch.empty(1, dtype=torch.float64, device=dev)
    for (lg, cond, seed), fu in futs.items():
        px, py, exact = fu.result()
        xt = torch.from_numpy(np.load(px)).to(dev)
        yt = torch.from_numpy(np.load(py)).to(dev)
        os.remove(px)
        os.remove(py)
        n = 1 << lg
        ms = timeit(lambda: rbs.rbs_exdot(xt, yt, o), reps=10 if lg >= 24 else 50)
        got = float(o.item())
        grid.append({"n": n, "cond": cond, "seed": seed, "us": ms * 1e3, "GB/s": 16 * n / (ms * 1e-3) / 1e9,
                     "frac_of_hbm": 16 * n / (ms * 1e-3) / 1e9 / hbm,
                     "matches_exact": None if exact is None else got == float(Fraction(exact))})
        del xt, yt
    out["exdot_grid"] = grid
    out["exdot_grid_all_exact"] = all(g["matches_exact"] is not False for g in grid)
    A = gen.poisson3d(128)
    Ad = rbs.to_device(A, dev)
    xv = torch.from_numpy(gen.random_vector(A.n, 1)).to(dev)
    yv = torch.empty_like(xv)
    ms = timeit(lambda: rbs.rbs_spmv_csr(Ad, xv, yv))
    byt = 12 * A.nnz + 8 * (A.n + 1) + 16 * A.n
    out["spmv_poisson128"] = {"us": ms * 1e3, "GB/s": byt / (ms * 1e-3) / 1e9, "frac_of_hbm": byt / (ms * 1e-3) / 1e9 / hbm}
    del Ad, xv, yv
    # the 27-point e-type stencil at the paper's scalability size (159^3 =
    # 4,019,679 unknowns, 27 nonzeros per interior row: the register-staged
    # long-row schedule)
    A = gen.stencil27(159)
    Ad = rbs.to_device(A, dev)
    xv = torch.from_numpy(gen.random_vector(A.n, 1)).to(dev)
    yv = torch.empty_like(xv)
    ms = timeit(lambda: rbs.rbs_spmv_csr(Ad, xv, yv))
    byt = 12 * A.nnz + 8 * (A.n + 1) + 16 * A.n
    out["spmv_stencil27_159"] = {"us": ms * 1e3, "GB/s": byt / (ms * 1e-3) / 1e9,
                                 "frac_of_hbm": byt / (ms * 1e-3) / 1e9 / hbm}
    return out


def _c1(rbs, gen, dev, reps=30):
    """C1: Poisson 7-point 16^3 (n = 4096), classic, tol 1e-8 -- launch- and
    latency-bound: us per iteration and iterations/s with the device-side
    graph loop and with the host loop."""
    import torch
    A = gen.poisson3d(16)
    Ad = rbs.to_device(A, dev)
    b = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
    x = torch.empty(A.n, dtype=torch.float64, device=dev)
    out = {}
    for name, loop in (("graph_loop", 0), ("host_loop", 1)):
        for _ in range(3):
            r = rbs.rbs_solve(Ad, b, tol=1e-8, maxit=1000, x_out=x, loop_mode=loop, history=False)
        torch.cuda.synchronize()
        t = time.perf_counter()
        its = 0
        for _ in range(reps):
            its += rbs.rbs_solve(Ad, b, tol=1e-8, maxit=1000, x_out=x, loop_mode=loop, history=False)["iters"]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        out[name] = {"iters_per_s": its / dt, "us_per_iter": dt / its * 1e6, "iters": r["iters"],
                     "solves_per_s": reps / dt}
    return out


def _c27(rbs, gen, dev, reps=3):
    """The paper's scalability workload (Sec. 5.2), the 27-point e-type
    stencil, at 159^3 (n = 4,019,679, nnz = 107,171,875): classic and pipelined
    reproducible solves to tol 1e-10, iterations/s and the whole iteration's
    algorithmic bytes against the HBM peak (classic: two SpMV + dot passes of
    12 nnz + 32 n + 8 bytes and 152 n bytes of vector updates; pipelined: two
    SpMV of 12 nnz + 24 n + 8 and 304 n bytes in P1 and P3)."""
    import torch
    A = gen.stencil27(159)
    Ad = rbs.to_device(A, dev)
    b = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
    x = torch.empty(A.n, dtype=torch.float64, device=dev)
    hbm, _ = _peaks()
    per_iter = {"classic": 2 * (12 * A.nnz + 32 * A.n + 8) + 152 * A.n,
                "pipelined": 2 * (12 * A.nnz + 24 * A.n + 8) + 304 * A.n}
    out = {"n": int(A.n), "nnz": int(A.nnz)}
    for name, v in (("classic", 0), ("pipelined", 1)):
        rbs.rbs_solve(Ad, b, tol=TOL, maxit=MAXIT, variant=v, x_out=x, history=False)
        torch.cuda.synchronize()
        t = time.perf_counter()
        its = 0
        for _ in range(reps):
            its += rbs.rbs_solve(Ad, b, tol=TOL, maxit=MAXIT, variant=v, x_out=x, history=False)["iters"]
        torch.cuda.synchronize()
        ips = its / (time.perf_counter() - t)
        out[name] = {"iters_per_s": ips, "iters": its // reps,
                     "frac_of_hbm": per_iter[name] * ips / 1e9 / hbm}
    return out


def _c3b(rbs, gen, dev, reps=3):
    """C3b: upwind convection-diffusion 192^3 (Pe 10, velocity (1,1,1)),
    classic and pipelined reproducible solves to tol 1e-10, iterations/s."""
    import torch
    A = gen.convdiff3d(192, 10.0)
    Ad = rbs.to_device(A, dev)
    b = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
    x = torch.empty(A.n, dtype=torch.float64, device=dev)
    out = {"n": int(A.n), "nnz": int(A.nnz)}
    for name, v in (("classic", 0), ("pipelined", 1)):
        rbs.rbs_solve(Ad, b, tol=TOL, maxit=MAXIT, variant=v, x_out=x, history=False)
        torch.cuda.synchronize()
        t = time.perf_counter()
        its = 0
        for _ in range(reps):
            its += rbs.rbs_solve(Ad, b, tol=TOL, maxit=MAXIT, variant=v, x_out=x, history=False)["iters"]
        torch.cuda.synchronize()
        out[name] = {"iters_per_s": its / (time.perf_counter() - t), "iters": its // reps}
    return out


def run_serving(args):
    """Serving sweep (10k requests per arrival rate) as its own JSON line."""
    import torch
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    import __graft_entry__ as ge
    ge.build()
    import paper_2302_04180_gb300 as rbs
    from paper_2302_04180_gb300 import gen
    sweep = _serving(rbs, gen, dev, rates=tuple(float(r) for r in args.rates.split(",")), count=args.requests)
    best = max(r["solves_per_s"] for r in sweep)
    print(json.dumps({"metric": "serving solves/s at p99", "value": best, "unit": "solves/s",
                      "n_gpus": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "Poisson arrivals, 48-system pool (3D conv-diff, "
                                             "3D Poisson up to 128^3), tol 1e-8"},
                      "sweep": sweep}), flush=True)
    return 0


def run_solve_only(args):
    """Warm-up and timed solves of one variant on the Poisson --grid workload
    (host loop, per-kernel CUDA events), one JSON line: a profiling target."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2302_04180_gb300 as rbs
    from paper_2302_04180_gb300 import gen
    dev = torch.device("cuda:0")
    A = gen.poisson3d(GRID)
    Ad = rbs.to_device(A, dev)
    b = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
    x = torch.empty(A.n, dtype=torch.float64, device=dev)
    variant = 1 if args.solve_only == "pipelined" else 0
    for _ in range(args.warmup):
        rbs.rbs_solve(Ad, b, tol=TOL, maxit=MAXIT, variant=variant, x_out=x, loop_mode=1)
    tot, iters, traces = {}, 0, []
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        r = rbs.rbs_solve(Ad, b, tol=TOL, maxit=MAXIT, variant=variant, x_out=x, profile=True,
                          loop_mode=1, trace=(1 << 15) if args.trace else 0)
        if args.trace:
            traces.append((r["iters"], r["trace"]))
        iters += r["iters"]
        for k, (nl, ms) in r["prof"].items():
            a = tot.setdefault(k, [0, 0.0])
            a[0] += nl
            a[1] += ms
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    line = {"variant": args.solve_only, "grid": GRID, "iters": iters, "iters_per_s": iters / dt,
            "us_per_launch": {k: v[1] * 1e3 / max(v[0], 1) for k, v in tot.items() if v[0]},
            "launches": {k: v[0] for k, v in tot.items() if v[0]}}
    if args.trace:
        line["trace"] = _trace_buckets(traces)
    print(json.dumps(line), flush=True)
    return 0


def _trace_buckets(traces, width=25):
    """Per-launch traces of several solves -> per kernel kind, the median
    launch time (us) in buckets of `width` iterations (launches that ran only)."""
    import collections
    b = collections.defaultdict(list)
    for iters, tr in traces:
        for kind, it, ms in tr:
            if 0 <= it < iters:
                b[(kind, it // width)].append(ms * 1e3)
    out = {}
    for (kind, k), v in sorted(b.items()):
        out.setdefault(kind, {})[f"{k * width}-{k * width + width - 1}"] = round(statistics.median(v), 1)
    return out


def run_batched_only(args):
    """Only the batched solve (C4): `--systems` of the seeded 512-system
    workload under a given schedule (cluster:split; 0:0 is the stepped
    schedule with rows per block chosen per chunk), one warm-up and `--steps`
    timed calls; the profiling target of the batch kernels."""
    import torch
    import paper_2302_04180_gb300 as rbs
    from paper_2302_04180_gb300 import gen
    dev = torch.device("cuda:0")
    cl, sp = (int(t) for t in args.schedule.split(":"))
    work = gen.batch_workload(512, seed=0)[: args.systems]
    systems = []
    for A, v in work:
        Ad = rbs.to_device(A, dev)
        b = rbs.rbs_spmv_csr(Ad, torch.ones(A.n, dtype=torch.float64, device=dev))
        systems.append({"A": Ad, "b": b, "x": torch.empty(A.n, dtype=torch.float64, device=dev),
                        "tol": 1e-8, "maxit": 5000, "variant": v})
    for _ in range(max(args.warmup, 1)):
        res = rbs.rbs_solve_batched(systems, history=False, schedule={"cluster": cl, "split": sp})
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        res = rbs.rbs_solve_batched(systems, history=False, schedule={"cluster": cl, "split": sp})
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / max(args.steps, 1)
    alg = sum(r["iters"] * (24 * A.nnz + (352 if v else 216) * A.n) for r, (A, v) in zip(res, work))
    hbm, _ = _peaks()
    print(json.dumps({"section": "batched", "systems": len(systems), "schedule": args.schedule, "seconds": dt,
                      "total_iters": int(sum(r["iters"] for r in res)),
                      "frac_of_hbm": alg / dt / 1e9 / hbm}), flush=True)
    return 0


def run_micro_spmv(args):
    """Standalone CSR SpMV on the named matrices (poisson:SIDE, the 7-point
    Poisson matrix; stencil27:SIDE, the 27-point e-type one), one JSON line per
    case; the profiling target of the SpMV kernels."""
    import torch
    import paper_2302_04180_gb300 as rbs
    from paper_2302_04180_gb300 import gen
    dev = torch.device("cuda:0")
    hbm, _ = _peaks()
    makers = {"poisson": gen.poisson3d, "stencil27": gen.stencil27}
    for case in args.micro_spmv.split(","):
        kind, side = case.split(":")
        A = makers[kind](int(side))
        Ad = rbs.to_device(A, dev)
        xv = torch.from_numpy(gen.random_vector(A.n, 1)).to(dev)
        yv = torch.empty_like(xv)
        for _ in range(args.warmup):
            rbs.rbs_spmv_csr(Ad, xv, yv)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            rbs.rbs_spmv_csr(Ad, xv, yv)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / max(args.steps, 1)
        byt = 12 * A.nnz + 8 * (A.n + 1) + 16 * A.n
        print(json.dumps({"kernel": "spmv", "matrix": case, "n": int(A.n), "nnz": int(A.nnz), "us": ms * 1e3,
                          "GB/s": byt / (ms * 1e-3) / 1e9, "frac_of_hbm": byt / (ms * 1e-3) / 1e9 / hbm}),
              flush=True)
        del Ad, xv, yv
    return 0


def run_micro_exdot(args):
    """Standalone exact dots of seeded ill-conditioned vectors with known exact
    results (the kernel microbenchmark's dot cases), one JSON line per case."""
    import torch
    import paper_2302_04180_gb300 as rbs
    from paper_2302_04180_gb300 import gen
    dev = torch.device("cuda:0")
    for case in args.micro_exdot.split(","):
        lg, cond = case.split(":")
        n = 1 << int(lg)
        x, y, exact = gen.ill_conditioned_dot(n, float(cond), 0)
        xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
        del x, y
        o = torch.empty(1, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            rbs.rbs_exdot(xt, yt, o)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            rbs.rbs_exdot(xt, yt, o)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / max(args.steps, 1)
        print(json.dumps({"kernel": "exdot", "n": n, "cond": float(cond), "us": ms * 1e3,
                          "GB/s": 16 * n / (ms * 1e-3) / 1e9,
                          "matches_exact": None if exact is None else bool(float(o.cpu()) == float(exact))}),
              flush=True)
        del xt, yt
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--grid", type=int, default=256,
                    help="Poisson grid side (profiling runs on smaller cases; the metric is 256)")
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="solver loop driver for untimed solves (timed solves use the host "
                         "driver, which records per-kernel CUDA events)")
    ap.add_argument("--serving", action="store_true",
                    help="only the serving sweep: 10k Poisson-arrival requests per rate")
    ap.add_argument("--requests", type=int, default=10000, help="with --serving: requests per arrival rate")
    ap.add_argument("--rates", default="100,300,1000,3000", help="with --serving: arrival rates per second")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip e2e, comparators and kernel microbenchmarks")
    ap.add_argument("--solve-only", default=None, choices=["classic", "pipelined"],
                    help="only warm-up + timed solves of this variant on the --grid workload, "
                         "with per-kernel CUDA-event times (a profiling target)")
    ap.add_argument("--trace", action="store_true",
                    help="with --solve-only: per-launch CUDA-event trace, reported as per-kernel "
                         "medians over buckets of 25 iterations")
    ap.add_argument("--micro-exdot", default=None, metavar="LOG2N:COND[,...]",
                    help="only the standalone exact-dot microbenchmark on these cases "
                         "(e.g. 24:1e32 or 20:1,27:1e48); the profiling target of the exdot")
    ap.add_argument("--micro-spmv", default=None, metavar="KIND:SIDE[,...]",
                    help="only the standalone SpMV microbenchmark on these matrices "
                         "(e.g. stencil27:159 or poisson:128); the profiling target of the SpMV")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched solve (C4) under --schedule; the profiling target of the batch kernels")
    ap.add_argument("--systems", type=int, default=512, help="with --batched-only: systems of the workload")
    ap.add_argument("--schedule", default="0:0", help="with --batched-only: cluster:split")
    args = ap.parse_args()
    global GRID
    GRID = args.grid
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)
    if args.micro_exdot:
        return run_micro_exdot(args)
    if args.micro_spmv:
        return run_micro_spmv(args)
    if args.batched_only:
        return run_batched_only(args)
    if args.solve_only:
        return run_solve_only(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
