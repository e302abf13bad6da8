#!/usr/bin/env python3
"""Benchmark of the transmission hot path on the bulk fcc Cu [001] workload.

Workload: bulk fcc Cu along [001], a = 6.82 bohr, 20x20x480 grid (h = 0.341 bohr),
order-12 stencil, Gaussian-atom potential with +-2% jitter, 64-plane quadratic CAPs
of peak 0.3 Ha, 8x8 Monkhorst-Pack k-mesh, 256 energies in E_F +- 0.3 Ha; solver
residual 1e-10.

Default form (--form sketch): a step is the full trace T(E, k) and T(E, -k) of one
seeded k-pair of the mesh at a window of 16 consecutive energies of the 256 (seeded
position), from a two-sided randomized sketch of Gamma_R^1/2 G Gamma_L^1/2 (12 runs
with random left-CAP right-hand sides, 24 with random right-CAP ones), every run a
multi-shift transpose BiCG over the window in double-float arithmetic: the whole hot
path (operator, right-hand sides, stencil, Krylov and per-shift updates, convergence,
retirement, the trace reduction) on the GPU.  value = (E, k) values per second = 32 per
step / step time.

--form fp64 / mixed: the plain engine on seeded (E, k, column) samples, each column
solved to convergence; value = 2 * column-solves/s / n_rhs (each column gives the k
and -k columns).  --form columns: the multi-shift engine on sampled unit columns.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "converged (E,k) T(E) solves/sec at |ΔT|≤1e-6 vs plain FP64 GPU; stencil HBM %peak"
UNIT = "(E,k) solves/s"
WORKLOAD = ("bulk fcc Cu [001] a=6.82, 20x20x480 h=0.341, order 12, V0=1.2 sigma=0.9 +-2% "
            "jitter, 64-plane CAPs 0.3 Ha, 8x8 MP k-mesh, 256 energies in E_F+-0.3 Ha, tol 1e-10")
WORKLOAD_IDEAL = ("ideal bulk fcc Cu [001] (no jitter, V invariant under the in-plane inversion about an "
                  "atom), otherwise as the bulk Cu workload: 20x20x480 h=0.341, order 12, 64-plane CAPs 0.3 Ha, "
                  "8x8 MP k-mesh, 256 energies in E_F+-0.3 Ha, tol 1e-10")
WORKLOAD_RH = ("Rh periodic point contact [001] a=7.18, 3x3 cells, 60x60x512 h=0.359, order 12, "
               "V0=1.4 sigma=0.95, hyperboloid neck r0=4, 1% vacancies, 64-plane CAPs 0.3 Ha, "
               "4x4 MP k-mesh, 512 energies in E_F+-0.3 Ha, tol 1e-10")
HBM_FALLBACK_GBS = 6800.0
# DRAM bytes per point-half of one FP64 stencil launch, from the ncu capture of that
# kernel on the bulk Cu workload (900.5 MB for 12.29 M point-halves); scaled by the
# point-halves of each launch for the roofline's traffic.  Reset to None whenever the
# kernel changes.
FP64_STENCIL_DRAM_PER_POINT_HALF = 900.5e6 / 12.288e6
# FP64 ALU roofline: 2 FP64 FMA per clock per SM x 152 SMs x 2070 MHz x 2 flops
FP64_PEAK_TFLOPS = 2 * 152 * 2.070e9 * 2 / 1e12
# FP32 pipe roofline of the double-float stencil, in FP32 operations (add, multiply or
# FMA, one each): 128 FP32 lanes per SM x 152 SMs x 2070 MHz
FP32_OPS_PEAK_T = 128 * 152 * 2.070e9 / 1e12
# DRAM bytes per point-half of one double-float stencil launch, from the ncu capture of
# that kernel on the bulk Cu workload (294.4 MB for 4.608 M point-halves, 4 + 8 runs,
# slabs of 40 planes); reset to None whenever the kernel changes
DF_STENCIL_DRAM_PER_POINT_HALF = 294.4e6 / 4.608e6


def stencil_flops_per_point(order: int) -> int:
    """Algorithmic flops of one stencil launch per grid point and half:
    p = r + beta p (8), diagonal term (6), 3 axes x R neighbour pairs x (pair add 2,
    weight 2, accumulate 2) = 18R, pairing dot (8)."""
    return 18 * (order // 2) + 22


def stencil_df_ops_per_point(order: int, iso: bool = False) -> int:
    """FP32 operations of the double-float stencil per grid point and half, counted
    from its algorithm (halo recomputation excluded): p = r + beta p (complex
    double-float multiply 38 + accurate add 2 x 20 = 78), diagonal term (accurate
    subtraction 20, four products 16, four accumulations 32 = 68), per distance m and
    component either 3 x (TwoSum pair 8, product 4, accumulation 8) = 60, or, with the
    same spacing on the three axes (iso), three pairs 24, their two sums 16, one
    product 4 and one accumulation 8 = 52; combining the axes 54, pairing dot with its
    scaling 56."""
    per_m = 2 * (52 if iso else 60)
    return 78 + 68 + per_m * (order // 2) + 54 + 56


def stencil_bytes_per_point(elem: int) -> int:
    """Algorithmic HBM bytes of one stencil launch per point and half: read r and p,
    write p and q (complex elements of ``elem`` bytes)."""
    return 4 * elem


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int = 0):
        self.p = None
        self.dev = device_index

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def k_representatives(kfrac) -> list[int]:
    """k-points that stand for a (k, -k) pair of the mesh (kappa_a > 0, or = 0 and
    kappa_b > 0)."""
    return [i for i, (a, b) in enumerate(kfrac) if a > 1e-12 or (abs(a) <= 1e-12 and b > 1e-12)]


def draw_items(inst, reps, n_rhs, count, seed):
    rng = np.random.default_rng(seed)
    e = inst.energies[rng.integers(0, len(inst.energies), count)]
    k = np.asarray(reps, np.int32)[rng.integers(0, len(reps), count)]
    c = rng.integers(0, n_rhs, count).astype(np.int64)
    return e.astype(np.float64), k.astype(np.int32), c


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


_ORACLE_CACHE = {}


def _oracle_worker(args):
    """One host process of the CPU baseline: the oracle's transpose BiCG (as it stands)
    on one seeded column of the workload for a bounded number of iterations; returns
    the seconds per iteration.  The workload's operator is built once per process."""
    workload, e, kf, col, budget_s = args
    from workloads import cu_bulk, rh_point_contact, uneven_batch
    from oracle.hamiltonian import system_matrix
    from oracle.transmission import bicg_transpose, left_support

    key = (workload, e, kf)
    if key not in _ORACLE_CACHE:
        inst = _ORACLE_CACHE.get(workload)
        if inst is None:
            if workload.startswith("uneven_batch:"):
                inst = uneven_batch(96, only=[int(workload.split(":")[1])])[0]
            else:
                inst = rh_point_contact() if workload == "rh_point_contact" else cu_bulk()
            _ORACLE_CACHE[workload] = inst
        g = inst.grid
        _ORACLE_CACHE.clear()
        _ORACLE_CACHE[workload] = inst
        _ORACLE_CACHE[key] = system_matrix(g, inst.v, inst.gamma_l, inst.gamma_r, float(e), tuple(kf))
    inst = _ORACLE_CACHE[workload]
    g = inst.grid
    a = _ORACLE_CACHE[key]
    j = int(left_support(g, inst.gamma_l)[int(col)])
    b = np.zeros((g.n, 1), complex)
    b[j, 0] = 1.0
    bicg_transpose(a, b, 1e-30, 2)  # warm caches
    n_it = 4
    while True:
        t0 = time.perf_counter()
        bicg_transpose(a, b, 1e-30, n_it)
        dt = time.perf_counter() - t0
        if dt > budget_s / 3 or n_it >= 4096:
            break
        n_it *= 2
    return dt / n_it, n_it, dt


def golden_mean_iterations() -> float:
    """Mean iterations of the oracle's transpose BiCG to 1e-10 over the committed
    full-size bulk Cu columns: the one iteration basis of both CPU figures."""
    with open(os.path.join(ROOT, "tests", "golden", "cu_bulk_columns.json")) as f:
        return float(np.mean([it["iters_1e-10"] for it in json.load(f)["items"]]))


class OraclePool:
    """The oracle timed on the host cores: one single-threaded process per core (spawned,
    so no process inherits a CUDA context), each running the transpose BiCG on its own
    seeded column of the workload."""

    def __init__(self, workload: str, procs: int | None = None):
        import multiprocessing as mp

        self.workload = workload
        self.procs = procs or min(os.cpu_count() or 1, 64)
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs)
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old

    def rate(self, inst, items, iters_per_column: float, budget_s: float):
        """Column-solves/s of all processes together: every process's column time is its
        time per iteration x iters_per_column, and the processes' rates add up.  Returns
        (column-solves/s, median iterations timed per process, wall seconds)."""
        e, k, c = items
        jobs = [(self.workload, float(e[u % len(e)]), tuple(map(float, inst.kfrac[int(k[u % len(k)])])),
                 int(c[u % len(c)]), budget_s) for u in range(self.procs)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        rate = sum(1.0 / (per_it * iters_per_column) for per_it, _, _ in res)
        return rate, int(np.median([r[1] for r in res])), wall

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_reference(args):
    """The CPU oracle timed on the host cores, as the reference arm."""
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    from workloads import cu_bulk

    inst = cu_bulk()
    n_rhs = inst.n_rhs
    reps = k_representatives(inst.kfrac)
    mean_its = golden_mean_iterations()
    rates = []
    t_all = 0.0
    # the processes keep one operator each: every step draws new columns at the same
    # (E, k) per process, so the timed steps measure iterations, not matrix assembly
    items0 = draw_items(inst, reps, n_rhs, 64, 7000)
    with OraclePool("cu_bulk") as op:
        procs = op.procs
        for step in range(args.warmup + args.steps):
            items = (items0[0], items0[1], draw_items(inst, reps, n_rhs, 64, 7000 + step)[2])
            col_rate, n_it, wall = op.rate(inst, items, mean_its, budget_s=1.5)
            if step >= args.warmup:
                rates.append(col_rate)
                t_all += wall
    col_rate = float(np.mean(rates))
    value = 2.0 * col_rate / n_rhs
    sample = (f"oracle transpose BiCG (numpy/scipy, complex128), one single-threaded process per "
              f"core ({procs}), each on its own seeded column of the workload for a bounded "
              f"iteration count (~1.5 s per step); column time = time per iteration x {mean_its:.0f} (oracle "
              f"mean iterations to 1e-10 over the committed golden columns); rates summed")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": {"workload": WORKLOAD, "column_solves_per_s": col_rate},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_uneven_batch(args):
    """Configuration 4: 96 seeded Cu/Rh bulk and point-contact cells of uneven size.
    A step takes one seeded (E at mid-window, k, column) item from each of 16 seeded
    cells and solves them together in one batched call (one slot engine, the cells'
    operators in a table) in the mixed FP32/FP64 form (``--form fp64``: plain FP64),
    with the tile height, slab depth and slots chosen by transec_autotune on the driver
    context; the same items solved one cell at a time in plain FP64 give the looped
    time-to-T figure.  Reports column-solves/s of both and their ratio."""
    import torch

    from workloads import uneven_batch
    import paper_2208_02783_gb300 as pkg
    from paper_2208_02783_gb300 import build

    pkg.load(build.build())
    prec = pkg.PREC_FP64 if args.form == "fp64" else pkg.PREC_MIXED
    insts = uneven_batch(96)
    ctxs = [pkg.Transec.from_instance(i, device=0, tol=1e-10, precision=prec) for i in insts]
    per_step = 16
    tuned = ctxs[0].autotune(float(insts[0].energies[len(insts[0].energies) // 2]), 0)

    def items(step):
        rng = np.random.default_rng(4000 + step)
        cells = rng.choice(len(insts), per_step, replace=False)
        e = np.array([insts[c].energies[len(insts[c].energies) // 2] for c in cells])
        k = np.array([rng.integers(0, len(insts[c].kfrac)) for c in cells], np.int32)
        col = np.array([rng.integers(0, insts[c].n_rhs) for c in cells], np.int64)
        return cells.astype(np.int32), e, k, col

    def set_all(**kw):
        for c in ctxs:
            c.set_solver(**kw)

    for s in range(args.warmup):
        cells, e, k, col = items(s)
        pkg.batch_column_contributions(ctxs, cells, e, k, col)
    torch.cuda.synchronize()
    ctxs[0].stats_reset()
    t_batch = 0.0
    t_loop = 0.0
    its = 0
    fails = 0
    dt_max = 0.0
    rel_max = 0.0
    statuses = []
    its_items = []
    clocks = Clocks(0)
    clocks.start()
    for s in range(args.steps):
        cells, e, k, col = items(args.warmup + s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = pkg.batch_column_contributions(ctxs, cells, e, k, col)
        t_batch += time.perf_counter() - t0
        its += int(r["iters"].sum())
        fails += int((r["status"] != 0).sum())
        set_all(precision=pkg.PREC_FP64)
        t0 = time.perf_counter()
        for u, c in enumerate(cells):
            q = ctxs[c].column_contributions(e[u:u + 1], k[u:u + 1], col[u:u + 1])
            statuses.append((int(r["status"][u]), int(q["status"][0])))
            its_items.append((int(c), float(e[u]), int(k[u]), int(col[u]), int(q["iters"][0])))
            d = abs(q["t"][0] - r["t"][u])
            dt_max = max(dt_max, d)
            rel_max = max(rel_max, d / max(abs(q["t"][0]), 1e-300))
        t_loop += time.perf_counter() - t0
        set_all(precision=prec)
    clk = clocks.stop()
    st = ctxs[0].stats()
    n = per_step * args.steps
    value = n / t_batch

    # profiled pass (separate): one step's items with the driver's stencil launches timed
    cells, e, k, col = items(args.warmup + args.steps)
    ctxs[0].set_solver(profile=1, maxit=400)
    ctxs[0].stats_reset()
    pkg.batch_column_contributions(ctxs, cells, e, k, col)
    stp = ctxs[0].stats()
    ctxs[0].set_solver(profile=0, maxit=100000)
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    order = insts[0].grid.order
    if prec == pkg.PREC_FP64:
        pa, sten_ms, nl = stp["point_applies"], stp["stencil_ms"], max(1, stp["stencil_launches"])
        flops = pa * stencil_flops_per_point(order)
        achieved = flops / (sten_ms / 1e3) / 1e12 if sten_ms > 0 else 0.0
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "k_stencil<double,6> (batched)",
                "per_launch": {"flops": flops / nl, "ms": sten_ms / nl},
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz"}
    else:
        pa, sten_ms, nl = stp["point_applies32"], stp["stencil32_ms"], max(1, stp["stencil32_launches"])
        byts = pa * stencil_bytes_per_point(8)
        achieved = byts / (sten_ms / 1e3) / 1e9 if sten_ms > 0 else 0.0
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "kernel": "k_stencil<float,6> (batched)",
                "per_launch": {"bytes": byts / nl, "ms": sten_ms / nl},
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    roof["timing"] = ("separate profiled pass: one step's 16 items, at most 400 iterations, CUDA events "
                      "around every stencil launch on the driver context's stream")
    line = {
        "metric": "uneven batch column-solves/s (batched one call vs looped per cell in plain FP64)",
        "value": value, "unit": "column-solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_batch / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128" if prec == pkg.PREC_FP64 else "c64+f64",
        "data": "synthetic",
        "config": {"workload": "96 seeded Cu/Rh bulk and point-contact cells, 1x1-4x4 cells wide, "
                               "12-40 cells long, h 0.30-0.40, order 12 (configuration 4)",
                   "form": ("plain FP64 transpose BiCG" if prec == pkg.PREC_FP64 else
                            "mixed: complex FP32 BiCG with FP64 scalars and residual replacement, FP64 fallback"),
                   "autotuned": tuned,
                   "items_per_step": per_step, "looped_fp64_column_solves_per_s": n / t_loop,
                   "batched_over_looped": t_loop / t_batch, "mean_iterations_batched": its / n,
                   "fp64_fallback_columns": int(st.get("fallbacks", 0)),
                   "failed_batched": fails, "max_abs_dt_batched_vs_looped_fp64": dt_max,
                   "max_rel_dt_batched_vs_looped_fp64": rel_max,
                   "statuses_batched_looped": sorted(set(statuses)),
                   "timing": "host wall clock around each call (host arrays in and out)"},
        "roofline": roof,
        "e2e": {"value": value, "unit": "column-solves/s", "h2d_bytes_per_step": per_step * (8 + 4 + 8 + 4),
                "d2h_bytes_per_step": per_step * (8 + 8 + 4 + 4),
                "note": "the timed value is already end to end: the public call with host arrays"},
        "gpu_launches": int(st["launches"]),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        # the oracle on the host cores: each process runs the oracle's transpose BiCG on
        # one timed item's cell and column; its column time is its time per iteration x
        # the FP64 iterations the looped GPU solve of that column took
        sample = its_items[:min(len(its_items), os.cpu_count() or 1, 16)]
        with OraclePool("cu_bulk", procs=len(sample)) as op:
            jobs = [(f"uneven_batch:{c}", e_, tuple(map(float, insts[c].kfrac[k_])), col_, 6.0)
                    for c, e_, k_, col_, _ in sample]
            res = op.pool.map(_oracle_worker, jobs, chunksize=1)
        crate = sum(1.0 / (per_it * max(1, it_)) for (per_it, _, _), (*_, it_) in zip(res, sample))
        line["cpu_baseline"] = {
            "value": crate, "unit": "column-solves/s", "cores": len(sample), "kind": "oracle",
            "sample": (f"oracle transpose BiCG (numpy/scipy complex128), one single-threaded process per core "
                       f"({len(sample)}), each on the cell and column of one timed item for a bounded number of "
                       "iterations (about 2 s); column time = time per iteration x the FP64 iterations of that "
                       "column on the GPU; rates summed"),
        }
    print(json.dumps(line))
    for c in ctxs:
        c.close()
    return 0


# 4 + 8 random right-hand sides with the library's sketch guard (1e-7): a result whose
# missed-energy estimate or whose two independent +-k estimates exceed the guard is
# computed again with a doubled sketch inside the call.  On ten seeded windows of the
# bulk Cu workload the guarded 4 + 8 results agreed with unguarded 16 + 32 sketches to
# 2.4e-8 and took 0.66 of the time of guarded 8 + 16
SKETCH_WINDOW, SKETCH_LEFT, SKETCH_RIGHT = 16, 4, 8


def sketch_plan(n_energy: int, reps, count: int, window: int, seed: int = 3000):
    """(k index, first energy index) of each sketch step: a seeded k-pair
    representative and a seeded window position, drawn per step from a generator of its
    own (step i's window does not depend on how many steps are drawn)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng([seed, i])
        out.append((int(reps[int(rng.integers(0, len(reps)))]), int(rng.integers(0, n_energy - window + 1))))
    return out


def run_sketch(args):
    """Full-trace T(E, +-k) over energy windows by the two-sided sketch (default form)."""
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from workloads import cu_bulk, cu_bulk_ideal, rh_point_contact
    import paper_2208_02783_gb300 as pkg
    from paper_2208_02783_gb300 import build, replicas

    pkg.load(build.build())
    rh = args.workload == "rh_point_contact"
    ideal = args.workload == "cu_bulk_ideal"
    inst = rh_point_contact() if rh else (cu_bulk_ideal() if ideal else cu_bulk())
    g = inst.grid
    reps = k_representatives(inst.kfrac)
    W, sl, sr = args.window, args.s_left, args.s_right
    prec = pkg.PREC_FP64 if args.form == "sketch_fp64" else pkg.PREC_DF64
    psym = 1 if args.psym else 0
    H = 1 if psym else 2  # halves per run
    tr = pkg.Transec.from_instance(inst, device=local, tol=1e-10, precision=prec, psym=psym)
    e2e_steps = min(args.steps, 2)
    plan = sketch_plan(len(inst.energies), reps, (args.warmup + args.steps) * ws, W)

    def window(i):
        k, e0 = plan[i * ws + rank]
        return k, inst.energies[e0:e0 + W].astype(np.float64)

    def step(i):
        k, en = window(i)
        return tr.transmission_sketch(en, [k], s_left=sl, s_right=sr, seed=1000 + i)

    if args.profile_case:
        # bounded case for the profilers: one window, 40 iterations (the shifts stop as
        # not converged), host-driven chunk graphs (profilers do not enter graphs with
        # conditional nodes); about 2 GB on the device
        tr.set_solver(maxit=40, host_loop=1)
        step(0)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "ok", "workload": args.workload, "form": "sketch"}))
        tr.close()
        return 0

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    tr.stats_reset()
    clocks = Clocks(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.start()
    ev0.record()
    results, step_s = [], []
    for i in range(args.steps):
        t0 = time.perf_counter()
        results.append(step(args.warmup + i))
        step_s.append(round(time.perf_counter() - t0, 2))
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    ms = replicas.max_over_ranks(ev0.elapsed_time(ev1), device=dev)
    st = tr.stats()
    sw = tr.sweep_stats()
    per_step = 2 * W  # T(E, k) and T(E, -k) for every energy of the window
    value = replicas.whole_job_rate(per_step * args.steps, ws, ms / 1e3)
    T = np.concatenate([r["T"][0] for r in results])
    Tm = np.concatenate([r["T_minus"][0] for r in results])
    status = np.concatenate([r["status"][0] for r in results])
    its = np.concatenate([r["iters"][0] for r in results])
    ok = status == 0
    pm_diff = float(np.abs(T[ok] - Tm[ok]).max()) if ok.any() else None

    # end to end through the public API with host arrays: the window's energies and k in,
    # T(E, +-k), ranks, statuses and iterations out, host wall clock; the same windows
    # as the first timed steps, so that the two figures compare like with like
    e2e_s = 0.0
    for i in range(e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(args.warmup + i)
        e2e_s += time.perf_counter() - t0
    e2e_s = replicas.max_over_ranks(e2e_s, device=dev)
    e2e_value = replicas.whole_job_rate(per_step * e2e_steps, ws, e2e_s)
    same_steps_value = replicas.whole_job_rate(per_step * e2e_steps, ws, sum(step_s[:e2e_steps]))

    # parity against the plain FP64 arithmetic on the first timed window: the same sketch
    # in the FP64 engine (the double-float form's metric bar is |dT| <= 1e-6 vs FP64)
    parity = None
    if rank == 0 and prec == pkg.PREC_DF64 and not args.no_parity:
        k, en = window(args.warmup)
        tr.set_solver(precision=pkg.PREC_FP64, psym=0)
        ref = tr.transmission_sketch(en, [k], s_left=sl, s_right=sr, seed=1000 + args.warmup)
        tr.set_solver(precision=prec, psym=psym)
        got = results[0]
        okp = (ref["status"][0] == 0) & (got["status"][0] == 0)
        parity = {"window_energies": W, "k_index": k,
                  "seed_iterations_mean_fp64": float(ref["iters"][0].mean()),
                  "seed_iterations_mean_df64": float(got["iters"][0].mean()),
                  "max_abs_dT_vs_fp64": float(np.abs(got["T"][0][okp] - ref["T"][0][okp]).max()),
                  "max_abs_dT_minus_vs_fp64": float(np.abs(got["T_minus"][0][okp] - ref["T_minus"][0][okp]).max()),
                  "fp64_all_converged": bool(np.all(ref["status"] == 0))}

    # profiled pass (separate from the timed steps): one window for 200 iterations with
    # every shift of every run active, each stencil and shift-update launch bracketed by
    # CUDA events on the context's stream
    prof_its = 200
    k, en = window(0)
    tr.set_solver(profile=1, maxit=prof_its)
    tr.stats_reset()
    pclk = Clocks(local)
    pclk.start()
    tr.transmission_sketch(en, [k], s_left=sl, s_right=sr, seed=1)
    prof_clk = pclk.stop()
    swp = tr.sweep_stats()
    tr.set_solver(profile=0, maxit=100000)
    runs = sl + sr
    ph_per_launch = runs * H * g.n  # every run active: every half of every grid point
    # the kernels of the form being timed (a bounded pass ends its runs unconverged, and
    # the double-float form then redoes them in FP64: those launches are counted apart)
    key = "_df" if prec == pkg.PREC_DF64 else ""
    st_ms = swp["stencil" + key + "_ms"] / max(1, swp["stencil" + key + "_launches"])
    sh_ms = swp["shift" + key + "_ms"] / max(1, swp["shift" + key + "_launches"])
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    if prec == pkg.PREC_DF64:
        iso = g.hx == g.hy == g.hz
        ops = stencil_df_ops_per_point(g.order, iso) * ph_per_launch
        achieved = ops / (st_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP32_OPS_PEAK_T, "unit": "T FP32-op/s",
                "frac": achieved / FP32_OPS_PEAK_T,
                "traffic": (DF_STENCIL_DRAM_PER_POINT_HALF * ph_per_launch
                            if DF_STENCIL_DRAM_PER_POINT_HALF and not rh else None),
                "kernel": f"k_stencil_df<{g.order // 2}> (double-float stencil fused with p = r + beta p and the "
                          "pairing dot)",
                "per_launch": {"point_halves": ph_per_launch, "fp32_ops": ops, "ms": st_ms,
                               "fp64_equivalent_tflops": stencil_flops_per_point(g.order) * ph_per_launch / (st_ms / 1e3) / 1e12,
                               "hbm_gbs": stencil_bytes_per_point(16) * ph_per_launch / (st_ms / 1e3) / 1e9},
                "peak_source": "derived: 128 FP32 lanes/SM x 152 SMs x 2070 MHz (one add, multiply or FMA "
                               "per lane and clock)",
                "fp64_equivalent_frac_of_fp64_peak": stencil_flops_per_point(g.order) * ph_per_launch
                / (st_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS}
    else:
        flops = stencil_flops_per_point(g.order) * ph_per_launch
        achieved = flops / (st_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": f"k_stencil<double,{g.order // 2}>",
                "per_launch": {"point_halves": ph_per_launch, "flops": flops, "ms": st_ms},
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz"}
    no = max(int(np.count_nonzero(inst.gamma_l)), int(np.count_nonzero(inst.gamma_r))) * g.nxy
    shift_bytes = runs * W * H * no * 64  # read/write p_sigma and x_sigma, 16 B each, per shift and half
    roof["shift_kernel"] = {"ms": sh_ms, "bytes_per_launch": shift_bytes,
                            "hbm_gbs": shift_bytes / (sh_ms / 1e3) / 1e9,
                            "hbm_frac_of_measured": shift_bytes / (sh_ms / 1e3) / 1e9 / hbm_peak}
    roof["timing"] = (f"separate profiled pass: one window, {runs} runs x {W} shifts, {prof_its} iterations, "
                      "CUDA events around every stencil and shift-update launch on the context's stream")
    roof["profile_clocks"] = prof_clk

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "df64+f64" if prec == pkg.PREC_DF64 else "c128",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD_RH if rh else (WORKLOAD_IDEAL if ideal else WORKLOAD),
            "form": ("full trace T(E, +-k) from a two-sided randomized sketch of Gamma_R^1/2 G Gamma_L^1/2: "
                     f"{sl} left + {sr} right random right-hand sides, each a multi-shift "
                     + ("P-symmetric COCG (one operator application per iteration)" if psym else "transpose BiCG")
                     + " over "
                     f"a window of {W} energies, " + ("double-float vectors and stencil, FP64 scalars"
                                                      if prec == pkg.PREC_DF64 else "FP64")),
            "step": f"one seeded k-pair x {W} consecutive energies (seeded position) = {per_step} (E, k) values",
            "value_derivation": f"{per_step} (E, k) values per step / step time (T(E, k) and T(E, -k) are "
                                "estimated from independent halves of the runs)",
            "mean_seed_iterations": float(its.mean()), "max_seed_iterations": int(its.max()),
            "failed_results": int((~ok).sum()), "max_abs_T_k_minus_T_mk": pm_diff,
            "results_redone_in_fp64": int(sw.get("fp64_redone", 0)),
            "results_redone_with_doubled_sketch": int(sw.get("guard_redone", 0)),
            "sketch_guard": "a result whose missed-energy estimate (4 ||(1 - P) M omega_last||^2) or whose "
                            "T(E, k) and T(E, -k) differ by more than 1e-7 is computed again with twice the "
                            "sketch sizes inside the call",
            "max_missed_energy_estimate": float(np.nanmax(np.concatenate([r["miss"][0] for r in results]))),
            "step_seconds": step_s,
            "min_rank": int(np.concatenate([r["rank"][0] for r in results]).min()),
            "parity_vs_fp64": parity,
            "l2": f"per-step working set ({runs} runs x {H} halves x {g.n:,} points x 4 vectors x 16 B = "
                  f"{runs * H * g.n * 64 / 1e9:.2g} GB, plus the per-shift planes) exceeds L2; no flush needed",
            "sampling": "steps draw (k-pair, window position) from a seeded generator; ranks take disjoint steps",
        },
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": W * 8 + 4,
                "d2h_bytes_per_step": W * (8 + 8 + 4 + 4 + 4),
                "windows": f"the first {e2e_steps} timed windows again (their timed rate: {same_steps_value:.4g})"},
        "gpu_launches": int(st["launches"]),
        "clocks": clk,
    }
    # (the oracle's iteration basis is the jittered bulk Cu workload's golden columns: no
    # CPU figure is printed for the ideal cell)
    if rank == 0 and not args.no_cpu_baseline and not ideal:
        mean_its = golden_mean_iterations()
        items = draw_items(inst, reps, inst.n_rhs, 64, 7000)
        with OraclePool("rh_point_contact" if rh else "cu_bulk") as op:
            op.rate(inst, items, mean_its, budget_s=1.0)  # operators built, caches warm
            crate, n_it, dt = op.rate(inst, items, mean_its, budget_s=12.0)
            procs = op.procs
        line["cpu_baseline"] = {
            "value": 2.0 * crate / inst.n_rhs, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": (f"oracle transpose BiCG (numpy/scipy complex128), one single-threaded process per core "
                       f"({procs}), each on its own seeded left-CAP column of the workload for {n_it} iterations "
                       f"(median; {dt:.1f} s wall); column time = time per iteration x {mean_its:.0f} (oracle "
                       f"mean iterations to 1e-10 over the committed golden columns); (E, k) rate = 2 x "
                       f"column rate / {inst.n_rhs} columns (the oracle's T(E, k) is the sum over every "
                       "left-CAP column, each giving the k and -k columns)"),
        }
    if rank == 0:
        print(json.dumps(line))
    tr.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_eigen_stage(args):
    """The paper's eigen route, its per-energy stage, on the bulk Cu cell: the transformed
    CAPs (two weighted Gram matrices of p eigenvectors' rows on the 25 600-point CAP
    supports) and the eigen-sum T(E) for the workload's 256 energies, from a supplied
    eigensolution (random unit-modulus rows and eigenvalues near E_F: the stage's cost
    does not depend on the values).  Timed through the public call with host arrays
    (e2e); kernel times from a profiled call."""
    import torch

    from workloads import cu_bulk
    import paper_2208_02783_gb300 as pkg
    from paper_2208_02783_gb300 import build

    pkg.load(build.build())
    inst = cu_bulk()
    g = inst.grid
    p = args.items or 1024
    rng = np.random.default_rng(11)
    nr = int(np.count_nonzero(inst.gamma_r)) * g.nxy
    nl = int(np.count_nonzero(inst.gamma_l)) * g.nxy
    vr = np.exp(2j * np.pi * rng.random((nr, p))) / np.sqrt(nr)
    wl = np.exp(2j * np.pi * rng.random((nl, p))) / np.sqrt(nl)
    lam = inst.fermi + rng.uniform(-0.3, 0.3, p) - 1j * rng.uniform(1e-3, 5e-2, p)
    en = inst.energies.astype(np.float64)
    tr = pkg.Transec.from_instance(inst, device=0)
    for _ in range(max(3, args.warmup)):
        tr.eigen_transmission(lam, vr, wl, en)
    torch.cuda.synchronize()
    steps = max(1, args.steps)
    clocks = Clocks(0)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(steps):
        tr.eigen_transmission(lam, vr, wl, en)
    dt = (time.perf_counter() - t0) / steps
    clk = clocks.stop()
    tr.set_solver(profile=1)
    tr.stats_reset()
    tr.eigen_transmission(lam, vr, wl, en)
    es = pkg.binding.transec_eigen_stats(tr.ctx)
    tr.set_solver(profile=0)
    tr.close()
    gram_flops = 8.0 * (p * (p + 1) / 2) * (nr + nl)  # Hermitian: one triangle
    sum_flops = 8.0 * p * p * en.size
    kern_s = (es["gram_ms"] + es["sum_ms"]) / 1e3
    achieved = gram_flops / (es["gram_ms"] / 1e3) / 1e12
    line = {
        "metric": "eigen route, per-energy stage: T(E) values per second from a supplied eigensolution",
        "value": en.size / dt, "unit": "T(E) values/s", "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup),
        "ms_per_step": 1e3 * dt, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128", "data": "synthetic",
        "config": {"workload": WORKLOAD + f"; {p} eigenpairs, {en.size} energies",
                   "step": "transformed CAPs (Gram matrices over 25 600 + 25 600 CAP rows) and the eigen-sum "
                           "for every energy of the window",
                   "kernel_ms": es},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS,
                     # the ncu capture of the Gram kernel predates the kernel's fused
                     # inner loop: no traffic figure for the current kernel
                     "traffic": None,
                     "kernel": "k_eig_gram (complex FP64 Hermitian Gram matrices, one triangle of 16 x 16 "
                               "shared-memory tiles)",
                     "flops": {"gram": gram_flops, "sum": sum_flops},
                     "sum_kernel_tflops": sum_flops / (es["sum_ms"] / 1e3) / 1e12 if es["sum_ms"] > 0 else None,
                     "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz"},
        "e2e": {"value": en.size / dt, "unit": "T(E) values/s",
                "h2d_bytes_per_step": int((nr + nl) * p * 16 + p * 16 + en.size * 8),
                "d2h_bytes_per_step": int(en.size * 8),
                "kernel_share": kern_s / dt},
        "gpu_launches": 3 * steps,
        "clocks": clk,
    }
    print(json.dumps(line))
    return 0


UNET_LAYERS = [(4, 16, 0), (16, 16, 0), (16, 32, 1), (32, 32, 1), (32, 64, 2), (64, 64, 2),
               (96, 32, 1), (32, 32, 1), (48, 16, 0), (16, 16, 0), (16, 2, 0)]  # (cin, cout, level)


def unet_forward_flops(nvox: int, padded: bool) -> float:
    """Multiply-add flops of one U-Net forward: 2 x 27 x cin x cout per voxel of each
    convolution's level (level l has nvox / 8^l voxels); padded=True counts the channels
    rounded up to 16 as the tensor cores execute them."""
    pad = (lambda c: (c + 15) // 16 * 16) if padded else (lambda c: c)
    return float(sum(2 * 27 * pad(ci) * pad(co) * nvox / 8 ** lv for ci, co, lv in UNET_LAYERS))


def run_learned(args):
    """Learned right preconditioner (an extension of the method): the U-Net forward on
    the bulk Cu volume (20x20x480, the network's per-Arnoldi-step cost), timed with
    CUDA events, and
    the FGMRES(30) gain on a 16x16x32 order-4 cell (operator applications and time per
    column with the network on alternate steps, without it, and with the plain FP64
    engine)."""
    import torch

    from workloads import cu_bulk, small_instance
    import paper_2208_02783_gb300 as pkg
    from paper_2208_02783_gb300 import build

    pkg.load(build.build())
    inst = cu_bulk()
    tr = pkg.Transec.from_instance(inst, device=0)
    lp = pkg.LearnedPreconditioner(tr, seed=1)
    n = tr.n
    x = torch.randn(n, 4, device="cuda", dtype=torch.float32)
    y = torch.empty(n, 2, device="cuda", dtype=torch.float32)
    if args.profile_case:
        # bounded case for the profilers: 3 forwards and 2 training steps on the bulk Cu
        # volume (33 + 2 x 22 convolution launches), then exit
        for _ in range(3):
            pkg.transec_unet_forward(lp.net, x, y)
        tgt = torch.randn(n, 2, device="cuda", dtype=torch.float32)
        for _ in range(2):
            pkg.transec_unet_train_step(lp.net, x, tgt, 1e-4)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "ok", "workload": "learned"}))
        lp.close()
        tr.close()
        return 0
    for _ in range(max(3, args.warmup)):
        pkg.transec_unet_forward(lp.net, x, y)
    torch.cuda.synchronize()
    steps = max(400, args.steps)  # ~0.3 s: long enough for the 200 ms clock samples
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    clocks.start()
    ev0.record()
    for _ in range(steps):
        pkg.transec_unet_forward(lp.net, x, y)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / steps
    # end to end: host input in, host output out
    xh = x.cpu().pin_memory()
    yh = torch.empty(n, 2, dtype=torch.float32).pin_memory()
    t0 = time.perf_counter()
    for _ in range(50):
        pkg.transec_unet_forward(lp.net, xh, yh)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / 50
    lp.close()
    tr.close()
    fl_alg = unet_forward_flops(n, False)
    fl_pad = unet_forward_flops(n, True)
    peaks = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    achieved = fl_alg / (ms / 1e3) / 1e12

    # FGMRES gain on the small cell
    cell = small_instance(16, 16, 32, 0.4, 4, 8, energies=(0.3,), seed=3)
    cols = np.array([0, 37, 100, 511, 1500])
    e = np.full(cols.size, 0.3)
    ik = np.zeros(cols.size, np.int32)
    gain = {}
    with pkg.Transec.from_instance(cell) as tc:
        t0 = time.perf_counter()
        plain = tc.column_contributions(e, ik, cols)
        gain["plain_engine"] = {"applies_per_column": float(plain["iters"].mean()),
                                "ms_per_column": (time.perf_counter() - t0) * 1e3 / cols.size}
        lpc = pkg.LearnedPreconditioner(tc, seed=1)
        t0 = time.perf_counter()
        g0 = lpc.fgmres_columns(e, ik, cols, precondition=False, maxit=6000)
        gain["gmres30"] = {"applies_per_column": float(g0["iters"].mean()),
                           "ms_per_column": (time.perf_counter() - t0) * 1e3 / cols.size,
                           "fallbacks": int(g0["fallback"].sum())}
        t0 = time.perf_counter()
        loss = lpc.train(1500, 0.2, 0.4, lr=1e-3, seed=5, source="krylov")
        gain["training"] = {"steps": 1500, "s": time.perf_counter() - t0,
                            "loss_first100": float(loss[:100].mean()), "loss_last100": float(loss[-100:].mean())}
        t0 = time.perf_counter()
        g1 = lpc.fgmres_columns(e, ik, cols, maxit=6000, net_every=2)
        gain["fgmres30_net_alternate"] = {"applies_per_column": float(g1["iters"].mean()),
                                          "ms_per_column": (time.perf_counter() - t0) * 1e3 / cols.size,
                                          "fallbacks": int(g1["fallback"].sum()),
                                          "max_abs_dt_vs_plain": float(np.abs(g1["t"] - plain["t"]).max())}
        lpc.close()
    line = {
        "metric": "learned preconditioner: U-Net forward voxels/s on the bulk Cu volume",
        "value": n / (ms / 1e3), "unit": "voxels/s", "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": "U-Net 16/32/64 on 20x20x480 (bulk fcc Cu [001] volume), FP32 input/output, "
                               "BF16 activations and weights, FP32 accumulation",
                   "fgmres_gain_16x16x32_order4": gain,
                   "l2": "activations ~60 MB per forward fit in L2; no flush (the preconditioner re-reads "
                         "its weights every Arnoldi step)"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "whole forward (11 convolutions: k_conv_tc on tcgen05 where the level's plane fits, else "
                               "k_conv on mma.sync; + pool/upsample/concat)",
                     "flops_algorithmic": fl_alg, "flops_padded_channels": fl_pad,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops (measured cuBLAS burst)"},
        "e2e": {"value": n / (e2e_ms / 1e3), "unit": "voxels/s", "h2d_bytes_per_step": n * 16,
                "d2h_bytes_per_step": n * 8},
        "gpu_launches": 18 * steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        # the oracle's forward (NumPy, float64 with the same BF16 rounding points) on a
        # bounded slab of the volume, 20 x 20 x 16 voxels, on one host core
        from oracle import unet as ref

        p = ref.init_params(1)
        xs = np.random.default_rng(0).normal(size=(16, 20, 20, 4))
        ref.forward(p, xs, bf16=True)
        t0 = time.perf_counter()
        reps_cpu = 0
        while time.perf_counter() - t0 < 10.0:
            ref.forward(p, xs, bf16=True)
            reps_cpu += 1
        dt = (time.perf_counter() - t0) / reps_cpu
        line["cpu_baseline"] = {"value": xs[..., 0].size / dt, "unit": "voxels/s", "cores": 1, "kind": "oracle",
                                "sample": f"oracle.unet.forward on a 20x20x16 slab, {reps_cpu} forwards in "
                                          f"{dt * reps_cpu:.1f} s (NumPy; its BLAS kept to one thread by the "
                                          "environment when OMP_NUM_THREADS=1)"}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--form", default="sketch", choices=["sketch", "sketch_fp64", "fp64", "mixed"],
                    help="sketch: full trace from the two-sided sketch (double-float); sketch_fp64: the "
                         "same in FP64; fp64 / mixed: the plain engine on sampled columns")
    ap.add_argument("--window", type=int, default=SKETCH_WINDOW, help="energies per sketch step")
    ap.add_argument("--s-left", type=int, default=SKETCH_LEFT)
    ap.add_argument("--s-right", type=int, default=SKETCH_RIGHT)
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--slots", type=int, default=0)
    ap.add_argument("--items", type=int, default=0, help="column solves per step and GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="small bounded run for ncu: 32 columns, 40 iterations each (with "
                         "--workload learned: 3 forwards and 2 training steps), then exit")
    ap.add_argument("--psym", action="store_true",
                    help="sketch forms: P-symmetric COCG runs (needs --workload cu_bulk_ideal)")
    ap.add_argument("--workload", default="cu_bulk",
                    choices=["cu_bulk", "cu_bulk_ideal", "rh_point_contact", "uneven_batch", "learned",
                             "eigen_stage"],
                    help="rh_point_contact: the 60x60x512 Rh point contact (use --items 16); "
                         "uneven_batch: the 96-cell mixed batch, batched vs looped per cell; "
                         "learned: the U-Net preconditioner's forward and FGMRES gain")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven_batch":
        return run_uneven_batch(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "eigen_stage":
        return run_eigen_stage(args)
    if args.form in ("sketch", "sketch_fp64"):
        return run_sketch(args)

    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from workloads import cu_bulk, rh_point_contact
    import paper_2208_02783_gb300 as pkg
    from paper_2208_02783_gb300 import build, replicas

    pkg.load(build.build())
    rh = args.workload == "rh_point_contact"
    inst = rh_point_contact() if rh else cu_bulk()
    workload_name = WORKLOAD_RH if rh else WORKLOAD
    g = inst.grid
    n_rhs = inst.n_rhs
    reps = k_representatives(inst.kfrac)
    prec = pkg.PREC_MIXED if args.form == "mixed" else pkg.PREC_FP64
    # the timed steps run the library's default path (profile = 0: one graph launch per
    # solve with a device-side loop); kernel times come from a separate profiled pass
    tr = pkg.Transec.from_instance(inst, device=local, tol=1e-10, precision=prec, slots=args.slots,
                                   profile=0)
    slots = args.slots or (16 if prec == pkg.PREC_FP64 else 64)
    tr.set_solver(slots=slots)
    items_per_step = args.items or 2 * slots

    def barrier():
        if ws > 1:
            dist.barrier()

    def step_items(step):
        # one seeded sample of distinct (E, k, column) items per step, split across ranks
        ei, k, c = replicas.step_items(len(inst.energies), reps, n_rhs, items_per_step, step, rank, ws)
        return inst.energies[ei].astype(np.float64), k, c

    dev_items = {}

    def stage(step):
        e, k, c = step_items(step)
        dev_items[step] = (torch.tensor(e, device=dev), torch.tensor(k, device=dev), torch.tensor(c, device=dev))

    def run_device(step):
        return tr.column_contributions(*dev_items.pop(step))

    if args.profile_case:
        # bounded case for the profilers: 32 columns x 40 iterations (they stop as
        # not converged), inputs ~0.4 GB per stencil launch (> L2)
        tr.set_solver(slots=32, maxit=40, profile=1)
        items_per_step = 32
        for s in range(2):
            stage(s)
            run_device(s)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "ok", "stats": tr.stats()}))
        tr.close()
        return 0

    for s in range(args.warmup + args.steps):
        stage(s)
    # warm-up
    for s in range(args.warmup):
        run_device(s)
    torch.cuda.synchronize()
    tr.stats_reset()
    iters_total = 0
    fails = 0
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.start()
    ev0.record()
    results = []
    for s in range(args.steps):
        results.append(run_device(args.warmup + s))
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = ev0.elapsed_time(ev1)
    for r in results:
        iters_total += int(r["iters"].sum().item())
        fails += int((r["status"] != 0).sum().item())
    st = tr.stats()
    ms = replicas.max_over_ranks(ms, device=dev)
    cols = items_per_step * args.steps * ws
    col_rate = replicas.whole_job_rate(items_per_step * args.steps, ws, ms / 1e3)
    value = 2.0 * col_rate / n_rhs

    # parity of the timed form against the plain FP64 form on the first columns of the
    # first timed step (the metric's |dT| <= 1e-6 vs plain FP64 on the GPU)
    parity = None
    if prec == pkg.PREC_MIXED:
        npar = min(16, items_per_step)
        e, k, c = step_items(args.warmup)
        got = results[0]
        tr.set_solver(precision=pkg.PREC_FP64, slots=npar)
        ref = tr.column_contributions(e[:npar], k[:npar], c[:npar])
        tr.set_solver(precision=prec, slots=slots)
        dt_p = np.abs(got["t"][:npar].cpu().numpy() - ref["t"])
        dt_m = np.abs(got["t_minus"][:npar].cpu().numpy() - ref["t_minus"])
        mx = float(max(dt_p.max(), dt_m.max()))
        parity = {"columns": npar, "max_abs_dt_j": mx, "dT_bound_per_Ek": mx * n_rhs,
                  "fp64_status_ok": bool(np.all(ref["status"] == 0))}

    # end to end: host (pinned) item arrays in, host results out, through the C ABI
    e2e_ms = 0.0
    h2d = items_per_step * (8 + 4 + 8)
    d2h = items_per_step * (8 + 8 + 4 + 4)
    barrier()
    for s in range(args.steps):
        e, k, c = step_items(args.warmup + args.steps + s)
        pe, pk, pc = (torch.tensor(e).pin_memory(), torch.tensor(k).pin_memory(), torch.tensor(c).pin_memory())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tr.column_contributions(pe, pk, pc)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = replicas.max_over_ranks(e2e_ms, device=dev)
    e2e_value = 2.0 * replicas.whole_job_rate(items_per_step * args.steps, ws, e2e_ms / 1e3) / n_rhs

    # profiled pass (separate from the timed steps): every slot busy for 400 iterations,
    # each stencil and update launch bracketed by CUDA events on the context's stream
    prof_its = 400
    e, k, c = step_items(args.warmup + 2 * args.steps)
    tr.set_solver(profile=1, maxit=prof_its)
    tr.stats_reset()
    tr.column_contributions(e[:slots], k[:slots], c[:slots])
    stp = tr.stats()
    tr.set_solver(profile=0, maxit=100000)

    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    elem = 16 if prec == pkg.PREC_FP64 else 8
    if prec == pkg.PREC_FP64:
        pa, sten_ms, launches_s = stp["point_applies"], stp["stencil_ms"], stp["stencil_launches"]
    else:  # the FP32 stencil of the mixed form (fallback FP64 work is counted apart)
        pa, sten_ms, launches_s = stp["point_applies32"], stp["stencil32_ms"], stp["stencil32_launches"]
    sten_s = sten_ms / 1e3
    launches_s = max(1, launches_s)
    flops = pa * stencil_flops_per_point(g.order)
    bytes_alg = pa * stencil_bytes_per_point(elem)
    if prec == pkg.PREC_FP64:
        achieved = flops / sten_s / 1e12 if sten_s > 0 else 0.0
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": (FP64_STENCIL_DRAM_PER_POINT_HALF * pa / launches_s
                            if FP64_STENCIL_DRAM_PER_POINT_HALF and not rh else None),
                "kernel": "k_stencil<double,6> (FP64 stencil fused with p = r + beta p and the pairing dot)",
                "per_launch": {"flops": flops / launches_s, "bytes": bytes_alg / launches_s,
                               "ms": sten_ms / launches_s},
                "timing": f"separate profiled pass: {slots} columns x {prof_its} iterations, CUDA events "
                          "around every stencil launch on the context's stream",
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz",
                "hbm_gbs": bytes_alg / sten_s / 1e9 if sten_s > 0 else 0.0,
                "hbm_frac_of_measured": (bytes_alg / sten_s / 1e9) / hbm_peak if sten_s > 0 else 0.0}
    else:
        achieved = bytes_alg / sten_s / 1e9 if sten_s > 0 else 0.0
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None,
                "kernel": "k_stencil<float,6>",
                "per_launch": {"flops": flops / launches_s, "bytes": bytes_alg / launches_s,
                               "ms": sten_ms / launches_s},
                "timing": f"separate profiled pass: {slots} columns x {prof_its} iterations, CUDA events "
                          "around every stencil launch on the context's stream",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128" if prec == pkg.PREC_FP64 else "c64+f64",
        "data": "synthetic",
        "config": {
            "workload": workload_name, "form": ("FP64 transpose BiCG (+-k)" if prec == pkg.PREC_FP64
                                           else "complex FP32 BiCG with FP64 scalars and residual replacement"),
            "column_solves_per_step_per_gpu": items_per_step, "slots": slots,
            "column_solves_per_s": col_rate, "n_rhs_per_Ek": n_rhs,
            "value_derivation": "2 x column-solves/s / n_rhs (each column gives the k and -k columns)",
            "mean_iterations_per_column": iters_total / max(1, cols // ws),
            "failed_columns": fails, "fp64_fallback_columns": int(st.get("fallbacks", 0)), "l2": "working set of the slots (~GBs) exceeds L2; no flush needed",
            "parity_vs_fp64": parity,
            "sampling": "one seeded sample of distinct (energy, k-pair, left-CAP column) items per "
                        "step, split across ranks (rank r takes every N-th item from r)",
        },
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(st["launches"]),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        mean_its = golden_mean_iterations()
        items = draw_items(inst, reps, n_rhs, 64, 7000)
        with OraclePool("rh_point_contact" if rh else "cu_bulk") as op:
            op.rate(inst, items, mean_its, budget_s=1.0)  # operators built, caches warm
            crate, n_it, dt = op.rate(inst, items, mean_its, budget_s=12.0)
            procs = op.procs
        line["cpu_baseline"] = {
            "value": 2.0 * crate / n_rhs, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": (f"oracle transpose BiCG (numpy/scipy complex128), one single-threaded process "
                       f"per core ({procs}), each on its own seeded column of the workload for "
                       f"{n_it} iterations (median; {dt:.1f} s wall); column time = time per iteration "
                       f"x {mean_its:.0f} (oracle mean iterations to 1e-10 over the committed golden "
                       f"columns); rates summed"),
        }
    if rank == 0:
        print(json.dumps(line))
    tr.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
