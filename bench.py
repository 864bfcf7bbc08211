#!/usr/bin/env python3
"""Benchmark of the LS-AMG-DD solve phase on one GB300 (or N replicas).

Workload (default): 512 x 512 Q1 cells (261,121 unknowns), K = R diag(1, eps)
R^T with theta = pi/6, eps = 1e-4, 4 x 4 level-0 aggregates, overlap 1,
LS_{2,3,4} coarsening to <= 2000 unknowns, one N(0,1) right-hand side per
solve, CG to 1e-8 relative residual.

A step is one V-cycle-preconditioned CG solve to 1e-8 of a fresh
right-hand side already resident in device memory (the hierarchy is built
once, before timing).  `value` is solves/s of the mixed-precision form (FP32
V-cycle under FP64 flexible CG); the plain FP64 GPU path is timed on the
same inputs beside it.  `e2e` repeats the timing through the C ABI with
pinned host buffers (host->device copy of b and device->host copy of x
inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank is an independent replica (its own right-hand
sides); value = all solves / max over ranks of the timed wall time.
"""
from __future__ import annotations

import argparse
import csv
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

METRIC = "V-cycles/s & solves/s to 1e-8 rel. residual (mixed vs FP64); p50/p99 latency"
WORKLOAD = "q1_512_rot"
# DRAM bytes per V-cycle by (precision, kernel family), from an ncu capture
# of WORKLOAD (dram__bytes_read.sum + dram__bytes_write.sum summed over one
# V-cycle's launches, FP32 cycle; profiles/).  Entries are removed when their
# kernels change.
TRAFFIC = {(1, "k_seg"): 881.04e6, (1, "k_ell"): 41.80e6, (1, "k_dense"): 29.42e6}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--theta", type=float, default=None)
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--N", type=int, default=None, help="cells per axis (smaller captures)")
    ap.add_argument("--sweep", action="store_true",
                    help="run the eps x theta sweep of the workload instead (one setup per point)")
    ap.add_argument("--serve", action="store_true",
                    help="run the serving workload (many operators and right-hand-side counts) instead")
    ap.add_argument("--no-serving", action="store_true", help="skip the small serving run of the default line")
    ap.add_argument("--serve-kappa", action="store_true",
                    help="with --serve-mix: operators by the kappa threshold (Section 3.4) instead of LS_{2,3,4}")
    ap.add_argument("--serve-mix", action="store_true",
                    help="run the serving mix with setup on the request path (operators carried by the requests; "
                         "sides 32..256, 1..64 right-hand sides; a one-at-a-time FP64 loop beside it) instead")
    ap.add_argument("--additive", action="store_true",
                    help="time PCG with the additive two-level method (cycle = 1) beside the multiplicative two-level "
                         "cycle, FP64, on the 64x64 workload's two-level hierarchy, instead")
    ap.add_argument("--deterministic", action="store_true",
                    help="build the hierarchy in deterministic mode (no atomics; bitwise repeatable solves)")
    ap.add_argument("--tune-mode", choices=("timed", "defaults", "staged", "shifted", "lanes"), default="timed",
                    help="setup-time kernel choices: timed (default), fixed defaults, or the staged kernel, "
                         "shifted vector loads or lanes per row wherever a plan allows them (profiling)")
    ap.add_argument("--tune-cache", default=None,
                    help="file of setup-time kernel choices: read if present, written after tuning "
                         "(profiling runs replay the choices of a plain run)")
    ap.add_argument("--ls-study", choices=("eps", "size", "angle"), default=None,
                    help="Section 4.1's finite-difference studies of the LS variants (FP64 iterations per digit, "
                         "convergence factor, operator complexity) over eps, grid size or angle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="setup + a few solves, no timing line")
    ap.add_argument("--oracle-solve", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def setup_rates(stats, fp64_gflops):
    """Setup phases: counted FP64 GFLOP (a model from the block sizes), milliseconds, GFLOP/s and the fraction of
    the device's measured FP64 FMA rate (amgdd_measure_fp64)."""
    out = {"fp64_gflops_measured": round(fp64_gflops, 1), "phases": {}}
    for k, gf in stats.get("setup_phases_gflop", {}).items():
        ms = stats["setup_phases_ms"].get(k, 0.0)
        rate = gf / (ms * 1e-3) if ms > 0 else None
        out["phases"][k] = {"gflop": round(gf, 3), "ms": round(ms, 1), "gflops": None if rate is None else round(rate, 1),
                            "frac_of_fp64": None if rate is None else round(rate / fp64_gflops, 4)}
    return out


def replica_max(v, world, device="cuda"):
    """Max of a per-rank value over the replicas (the slowest rank's time
    sets whole-job throughput); the identity with one rank."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, seconds, world, device="cuda"):
    """Whole-job rate of independent replicas: every rank's units over the
    slowest rank's time (weak scaling: per-rank work fixed)."""
    return units_per_rank * world / replica_max(seconds, world, device)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 50 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for row in csv.reader(f):
                if len(row) < 9:
                    continue
                try:
                    sm.append(float(row[1]))
                    mx = float(row[2])
                except ValueError:
                    continue
                for nm, v in zip(names, row[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def workload_desc(cfg):
    if cfg.get("field") == "fd":
        return (f"{cfg['N']}x{cfg['N']} finite-difference unknowns (G = B^T grad^+, Dirichlet), "
                f"theta={cfg['theta']:.6f}, eps={cfg['eps']:g}, "
                + (f"{cfg['bs']}x{cfg['bs']} aggregates, " if cfg['bs'] else
                   f"standard aggregation ({cfg.get('agg_passes', 1)} pass), ") +
                f"overlap {cfg['overlap']}, LS_{{{','.join(str(c) for c in cfg['c_min'])}}}, "
                f"thresh from kappa={cfg['kappa']:g}, n_coarse {cfg['n_coarse']}, 1 RHS, tol 1e-8")
    if cfg.get("dim", 2) == 3:
        return (f"{cfg['N']}^3 Q1 hexahedral cells ({(cfg['N'] - 1) ** 3:,} unknowns), K = eps I + (1-eps) b b^T with "
                f"b a smooth seeded Fourier field, eps={cfg['eps']:g}, greedy strength-graph aggregates "
                f"(theta {cfg.get('soc', 0.03)}), overlap {cfg['overlap']}, "
                f"LS_{{{','.join(str(c) for c in cfg['c_min'])}}}, n_coarse {cfg['n_coarse']}, 1 RHS, tol 1e-8")
    field = (f"theta={cfg['theta']:.6f}" if cfg.get("field", "rot") == "rot"
             else "circular field theta=atan2(y-1/2, x-1/2)+pi/2")
    d1 = f", D1={cfg['d1']:g} h^2" if cfg.get("d1") else ""
    ov = f"overlap {cfg['overlap']}" + (f" (level 0), {cfg['coarse_overlap']} (coarse levels)"
                                        if cfg.get("coarse_overlap") else "")
    return (f"{cfg['N']}x{cfg['N']} Q1 cells ({(cfg['N'] - 1) ** 2:,} unknowns), {field}, "
            f"eps={cfg['eps']:g}{d1}, {cfg['bs']}x{cfg['bs']} aggregates, {ov}, "
            f"LS_{{{','.join(str(c) for c in cfg['c_min'])}}}, n_coarse {cfg['n_coarse']}, 1 RHS, tol 1e-8")


def oracle_setup(prob, cfg):
    """The oracle's own hierarchy for the workload (not timed)."""
    import oracle

    t0 = time.time()
    agg = prob.agg
    if agg is None:  # the oracle's own standard aggregation (Section 3.3)
        sups, _ = oracle.construct.row_groups_from_csr(prob.rowptr, prob.col, prob.val, prob.n, prob.D1)
        agg, _ = oracle.standard_aggregation(sups, prob.n, cfg.get("agg_passes", 1))
    ho = oracle.setup(prob.rowptr, prob.col, prob.val, prob.n, prob.D1, agg, overlap=cfg["overlap"],
                      c_min=cfg["c_min"], n_coarse=cfg["n_coarse"], thresh=cfg["thresh"],
                      kappa=cfg.get("kappa") or None, coarse_overlap=cfg.get("coarse_overlap", 0))
    setup_s = time.time() - t0
    return ho, setup_s


def convergence(info):
    """Average convergence factor rho = (||r_k|| / ||r_0||)^(1/k) of an FP64 solve and the iterations per
    tenfold residual reduction, log(0.1) / log(rho) (the measure of Section 4.1's studies)."""
    k, rr = info["iters"], info["relres"]
    if k < 1 or not rr > 0:
        return {"rho_fp64": None, "iters_per_digit": None}
    rho = rr ** (1.0 / k)
    return {"rho_fp64": round(rho, 4), "iters_per_digit": round(math.log(0.1) / math.log(rho), 3) if rho < 1 else None}


def cpu_threads():
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return os.cpu_count() or 1


def oracle_solve_sample(args):
    """One oracle CG solve of a given right-hand side (runs in its own process)."""
    import numpy as np

    import oracle
    from inputs.q1 import config_problem

    d = np.load(args.oracle_solve)
    over = {k: float(d[k]) for k in ("theta", "eps") if k in d}
    if "N" in d:
        over["N"] = int(d["N"])
    prob, cfg = config_problem(args.workload, **over)
    ho, setup_s = oracle_setup(prob, cfg)
    t0 = time.time()
    xo, io = oracle.pcg(ho, d["b"], tol=1e-8)
    solve_s = time.time() - t0
    err = float(np.abs(xo - d["x"]).max() / np.abs(xo).max())
    out = {"setup_s": setup_s, "solve_s": solve_s, "iters": io["iters"], "err": err, "cores": cpu_threads()}
    # all cores: one single-threaded solve per core, each of its own seeded
    # right-hand side, in forked workers sharing the hierarchy (this process
    # never touches a GPU, so forking is safe here)
    ncores = os.cpu_count() or 1
    if ncores > 1:
        import multiprocessing as mp

        from inputs import seeded_rhs

        global _ORACLE_H
        _ORACLE_H = ho
        B = seeded_rhs(prob.n, ncores, 7919)
        t0 = time.time()
        with mp.get_context("fork").Pool(ncores) as pool:
            its = pool.map(_oracle_pcg_iters, [B[:, j].copy() for j in range(ncores)])
        wall = time.time() - t0
        out["all_cores"] = {"solves": ncores, "wall_s": wall, "iters": its, "cores": ncores}
    print(json.dumps(out), flush=True)


_ORACLE_H = None


def _oracle_pcg_iters(b):
    """Worker of the all-cores oracle sample: one CG solve on the inherited hierarchy."""
    import oracle

    return int(oracle.pcg(_ORACLE_H, b, tol=1e-8)[1]["iters"])


def run_reference(args):
    """The oracle on the host cores, same workload, metric and unit."""
    rank, world, local = dist_info()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from inputs.q1 import config_problem, seeded_rhs

    over = {}
    if args.theta is not None:
        over["theta"] = args.theta
    if args.eps is not None:
        over["eps"] = args.eps
    if args.N is not None:
        over["N"] = args.N
    prob, cfg = config_problem(args.workload, **over)
    ho, setup_s = oracle_setup(prob, cfg)
    b = seeded_rhs(prob.n, 1, cfg["seed"] * 1000)[:, 0]
    # one full solve gives the iteration count; each timed step is one
    # CG iteration (A-apply, V-cycle, updates) of that solve
    t0 = time.time()
    x, info = oracle.pcg(ho, b, tol=1e-8)
    full_s = time.time() - t0
    iters = info["iters"]
    # one preconditioned CG iteration (the recurrences of oracle.pcg)
    A0 = ho.levels[0]
    r = b.copy()
    z = oracle.vcycle(ho, r)
    p = z.copy()
    xk = np.zeros_like(b)
    rz = float(r @ z)
    times = []
    for step in range(args.warmup + args.steps):
        t = time.time()
        q = oracle.apply_A(A0, p)
        alpha = rz / float(p @ q)
        xk += alpha * p
        r -= alpha * q
        z = oracle.vcycle(ho, r)
        rzn = float(r @ z)
        p = z + (rzn / rz) * p
        rz = rzn
        if step >= args.warmup:
            times.append(time.time() - t)
        if step + 1 >= iters:  # restart from the first iterate to stay on the solve's path
            r = b.copy()
            z = oracle.vcycle(ho, r)
            p = z.copy()
            rz = float(r @ z)
    t_iter = sum(times) / len(times)
    value = 1.0 / (t_iter * iters)
    cores = cpu_threads()
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_iter * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_desc(cfg)},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"oracle setup untimed ({setup_s:.1f} s); each step one CG iteration of the "
                                       f"oracle's solve, solves/s = 1/(mean step time x {iters} iterations); "
                                       f"one full oracle solve took {full_s:.1f} s"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serving_run(amg, seed, sides, nops, nreq, max_rhs, rate_frac=0.8, slots=4):
    """Requests over a pool of operators of several grid sizes through the
    continuous-batching server: throughput with every request queued at once,
    then latency under open-loop Poisson arrivals at rate_frac of it.
    Operators: sides cycle through `sides`, theta ~ U[0, pi), eps
    log-uniform in [1e-6, 1], 4x4 aggregates, LS_{2,3,4}, mixed precision;
    requests: a uniform operator and 1..max_rhs right-hand sides."""
    import numpy as np
    from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK, seeded_rhs

    rng = np.random.default_rng(seed)
    srv = amg.Server(slots=slots)
    ops = []
    t0 = time.perf_counter()
    for j in range(nops):
        N = sides[j % len(sides)]
        theta, eps = float(rng.uniform(0.0, math.pi)), float(10.0 ** rng.uniform(-6.0, 0.0))
        prob = q1_2d(N, rotated_sqrtK(theta, eps), agg=block_aggregates_2d(N, 4))
        op, _ = srv.add_operator(prob, key=j, c_min=(2, 3, 4), n_coarse=2000, precision=amg.MIXED32)
        ops.append((op, prob.n))
    setup_s = time.perf_counter() - t0
    reqs = []
    for i in range(nreq):
        k = int(rng.integers(nops))
        reqs.append((ops[k][0], seeded_rhs(ops[k][1], int(rng.integers(1, max_rhs + 1)), seed * 100000 + i)))
    cols = sum(B.shape[1] for _, B in reqs)
    # saturation: everything queued at once
    t0 = time.perf_counter()
    rids = [srv.submit(op, B) for op, B in reqs]
    for rid in rids:
        r = srv.poll(rid)
        assert r[3] == 0, r[1]
    sat = time.perf_counter() - t0
    s_sat = srv.stats()
    # open loop at rate_frac of the saturated request rate
    lam = rate_frac * nreq / sat
    gaps = rng.exponential(1.0 / lam, nreq)
    lats = []
    t0 = time.perf_counter()
    due = t0
    pending = []
    for (op, B), g in zip(reqs, gaps):
        due += g
        while time.perf_counter() < due:
            pass
        pending.append(srv.submit(op, B))
    for rid in pending:
        x, infos, lat, st = srv.poll(rid)
        assert st == 0
        lats.append(lat)
    s_all = srv.stats()
    srv.close()
    lats.sort()
    pct = lambda q: lats[min(len(lats) - 1, int(q * len(lats)))]
    return {"operators": nops, "sides": list(sides), "requests": nreq, "rhs_columns": cols, "slots": slots,
            "setup_s": setup_s, "saturated": {"requests_per_s": nreq / sat, "solves_per_s": cols / sat,
                                              "mean_batch_columns": s_sat["mean_batch_columns"],
                                              "p50_ms": s_sat["p50_ms"], "p99_ms": s_sat["p99_ms"]},
            "open_loop": {"rate_per_s": lam, "p50_ms": pct(0.5), "p99_ms": pct(0.99),
                          "mean_batch_columns": (s_all["mean_batch_columns"] * s_all["batches"] -
                                                 s_sat["mean_batch_columns"] * s_sat["batches"]) /
                          max(1, s_all["batches"] - s_sat["batches"])},
            "precision": "mixed", "data": "synthetic, seeded"}


def serving_mix_run(amg, seed, sides, nreq, max_rhs, pool=None, rate_fracs=(0.5, 0.8, 1.0), slots=4, kappa=False):
    """The serving mix with setup on the request path: every request carries its operator, a 2D Q1 problem with
    side drawn uniformly from `sides`, theta ~ U[0, pi), eps log-uniform in [1e-6, 1], 4x4 aggregates, LS_{2,3,4},
    mixed precision, and 1..max_rhs N(0,1) right-hand sides.  pool = None: a new operator per request (no
    reuse); pool = P: operators drawn from a seeded pool of P.  Latency is arrival -> result.  Reported: the
    saturated rate (everything arrives at once), open-loop Poisson arrivals at rate_fracs of it (each run with
    operators keyed afresh, so that setup stays on the request path), and a one-at-a-time FP64 loop over the same
    requests (setup and solve per request, nothing overlapped, each operator built once).  Both build with the
    fixed kernel choices (tune = 0).  kappa: every operator takes the kappa-derived threshold of Section 3.4
    (kappa = 50) with no cap on the kept eigenvectors instead of LS_{2,3,4}."""
    import numpy as np
    import torch
    from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK, seeded_rhs

    rng = np.random.default_rng(seed)
    nops = nreq if pool is None else pool
    opdefs = []
    for j in range(nops):
        N = int(sides[int(rng.integers(len(sides)))])
        theta, eps = float(rng.uniform(0.0, math.pi)), float(10.0 ** rng.uniform(-6.0, 0.0))
        opdefs.append(q1_2d(N, rotated_sqrtK(theta, eps), agg=block_aggregates_2d(N, 4)))
    reqs = []
    for i in range(nreq):
        k = i if pool is None else int(rng.integers(nops))
        reqs.append((k, seeded_rhs(opdefs[k].n, int(rng.integers(1, max_rhs + 1)), seed * 100000 + i)))
    cols = sum(B.shape[1] for _, B in reqs)
    # setup on the request path takes the fixed kernel choices (tune = 0): timing the forms of every new
    # operator costs more than it saves on a request's few solves, and builds overlap other work on the GPU
    lsk = dict(c_min=(1,), kappa=50.0) if kappa else dict(c_min=(2, 3, 4))
    kw = dict(n_coarse=2000, precision=amg.MIXED32, tune=0, **lsk)

    def run(key0, rate):
        srv = amg.Server(slots=slots)
        gaps = rng.exponential(1.0 / rate, nreq) if rate else np.zeros(nreq)
        t0 = time.perf_counter()
        due = t0
        sub = []
        for (k, B), g in zip(reqs, gaps):
            due += g
            while time.perf_counter() < due:
                time.sleep(0)
            sub.append(srv.submit_problem(opdefs[k], key=key0 + k, b=B, **kw)[0])
        lats = []
        for rid in sub:
            x, infos, lat, st = srv.poll(rid)
            assert st == 0 and all(i["relres_true"] <= 1e-8 for i in infos), infos
            lats.append(lat)
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lats.sort()
        pct = lambda q: lats[min(len(lats) - 1, int(q * len(lats)))]
        return {"requests_per_s": nreq / wall, "solves_per_s": cols / wall, "p50_ms": pct(0.5),
                "p99_ms": pct(0.99), "builds": st["builds"], "setup_ms_total": st["build_ms_total"],
                "cache_hits": st["cache_hits"], "mean_batch_columns": st["mean_batch_columns"],
                "evictions": st["evictions"], "waits_for_memory": st["waits_for_memory"]}

    sat = run(1 << 40, None)
    open_loop = []
    for j, f in enumerate(rate_fracs):
        r = run((j + 2) << 40, f * sat["requests_per_s"])
        r["rate_frac_of_saturation"] = f
        open_loop.append(r)
    # one request at a time, FP64, no server: setup and solve of each request in turn
    t0 = time.perf_counter()
    built = {}
    lat1 = []
    for k, B in reqs:
        t1 = time.perf_counter()
        if k not in built:  # the loop keeps what it built (a pool reuses its operators)
            built[k] = amg.Hierarchy.from_problem(opdefs[k], overlap=1, n_coarse=2000, tune=0, **lsk)
        H = built[k]
        _, inf = H.solve(B, tol=1e-8)
        assert all(i["relres_true"] <= 1e-8 for i in inf)
        lat1.append((time.perf_counter() - t1) * 1e3)
    torch.cuda.synchronize()
    loop_s = time.perf_counter() - t0
    lat1.sort()
    return {"requests": nreq, "rhs_columns": cols, "sides": list(sides), "max_rhs": max_rhs,
            "operators": "one per request" if pool is None else f"pool of {pool}", "slots": slots,
            "saturated": sat, "open_loop": open_loop,
            "fp64_one_at_a_time": {"requests_per_s": nreq / loop_s, "solves_per_s": cols / loop_s,
                                   "service_p50_ms": lat1[len(lat1) // 2],
                                   "service_p99_ms": lat1[min(len(lat1) - 1, int(0.99 * len(lat1)))]},
            "precision": "mixed (FP32 V-cycle, FP64 flexible CG) in the server", "data": "synthetic, seeded",
            "coarsening": "kappa = 50, no cap" if kappa else "LS_{2,3,4}"}


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    import paper_2601_04112_gb300 as amg
    from inputs.q1 import config_problem, seeded_rhs

    if args.additive:
        # the additive two-level method M_2 against the multiplicative two-level
        # V-cycle on the same two-level hierarchy (FP64 PCG to 1e-8)
        name = "q1_64_rot" if args.workload == WORKLOAD else args.workload
        prob, cfg = config_problem(name)
        b = torch.from_numpy(seeded_rhs(prob.n, 1, cfg["seed"])[:, 0]).cuda()
        out = {"metric": "solves/s to 1e-8 rel. residual, additive two-level M_2 vs multiplicative two-level cycle "
                         "(FP64)", "impl": "ours", "workload": workload_desc(cfg) + ", L_max 2"}
        for label, cyc in (("multiplicative", 0), ("additive", 1)):
            Hc = amg.Hierarchy.from_problem(prob, overlap=cfg["overlap"], c_min=cfg["c_min"],
                                            n_coarse=cfg["n_coarse"], thresh=cfg["thresh"], kappa=cfg.get("kappa", 0.0), agg_passes=cfg.get("agg_passes", 1), L_max=2, cycle=cyc)
            for _ in range(args.warmup):
                Hc.solve(b, tol=1e-8)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its = []
            for _ in range(args.steps):
                _, inf = Hc.solve(b, tol=1e-8)
                assert inf[0]["status"] == 0 and inf[0]["relres_true"] <= 1e-8, inf
                its.append(inf[0]["iters"])
            torch.cuda.synchronize()
            out[label] = {"solves_per_s": args.steps / (time.perf_counter() - t0), "iters": its[0],
                          "levels": Hc.stats()["n"]}
        if rank == 0:
            print(json.dumps(out), flush=True)
        return

    if args.sweep:
        # the (eps, theta) sweep of the 512x512 workload: setup, iterations and
        # solves/s in both precisions per point
        from inputs.q1 import SWEEP_EPS, SWEEP_THETA

        rows = []
        for eps in SWEEP_EPS:
            for theta in SWEEP_THETA:
                prob, cfg = config_problem(args.workload, eps=eps, theta=theta)
                t0 = time.time()
                Hs = amg.Hierarchy.from_problem(prob, overlap=cfg["overlap"], c_min=cfg["c_min"],
                                                n_coarse=cfg["n_coarse"], thresh=cfg["thresh"], kappa=cfg.get("kappa", 0.0), agg_passes=cfg.get("agg_passes", 1),
                                                coarse_overlap=cfg.get("coarse_overlap", 0))
                torch.cuda.synchronize()
                row = {"eps": eps, "theta": round(theta, 6), "setup_s": round(time.time() - t0, 3),
                       "levels": Hs.stats()["n"]}
                b = torch.from_numpy(seeded_rhs(prob.n, 1, cfg["seed"])[:, 0]).cuda()
                for name, prec in (("mixed", amg.MIXED32), ("fp64", amg.FP64)):
                    Hs.set_precision(prec)
                    Hs.solve(b, tol=1e-8)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    its, fb, ok = [], 0, True
                    for _ in range(5):
                        _, inf = Hs.solve(b, tol=1e-8)
                        ok = ok and inf[0]["status"] == 0 and inf[0]["relres_true"] <= 1e-8
                        its.append(inf[0]["iters"])
                        fb = inf[0]["fallback"]
                    torch.cuda.synchronize()
                    row[name] = {"iters": its[0], "solves_per_s": round(5 / (time.perf_counter() - t0), 2)}
                    if fb:
                        row[name]["fp64_fallback_after"] = inf[0]["iters_mixed"]
                    if not ok:
                        row[name]["failed"] = {"status": inf[0]["status"], "relres_true": inf[0]["relres_true"]}
                print(json.dumps(row), file=sys.stderr, flush=True)
                rows.append(row)
                del Hs
        if rank == 0:
            print(json.dumps({"metric": "eps x theta sweep (solves/s to 1e-8, iterations)", "impl": "ours",
                              "workload": args.workload, "points": rows}), flush=True)
        return

    if args.ls_study:
        # Section 4.1: theta = pi/6, eps from 1 to 1e-7 on 500^2; eps = 1e-5 up to 1000^2; angles in (0, pi/2)
        variants = {"LS_4": (4,), "LS_3,4": (3, 4), "LS_2,3": (2, 3), "LS_3": (3,), "LS_2,3,4": (2, 3, 4)}
        if args.ls_study == "eps":
            points = [dict(eps=10.0 ** -k) for k in range(8)]
        elif args.ls_study == "size":
            points = [dict(eps=1e-5, N=N) for N in (125, 250, 500, 1000)]
        else:
            points = [dict(eps=1e-5, theta=math.pi / 2 * j / 8) for j in range(1, 8)]
            variants = {"LS_2,3,4": (2, 3, 4)}
        rows = []
        for pt in points:
            for vname, cm in variants.items():
                prob, cfg = config_problem("fd_500_rot", c_min=cm, **pt)
                t0 = time.time()
                Hs = amg.Hierarchy.from_problem(prob, overlap=cfg["overlap"], c_min=cm, n_coarse=cfg["n_coarse"],
                                                thresh=cfg["thresh"], kappa=cfg["kappa"],
                                                agg_passes=cfg.get("agg_passes", 1))
                torch.cuda.synchronize()
                setup_s = time.time() - t0
                st = Hs.stats()
                b = torch.from_numpy(seeded_rhs(prob.n, 1, cfg["seed"])[:, 0]).cuda()
                _, inf = Hs.solve(b, tol=1e-8)
                row = {"variant": vname, **{k: (round(v, 6) if isinstance(v, float) else v) for k, v in pt.items()},
                       "n": prob.n, "iters": inf[0]["iters"], "status": inf[0]["status"],
                       "relres_true": inf[0]["relres_true"], **convergence(inf[0]),
                       "op_complexity": round(st["op_complexity"], 3), "levels": st["n"],
                       "thresh": [round(t, 4) for t in st["thresh"]], "setup_s": round(setup_s, 2)}
                print(json.dumps(row), file=sys.stderr, flush=True)
                rows.append(row)
                del Hs
        if rank == 0:
            print(json.dumps({"metric": f"LS variants over {args.ls_study} (FP64 PCG to 1e-8)", "impl": "ours",
                              "workload": workload_desc(config_problem("fd_500_rot")[1]), "points": rows}),
                  flush=True)
        return

    if args.serve_mix:
        # the serving mix with setup on the request path (literal: a new operator per request; and a pool of 16)
        out = {"metric": "serving with setup on the request path: solves/s and p50/p99 latency (mixed)",
               "impl": "ours", "n_gpus": world,
               "literal": serving_mix_run(amg, seed=5, sides=(32, 64, 128, 256), nreq=48, max_rhs=64,
                                          kappa=args.serve_kappa)}
        if not args.serve_kappa:
            out["pool"] = serving_mix_run(amg, seed=6, sides=(32, 64, 128, 256), nreq=192, max_rhs=64, pool=16)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return

    if args.serve:
        # the serving workload on its own: operators of 32^2 .. 512^2 cells,
        # 1..64 right-hand sides per request
        out = serving_run(amg, seed=5, sides=(32, 64, 128, 256, 512), nops=10, nreq=512, max_rhs=64)
        if rank == 0:
            print(json.dumps({"metric": "serving solves/s and p50/p99 latency (mixed)", "impl": "ours",
                              "n_gpus": world, **out}), flush=True)
        return

    over = {}
    if args.theta is not None:
        over["theta"] = args.theta
    if args.eps is not None:
        over["eps"] = args.eps
    if args.N is not None:
        over["N"] = args.N
    prob, cfg = config_problem(args.workload, **over)
    n = prob.n
    t0 = time.time()
    H = amg.Hierarchy.from_problem(prob, overlap=cfg["overlap"], c_min=cfg["c_min"], n_coarse=cfg["n_coarse"],
                                   thresh=cfg["thresh"], kappa=cfg.get("kappa", 0.0), agg_passes=cfg.get("agg_passes", 1), precision=amg.MIXED16, tune_cache=args.tune_cache,
                                   coarse_overlap=cfg.get("coarse_overlap", 0),
                                   tune={"timed": 1, "defaults": 0, "staged": 2, "shifted": 3, "lanes": 4}[args.tune_mode],
                                   deterministic=1 if args.deterministic else 0, batch_cols=32)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    stats = H.stats()
    nsol = args.warmup + args.steps
    Bh = seeded_rhs(n, nsol, cfg["seed"] * 1000 + rank)  # n x nsol, column-major
    B = torch.from_numpy(np.ascontiguousarray(Bh.T)).cuda()  # row j = right-hand side j
    X = torch.zeros_like(B)

    def timed(prec, start, count, bsrc, xdst):
        H.set_precision(prec)
        infos = []
        dev = bsrc.is_cuda
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k0 = amg.kernel_launches()
        w0 = time.perf_counter()
        e0.record()
        for j in range(start, start + count):
            _, inf = H.solve(bsrc[j] if dev else bsrc[j].numpy(), x=xdst[j] if dev else xdst[j].numpy())
            infos.append(inf[0])
        e1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        return e0.elapsed_time(e1) / 1e3, wall, infos, amg.kernel_launches() - k0

    def maxrank(v):
        return replica_max(v, world)

    # warm-up (every precision: graph capture, first-touch)
    for prec in (amg.FP64, amg.MIXED32, amg.MIXED16):
        timed(prec, 0, args.warmup, B, X)
    HEAD = amg.MIXED32  # the headline precision: FP32 V-cycle, FP64 flexible CG (MIXED16 reported beside it)
    if args.profile_only:
        H.set_precision(HEAD)
        # the NVTX range lets a profiler select these V-cycles (setup's own
        # tuning launches run the same kernels)
        torch.cuda.nvtx.range_push("vcycle_profile")
        ms, by, _ = H.profile_vcycle(10, graph=True)
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"stats": stats, "profile_ms": ms.tolist(), "profile_bytes": by.tolist()}))
        return
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)  # nvidia-smi's own start-up, so that its samples fall inside the timed region
    t_mix, w_mix, inf_mix, launches = timed(HEAD, args.warmup, args.steps, B, X)
    clocks = sampler.stop()
    t_16, w_16, inf_16, _ = timed(amg.MIXED16, args.warmup, args.steps, B, X)
    t_64, w_64, inf_64, _ = timed(amg.FP64, args.warmup, args.steps, B, X)
    t_mix = maxrank(t_mix)
    t_16 = maxrank(t_16)
    t_64 = maxrank(t_64)
    for inf in inf_mix + inf_16 + inf_64:
        assert inf["status"] == 0 and inf["relres_true"] <= 1e-8, inf
    fallbacks = sum(i["fallback"] for i in inf_mix)
    it_mix = [i["iters"] for i in inf_mix]
    it_64 = [i["iters"] for i in inf_64]
    solves = args.steps * world
    value = solves / t_mix
    fp64_value = solves / t_64
    m16_value = solves / t_16
    vc_mix = sum(i + 1 for i in it_mix) * world / t_mix
    vc_64 = sum(i + 1 for i in it_64) * world / t_64
    lat = sorted(i["solve_ms"] for i in inf_mix)

    # per-step V-cycle profile -> roofline.  The primary figures replay the
    # cycle as a CUDA graph with event record nodes between its kernels (the
    # solve replays its cycle as a graph too); the eager profile (events
    # between separately launched kernels, host launch gaps included) is
    # reported beside it.
    forms = [c["form"] for c in stats["coarse_A"]]
    dense_l = stats.get("dense_tail", {}).get("mixed", {}).get("from", 0)
    peak, peak_kind = hbm_peak()

    def families(ms, by):
        # kernel families by profile slot: slot 6 is the persistent tail (one
        # cooperative launch for every level from its first), slot 2 the two
        # residuals (k_seg over block rows or grouped k_apply), slots 1/5 casts
        fam_ms, fam_by, fam_n = {}, {}, {}
        for l in range(ms.shape[0]):
            for k in range(ms.shape[1]):
                if ms[l, k] <= 0:
                    continue
                if k == 6:
                    fam, nk = "k_persistent", 1
                elif k == 0 and dense_l > 0 and l == dense_l:
                    fam, nk = "k_dense", 1
                elif k == 2:
                    fam, nk = {"block rows": "k_seg", "ELL rows": "k_ell"}.get(forms[l], "k_apply"), 2
                elif k in (1, 5):
                    fam, nk = "k_cast", 1
                else:
                    fam, nk = "k_seg", 1
                fam_ms[fam] = fam_ms.get(fam, 0.0) + float(ms[l, k])
                fam_by[fam] = fam_by.get(fam, 0.0) + float(by[l, k])
                fam_n[fam] = fam_n.get(fam, 0) + nk
        return fam_ms, fam_by, fam_n

    def roofline_of(prec, kdesc_seg):
        H.set_precision(prec)
        ms, by, cyc_graph_ms = H.profile_vcycle(10, graph=True)
        ms_e, by_e = H.profile_vcycle(10)
        fam_ms, fam_by, fam_n = families(ms, by)
        fam_ms_e, fam_by_e, _ = families(ms_e, by_e)
        top = max(fam_ms, key=fam_ms.get)
        kdesc = {"k_seg": kdesc_seg,
                 "k_apply": "k_apply (grouped G then G^T residual; FP32)",
                 "k_persistent": "k_persistent (cooperative V-cycle tail: every phase of the coarse levels; FP32)",
                 "k_dense": "k_dense (dense V-cycle tail GEMV; FP32)",
                 "k_ell": "k_ell (level-0 residual by ELL rows of A; FP32)",
                 "k_cast": "k_cast"}
        # the event record nodes of the marked graph add their own gaps, so the
        # family's time inside the plain graph is taken as its share of the
        # marked cycle applied to the plain cycle's replay time
        kby = fam_by[top]
        share = fam_ms[top] / float(ms.sum())
        kms = cyc_graph_ms * share
        achieved = kby / (kms * 1e-3) / 1e9
        # DRAM bytes per V-cycle of a kernel family from an ncu capture of this
        # workload (profiles/); valid only while those kernels are unchanged
        traffic = (TRAFFIC.get((prec, top)) if args.workload == WORKLOAD and args.N is None and not args.deterministic
                   and args.tune_mode == "timed" else None)
        cyc_bytes = float(by.sum())
        kms_e = fam_ms_e.get(top, 0.0)
        rl = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
              "traffic": traffic, "traffic_unit": "bytes per V-cycle (kernel family)",
              "kernel": kdesc.get(top, top), "launches_per_vcycle": fam_n[top],
              "bytes_per_vcycle": kby, "ms_per_vcycle": kms,
              "timing": ("V-cycle replayed as a CUDA graph (CUDA events around the replay); the family's time is "
                         "its share of the same cycle replayed with event record nodes between its kernels"),
              "share_of_vcycle": share,
              "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
              "families": {f: {"ms_marked": round(fam_ms[f], 4),
                               "gbs": round(fam_by[f] / (cyc_graph_ms * fam_ms[f] / float(ms.sum()) * 1e-3) / 1e9,
                                            1),
                               "launches": fam_n[f]} for f in fam_ms},
              "eager": {"ms": round(kms_e, 4),
                        "frac": (fam_by_e.get(top, 0.0) / (kms_e * 1e-3) / 1e9 / peak) if kms_e > 0 else None,
                        "timing": "separate launches, CUDA events between them (host launch gaps included)"},
              "vcycle": {"ms_graph": cyc_graph_ms, "ms_marked_graph": float(ms.sum()), "bytes": cyc_bytes,
                         "achieved_gbs": cyc_bytes / (cyc_graph_ms * 1e-3) / 1e9,
                         "frac": cyc_bytes / (cyc_graph_ms * 1e-3) / 1e9 / peak}}
        return rl, ms, by

    roofline16, _, _ = roofline_of(
        amg.MIXED16, "k_seg (batched gather-GEMV-scatter: RAS, RAS-T, P, R, block-row residuals; FP16 matrices "
                     "where setup timed them faster, else FP32; FP32 vectors)")
    roofline, ms, by = roofline_of(
        HEAD, "k_seg (batched gather-GEMV-scatter: RAS, RAS-T, P, R, block-row residuals; FP32)")
    slot_names = {0: "ras_coarse_or_dense", 1: "cast_in", 2: "residual_applies", 3: "restrict", 4: "prolong",
                  5: "cast_out", 6: "persistent_tail", 7: "rast"}
    vprof = []
    for l in range(ms.shape[0]):
        vprof.append({slot_names[k]: [round(float(ms[l, k]) * 1e3, 1),
                                      round(float(by[l, k]) / max(float(ms[l, k]) * 1e-3, 1e-12) / 1e9)]
                      for k in slot_names if ms[l, k] > 0})

    # end to end through the C ABI with pinned host buffers
    Bp = torch.empty((nsol, n), dtype=torch.float64, pin_memory=True)
    Bp.copy_(B.cpu())
    Xp = torch.zeros_like(Bp).pin_memory()
    t_e2e, w_e2e, inf_e2e, _ = timed(HEAD, args.warmup, args.steps, Bp, Xp)
    t_e2e = maxrank(max(t_e2e, w_e2e))
    e2e = {"value": solves / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8}

    # batched right-hand sides: batches of 8 columns (each its own CG) share
    # every V-cycle launch; same right-hand sides, both precisions
    def timed_batched(prec, nbatch, K=8):
        H.set_precision(prec)
        Bk = torch.from_numpy(np.ascontiguousarray(seeded_rhs(n, K, cfg["seed"] * 1000 + 500 + rank))).cuda()
        H.solve(Bk, tol=1e-8)  # warm-up (graph capture)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        its = []
        for _ in range(nbatch):
            _, inf = H.solve(Bk, tol=1e-8)
            its.append(max(i["iters"] for i in inf))
            assert all(i["status"] == 0 and i["relres_true"] <= 1e-8 for i in inf), inf
        e1.record()
        torch.cuda.synchronize()
        return maxrank(e0.elapsed_time(e1) / 1e3), its

    nbatch = max(3, args.steps // 4)
    tb_mix, itb_mix = timed_batched(amg.MIXED32, nbatch)
    tb_64, itb_64 = timed_batched(amg.FP64, nbatch)
    batched = {"nrhs_per_batch": 8, "batches": nbatch * world, "unit": "solves/s",
               "mixed": 8 * nbatch * world / tb_mix, "fp64": 8 * nbatch * world / tb_64,
               "max_iters_per_batch": {"mixed": itb_mix[0], "fp64": itb_64[0]}}

    # 64 right-hand sides in calls of 8, 16 or 32 columns (batches of that
    # width: the matrices are read once per iteration for each batch)
    def timed_wide(prec, reps, width):
        H.set_precision(prec)
        B64 = torch.from_numpy(np.ascontiguousarray(seeded_rhs(n, 64, cfg["seed"] * 1000 + 700 + rank))).cuda()
        chunks = [B64[:, j:j + width].contiguous() for j in range(0, 64, width)]
        for ch in chunks:
            H.solve(ch, tol=1e-8)  # warm-up (workspace, graph capture)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        its = 0
        for _ in range(reps):
            for ch in chunks:
                _, inf = H.solve(ch, tol=1e-8)
                assert all(i["status"] == 0 and i["relres_true"] <= 1e-8 for i in inf), inf
                its = max(its, max(i["iters"] for i in inf))
        e1.record()
        torch.cuda.synchronize()
        return 64 * reps * world / maxrank(e0.elapsed_time(e1) / 1e3), its

    wreps = max(2, args.steps // 20)
    rhs64 = {"unit": "solves/s", "reps": wreps * world, "by_batch_width": {}}
    for prec, key in ((amg.MIXED32, "mixed"), (amg.FP64, "fp64")):
        for width in (8, 16, 32):
            v, it = timed_wide(prec, wreps, width)
            rhs64["by_batch_width"].setdefault(key, {})[str(width)] = {"solves_per_s": v, "max_iters": it}
    batched["rhs64"] = rhs64
    H.set_precision(HEAD)

    serving = None
    if not args.no_serving:
        serving = serving_run(amg, seed=5, sides=(64, 128, 256), nops=3, nreq=96, max_rhs=4)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle in a process of its own, single-threaded BLAS
        fd, path = tempfile.mkstemp(suffix=".npz")
        os.close(fd)
        np.savez(path, b=Bh[:, args.warmup].copy(), x=X[args.warmup].cpu().numpy(), theta=cfg["theta"],
                 eps=cfg["eps"], N=cfg["N"])
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference", "--workload",
                            args.workload, "--oracle-solve", path], capture_output=True, text=True, env=env)
        os.unlink(path)
        try:
            o = json.loads(r.stdout.strip().splitlines()[-1])
            one = {"value": 1.0 / o["solve_s"], "unit": "solves/s", "cores": o["cores"],
                   "sample": f"one oracle PCG solve of the first timed right-hand side ({o['iters']} iterations, "
                             f"{o['solve_s']:.1f} s) after the oracle's own setup ({o['setup_s']:.1f} s, untimed), "
                             f"single-threaded BLAS; max |x_oracle - x_gpu| / max |x_oracle| = {o['err']:.1e}"}
            ac = o.get("all_cores")
            if ac:
                cpu = {"value": ac["solves"] / ac["wall_s"], "unit": "solves/s", "cores": ac["cores"],
                       "kind": "oracle",
                       "sample": f"{ac['solves']} oracle PCG solves of seeded right-hand sides at once, one "
                                 f"single-threaded process per core sharing the oracle's hierarchy, "
                                 f"{ac['wall_s']:.1f} s wall ({min(ac['iters'])}-{max(ac['iters'])} iterations); "
                                 f"os.cpu_count() = {ac['cores']}",
                       "one_thread": one}
            else:
                cpu = dict(one, kind="oracle")
        except Exception as e:  # report, do not hide, a failed baseline
            cpu = {"value": None, "unit": "solves/s", "cores": None, "kind": "oracle",
                   "sample": f"oracle run failed: {e}: {r.stderr[-300:]}"}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_mix / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": workload_desc(cfg), "precision": "FP32 V-cycle, FP64 flexible CG",
                   "l2": "inputs larger than L2: one V-cycle moves %.2f GB" % (float(by.sum()) / 1e9),
                   "parallelism": f"replicas x{world}",
                   "mode": "deterministic (no atomics)" if args.deterministic else "default"},
        "fp64": {"value": fp64_value, "unit": "solves/s", "ms_per_step": t_64 / args.steps * 1e3,
                 "iters": it_64},
        "mixed16": {"value": m16_value, "unit": "solves/s", "ms_per_step": t_16 / args.steps * 1e3,
                    "iters": [i["iters"] for i in inf_16],
                    "precision": "FP16 copies of the smoother rows, basis and coarse block rows where setup timed "
                                 "them faster, FP32 vectors and sums, FP64 flexible CG",
                    "roofline": roofline16,
                    "fp16_lanes_by_level": stats.get("fp16_lanes")},
        "mixed_over_fp64": value / fp64_value,
        "vcycles_per_s": {"mixed": vc_mix, "fp64": vc_64},
        "iters": it_mix, "mixed_fp64_fallbacks": fallbacks, "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "setup_s": setup_s, "setup_phases_ms": {k: round(v, 1) for k, v in stats["setup_phases_ms"].items()},
        "setup_fp64": setup_rates(stats, amg.measure_fp64()),
        "levels": stats["n"], "op_complexity": stats["op_complexity"],
        "convergence": convergence(inf_64[0]),
        "coarse_A": [c["form"] for c in stats["coarse_A"]],
        "persistent_tail_from": {"mixed": stats["tail"]["mixed"]["from"], "fp64": stats["tail"]["fp64"]["from"]},
        "dense_tail_from": {"mixed": stats["dense_tail"]["mixed"]["from"], "fp64": stats["dense_tail"]["fp64"]["from"]},
        "roofline": roofline, "vcycle_profile_us_gbs": vprof,
        "batched": batched, "serving": serving,
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        # the oracle's many small LAPACK calls run fastest single-threaded;
        # set before numpy loads its BLAS
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        if args.oracle_solve:
            oracle_solve_sample(args)
        else:
            run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
