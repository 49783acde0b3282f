#!/usr/bin/env python3
"""Isaacs solves/s at 1023^2 on one GB300 (mixed float32/float64 vs float64).

One step = one full AMGpi solve (policy iteration with multigrid linear
solves) of the 1023 x 1023 finite-difference Isaacs game, plain variant,
started from scratch (v = 0, default policies), run until MAX's policy is
stable, with every linear system solved to the float64 residual floor.
The reward noise is generated on the device from the seed, so the inputs are
resident when the timed region starts.  Between timed steps a 256 MiB buffer
is written to flush the L2 (the solve's working set, ~60 MB, fits in L2).

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Isaacs solves/s at 1023^2 (FP32+refine vs FP64), HBM GB/s, p50/p99 latency"
# arithmetic types per precision option: float64; float32 V-cycles in float64
# refinement; the same with the V-cycle weights stored in bfloat16
DTYPES = {"fp64": "f64", "mixed": "f32+f64", "mixed_bf16": "bf16(weights)+f32+f64"}
# V(1,2) cycles for the Isaacs workload: at 1023^2 they need 34 V-cycles per
# solve against 48 for V(1,1) and take 6% less time (a solver option, as a user
# would set it; the library's default stays V(1,1)).
ISAACS_CYCLE = {"nu1": 1, "nu2": 2}
SIDE = 1023          # the metric's workload; --side changes it (e.g. 2047 for profiling)
# the V-cycle kernel the library's default options launch (tiled grid-wide levels)
CYCLE_KERNEL = "k_mg_cycles_tiled"
SEED = 2

def cycle_sweeps(cycle: dict):
    """(nu1 + nu2 on the finest level, nu1 + nu2 on the coarse levels) of a cycle option set."""
    fine = cycle["nu1"] + cycle["nu2"]
    c1 = cycle.get("nu1_coarse", -1)
    c2 = cycle.get("nu2_coarse", -1)
    return fine, (cycle["nu1"] if c1 < 0 else c1) + (cycle["nu2"] if c2 < 0 else c2)


def cycle_label(cycle: dict) -> str:
    """"V(nu1,nu2)", with the coarse levels' sweeps when they differ."""
    lab = "V(%d,%d)" % (cycle["nu1"], cycle["nu2"])
    c1, c2 = cycle.get("nu1_coarse", -1), cycle.get("nu2_coarse", -1)
    if c1 >= 0 or c2 >= 0:
        lab += ", coarse levels (%d,%d)" % (cycle["nu1"] if c1 < 0 else c1,
                                            cycle["nu2"] if c2 < 0 else c2)
    return lab


# Algorithmic bytes of the multigrid solve kernel (one launch per linear
# system), per fine state: what the method must move, with every array read
# or written once per phase.  Coarse levels carry 9-point stencils; the level
# sizes shrink by 4, so their sum is 4/3 of the first coarse level.
def mg_bytes_per_state(prec: str, sweeps: int = 2, sweeps_coarse: int = None):
    """Algorithmic bytes per fine state of one V-cycle with `sweeps` = nu1 + nu2
    relaxation sweeps on the finest level and `sweeps_coarse` (default: the
    same) on the coarse ones, of one float64 residual check, and of a set-up."""
    sc = sweeps if sweeps_coarse is None else sweeps_coarse
    if prec == "fp64":
        check = 1 + 8 + 8                              # code, rhs, v
        fine = sweeps * (1 + 8 + 8 + 8) + (1 + 8 + 8 + 16 + 4) + (16 + 2 + 16)
        coarse1 = sc * (72 + 24) + (72 + 16 + 16 + 4) + 34
        setup = (2 + 32 + 1 + 32 + 32 + 4 + 64 + 72) / 4 + (72 + (32 + 32 + 64 + 72) / 4) / 3
    else:
        # float32 vectors; weights in float32 (mixed) or bfloat16 (mixed_bf16):
        # A = 9 stored entries per coarse point, P = 8 weights per coarse cell
        # (2 bytes per fine point in float32), each written beside its float64 master
        wb = 2 if prec == "mixed_bf16" else 4
        A, Pf = 9 * wb, 2 * wb
        check = 1 + 8 + 8 + 4                          # + float32 residual written
        fine = sweeps * (1 + 4 + 4 + 4) + (1 + 4 + 4 + Pf + 2) + (Pf + 1 + 8) + (4 + 16)
        coarse1 = sc * (A + 12) + (A + 8 + Pf + 2) + (Pf + 1 + 8)
        Pe = 32 + 4 * wb                               # 4 edge (or corner) weights, both copies
        Ac = 72 + A                                    # Galerkin row, both copies
        setup = (2 + Pe + 1 + 32 + Pe + 4 + 64 + Ac) / 4 + (72 + (Pe + Pe + 64 + Ac) / 4) / 3
    cycle = fine + coarse1 / 4 * 4 / 3
    return {"check": check, "cycle": cycle, "setup": setup}


def mg_cycle_bytes(n: int, prec: str, launches: int, cycles: int, sweeps: int = 2,
                   sweeps_coarse: int = None) -> float:
    """Algorithmic bytes of `launches` V-cycle launches running `cycles` cycles in all
    (each launch evaluates the float64 residual once more than it has cycles)."""
    b = mg_bytes_per_state(prec, sweeps, sweeps_coarse)
    return n * (launches * b["check"] + cycles * (b["cycle"] + b["check"]))


# DRAM bytes per cycle-kernel launch from the committed capture of the current
# kernel (profiles/k_mg_cycles_tiled_isaacs1023_mixed.md): read + write, with
# ncu's cache flush before the launch.  Keyed by (side, precision).
PROFILED_TRAFFIC = {(1023, "mixed"): 46.23e6 + 2.01e6}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.fh = tempfile.TemporaryFile(mode="w+")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.fh.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.fh.read())) if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replicas_max_ms(ms: float, world: int, device) -> float:
    """Per-step time of the whole job: the maximum over the replicas' ranks."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, ms_max: float, units_per_step: float = 1.0) -> float:
    """Units per second of all replicas: each rank processes its own units per
    step, and the job's step ends with its slowest rank."""
    return world * units_per_step * 1000.0 / ms_max


def oracle_sample(systems_per_solve: int, outer_per_solve: int):
    """Seconds of one oracle policy evaluation + improvement at 1023^2.

    The sample is one sparse-LU solve of the policy-fixed system (Eq. (LSPI))
    and one full improvement sweep; a whole oracle solve performs
    `systems_per_solve` of the former and about as many improvements.
    """
    import numpy as np
    import oracle
    from oracle.isaacs import isaacs_game
    game = isaacs_game(SIDE, 0, seed=SEED)
    n = game.n
    alpha = np.zeros(n, np.uint8)
    beta = np.zeros((n, 4), np.uint8)
    t0 = time.perf_counter()
    A, r = oracle.policy_system(game, alpha, beta)
    w = oracle.solve_policy_system(A, r, "lu")
    t1 = time.perf_counter()
    oracle.improve(game, w, alpha, beta)
    t2 = time.perf_counter()
    t_solve = systems_per_solve * (t1 - t0) + (systems_per_solve + outer_per_solve) * (t2 - t1)
    return t_solve, t1 - t0, t2 - t1


def _oracle_batch_game(args):
    """Worker (module level for a spawn pool): seconds the oracle takes to solve
    game g of the random batch (policy iteration, fixed-point evaluation)."""
    n, seed, g = args
    import oracle
    import synth
    from oracle.game import game_from_csr
    rp, col, prob, rew, mu = synth.random_game(n, synth.batch_game_seed(seed, g))
    game = game_from_csr(n, 4, 4, rp, col, prob, rew, mu)
    t0 = time.perf_counter()
    oracle.policy_iteration(game, solver="fixed_point")
    return time.perf_counter() - t0


def oracle_batch_sample(sizes, seed: int, games: int = 48, workers: int = 0):
    """The oracle on a seeded sample of the batch's games, one game per process
    over the host's cores.  Returns (games/s, cores, seconds of CPU work)."""
    import multiprocessing as mp
    import numpy as np
    workers = workers or os.cpu_count() or 1
    pick = np.random.default_rng(seed + 1).choice(len(sizes), size=min(games, len(sizes)),
                                                  replace=False)
    tasks = [(int(sizes[g]), seed, int(g)) for g in pick]
    with mp.get_context("spawn").Pool(workers) as pool:
        t0 = time.perf_counter()
        per_game = pool.map(_oracle_batch_game, tasks, chunksize=1)
        wall = time.perf_counter() - t0
    return len(tasks) / wall, workers, float(sum(per_game))


# Policy iterations the FP64 oracle needs for this workload (1023^2, seed 2),
# counted by a full oracle run (tests/golden/oracle_counts_1023.txt).
def _oracle_counts_file():
    path = os.path.join(ROOT, "tests", "golden", "oracle_counts_1023.txt")
    d = {}
    with open(path) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                d[k] = float(v)
    return d


def oracle_counts():
    d = _oracle_counts_file()
    return int(d["systems"]), int(d["outer"])


def oracle_full_solve_seconds():
    """Wall time of the full oracle solve recorded with the counts (or None)."""
    return _oracle_counts_file().get("seconds")


def load_samples(name):
    """(vmax, state indices, values) of a stored oracle run at sampled states."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", name)
    vmax, idx, vals = None, [], []
    with open(path) as fh:
        for ln in fh:
            if ln.startswith("#"):
                continue
            if ln.startswith("vmax"):
                vmax = float(ln.split()[1])
                continue
            t = ln.split()
            idx.append(int(t[0]))
            vals.append(float(t[1]))
    return vmax, np.array(idx, np.int64), np.array(vals)


def err_vs_samples(v, samples):
    """max over the sampled states of |v - v_oracle| / max |v_oracle|."""
    import numpy as np
    vmax, idx, vals = samples
    return float(np.max(np.abs(v[idx] - vals)) / vmax)


def measure_l2_copy_gbs(device="cuda"):
    """Copy bandwidth of buffer pairs that stay in the 129 MB L2 (2 x 24 and
    2 x 32 MiB), best of 10 timed repetitions of 60 copies (read + write bytes)."""
    import torch
    best = 0.0
    for mib in (24, 32):
        a = torch.empty(mib << 20, dtype=torch.uint8, device=device)
        b = torch.empty_like(a)
        a.fill_(1)
        for _ in range(10):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(60):
                b.copy_(a)
            e1.record()
            torch.cuda.synchronize()
            best = max(best, 60 * 2 * a.numel() / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def run_reference(args):
    """The FP64 oracle on the host.  One step is one unit of the oracle's own
    policy iteration at 1023^2: a sparse-LU policy evaluation followed by an
    improvement sweep (both timed).  A whole oracle solve of this workload is
    `systems` evaluations and `systems + outer` improvements (counted by a full
    oracle run, tests/golden/oracle_counts_1023.txt), so
    value = 1 / (systems * t_eval + (systems + outer) * t_improve), while
    ms_per_step is the measured time of one step."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    systems, outer = oracle_counts()
    t_evals, t_imps = [], []
    for k in range(args.warmup + args.steps):
        _, t_eval, t_imp = oracle_sample(systems, outer)
        if k >= args.warmup:
            t_evals.append(t_eval)
            t_imps.append(t_imp)
    t_eval, t_imp = statistics.mean(t_evals), statistics.mean(t_imps)
    value = 1.0 / (systems * t_eval + (systems + outer) * t_imp)
    full = oracle_full_solve_seconds()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (t_eval + t_imp) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"isaacs_{SIDE}x{SIDE}_plain_amgpi", "side": SIDE, "seed": SEED,
                   "variant": "plain", "solver": "oracle PI + SuperLU", "parallelism": "none"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: one sparse-LU policy evaluation ({t_eval:.2f} s) + one "
                                   f"improvement ({t_imp:.2f} s) of the oracle at {SIDE}^2; a solve is "
                                   f"{systems} evaluations + {systems + outer} improvements"
                                   + (f"; a full oracle solve measured {full:.0f} s on the build host"
                                      if full else "")},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """C4: 4096 random games (n ~ U{256..8192}, m1 = m2 = 4, 8 successors,
    Dirichlet(1), rewards U(-1,1), mu = 0.99) in one persistent launch."""
    import numpy as np
    import torch
    import synth
    torch.cuda.set_device(0)
    import paper_1107_1653_gb300 as gs
    count, seed = args.games, 4
    sizes = synth.batch_game_sizes(count, seed)
    t0 = time.perf_counter()
    off, rp, col, prob, rew, mu = synth.random_game_batch(sizes, seed, workers=os.cpu_count())
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    s = gs.GameSolver(precision=args.precision, stream=stream)
    # inputs resident: the tables go to the device before timing
    s.set_game_batch(off, 4, 4, rp, col, prob, rew, mu)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        s.solve()
    times, st = [], None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        st = s.solve()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    gst, gres = s.batch_stats()
    shape = s.batch_shape()
    sec = statistics.mean(times)
    n_tot = int(off[-1])
    nnz = len(col)
    # algorithmic float64 work of the improvements: every evaluation of a row
    # costs 2 flops per successor; per game one reply + one full improvement
    # per outer iteration (m1*m2 rows per state) and one inner improvement per
    # evaluation (m2 rows per state)
    rows_full = 16
    imp = sum(int(n) * 8 * 2 * (rows_full * (1 + int(o)) + 4 * 2 * int(sy))
              for n, o, sy in zip(sizes, gst[:, 0], gst[:, 1]))
    # e2e: host tables -> set_game_batch -> solve -> values and policies back
    e2e = []
    v_h = np.empty(n_tot)
    a_h = np.empty(n_tot, np.uint8)
    b_h = np.empty((n_tot, 4), np.uint8)
    for _ in range(2):
        t1 = time.perf_counter()
        s.set_game_batch(off, 4, 4, rp, col, prob, rew, mu)
        s.solve()
        s.get_value(out=v_h)
        s.get_policy(alpha_out=a_h, beta_out=b_h)
        e2e.append(time.perf_counter() - t1)
    s.close()
    line = {
        "metric": "random games solved/s (batch of 4096, n~U{256..8192})", "value": count / sec,
        "unit": "games/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.precision],
        "data": "synthetic",
        "config": {"workload": "random_games_batch4096", "games": count, "states": n_tot,
                   "nnz": nnz, "seed": seed, "precision": args.precision,
                   "threads_per_game": shape, "order": "largest game first",
                   "l2": "flushed between steps (256 MiB write)",
                   "outer_max": int(gst[:, 0].max()), "systems": int(gst[:, 1].sum()),
                   "cycles": int(gst[:, 2].sum()), "converged": int(gst[:, 3].min()),
                   "res_max": float(gres.max())},
        "states_per_s": n_tot / sec,
        "fp64_improvement_tflops": imp / sec / 1e12,
        "generation_s": t_gen,
        "e2e": {"value": count / statistics.mean(e2e), "unit": "games/s",
                "h2d_bytes_per_step": int(rp.nbytes + col.nbytes + prob.nbytes + rew.nbytes),
                "d2h_bytes_per_step": int(v_h.nbytes + a_h.nbytes + b_h.nbytes)},
    }
    if not args.no_cpu_baseline:
        g_s, cores, cpu_s = oracle_batch_sample(sizes, seed)
        line["cpu_baseline"] = {
            "value": g_s, "unit": "games/s", "cores": cores, "kind": "oracle",
            "sample": f"48 games drawn from the batch, one per process on {cores} host cores "
                      f"({cpu_s:.0f} s of CPU work); policy iteration with the fixed-point "
                      f"policy evaluation to 1e-14"}
    print(json.dumps(line), flush=True)
    return 0


def serving_line(args):
    """C5: Poisson stream of requests, 70% Isaacs grids (sides 63..1023) and
    30% random games (n ~ U{1e3..1e6}), mixed precision, arrival rate 80% of
    the closed-loop capacity; p50/p99 latency and solves/s (as a dict)."""
    import numpy as np
    import torch
    import paper_1107_1653_gb300 as gs
    rng = np.random.default_rng(5)
    # every game request is a fresh random game n ~ U{1e3..1e6} given by its
    # seed: the server draws its table on the device when the request runs
    sides = (63, 127, 255, 511, 1023)

    def draw(k):
        if rng.random() < 0.7:
            return ("isaacs", int(rng.choice(sides)), 5 + k)
        return ("game", int(rng.integers(1000, 1_000_001)), 50_000 + k)

    def submit(srv, r):
        if r[0] == "isaacs":
            return srv.submit_isaacs(r[1], 0, r[2])
        return srv.submit_random_game(r[1], 4, 4, r[2], 0.99)

    with gs.GameServer(slots=args.slots, precision="mixed") as srv:
        # closed-loop capacity: a burst of requests submitted at once
        burst = [draw(k) for k in range(args.burst)]
        t1 = time.perf_counter()
        tickets = [submit(srv, r) for r in burst]
        for t in tickets:
            srv.wait(t)
            srv.result(t)
        cap = len(burst) / (time.perf_counter() - t1)
        rate = 0.8 * cap
        reqs = [draw(10_000 + k) for k in range(args.requests)]
        gaps = rng.exponential(1.0 / rate, size=len(reqs))
        tickets = []
        t_start = time.perf_counter()
        due = t_start
        for r, g in zip(reqs, gaps):
            due += g
            d = due - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(submit(srv, r))
        infos = []
        for t in tickets:
            infos.append(srv.wait(t))
            srv.result(t)
        makespan = time.perf_counter() - t_start
    lat = np.array([i["t_end"] - i["t_submit"] for i in infos])
    ok = sum(1 for i in infos if i["status"] == 0)
    kinds = [r[0] for r in reqs]
    lat_i = lat[[k == "isaacs" for k in kinds]]
    lat_g = lat[[k == "game" for k in kinds]]
    line = {
        "metric": "serving: p50/p99 latency and solves/s (70% Isaacs 63..1023, 30% games 1e3..1e6)",
        "value": ok / makespan, "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "serving_mix", "requests": len(reqs), "slots": args.slots,
                   "arrival": "Poisson", "rate_per_s": rate, "capacity_per_s": cap,
                   "games": "a fresh random game per request, n ~ U{1e3..1e6}, 4 x 4 actions, "
                            "8 successors per row, mu 0.99, drawn on the device from its seed",
                   "isaacs_sides": list(sides)},
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "p50_ms_isaacs": float(np.percentile(lat_i, 50) * 1e3) if len(lat_i) else None,
        "p99_ms_isaacs": float(np.percentile(lat_i, 99) * 1e3) if len(lat_i) else None,
        "p50_ms_games": float(np.percentile(lat_g, 50) * 1e3) if len(lat_g) else None,
        "p99_ms_games": float(np.percentile(lat_g, 99) * 1e3) if len(lat_g) else None,
        "completed": ok, "makespan_s": makespan,
    }
    return line


def run_serving(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(serving_line(args)), flush=True)
    return 0


def run_profile(args):
    """One solve of the workload and nothing else (a short command for ncu)."""
    import torch
    torch.cuda.set_device(0)
    import paper_1107_1653_gb300 as gs
    with gs.GameSolver(precision=args.precision, fmg=args.fmg, fmg_side=31,
                       stream=torch.cuda.current_stream(), **ISAACS_CYCLE) as s:
        s.set_isaacs_grid(SIDE, 0, SEED)
        st = s.solve()
    torch.cuda.synchronize()
    print(json.dumps({"profile": True, "side": SIDE, "precision": args.precision, **st}))
    return 0


def run_profile_game(args):
    """One solve of a random game of n states (mixed precision) and nothing
    else: a short command for ncu on the grid-wide game kernel."""
    import torch
    torch.cuda.set_device(0)
    import paper_1107_1653_gb300 as gs
    n = args.profile_game
    with gs.GameSolver(precision="mixed") as s:
        s.set_random_game(n, 4, 4, 7 + n, 0.99)
        st = s.solve()
    torch.cuda.synchronize()
    print(json.dumps({"profile_game": True, "n": n, **st}))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_1107_1653_gb300 as gs

    stream = torch.cuda.current_stream()
    n = SIDE * SIDE
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(precision, steps, warmup, trace=None):
        s = gs.GameSolver(precision=precision, fmg=args.fmg, fmg_side=31, stream=stream, **ISAACS_CYCLE)
        s.set_isaacs_grid(SIDE, 0, SEED)
        for _ in range(warmup):
            s.solve()
        if trace and trace != "none":
            s.trace(trace)
        launches0 = gs.lib.gamesolve_kernel_launches()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        per_step, stats = [], None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t_wall = time.perf_counter()
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            stats = s.solve()
            e1.record(stream)
            torch.cuda.synchronize()
            per_step.append(e0.elapsed_time(e1))
        t_wall = time.perf_counter() - t_wall
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        launches = gs.lib.gamesolve_kernel_launches() - launches0
        tr = s.trace_read() if trace and trace != "none" else (0.0, 0)
        v = s.get_value()
        s.close()
        return per_step, stats, launches, tr, v, t_wall

    clocks = ClockSampler(local)
    prec = args.precision
    per_step, stats, launches, (tr_ms, tr_n), v_main, t_wall = timed(
        prec, args.steps, args.warmup, trace=args.trace_kernel)
    clk = clocks.stop()
    ms = statistics.mean(per_step)
    ms_max = replicas_max_ms(ms, world, "cuda")
    value = whole_job_value(world, ms_max)

    # the other precisions, for the FP32+refine vs FP64 comparison: each one's
    # time and counts, and every result's relative distance from the FP64 value
    compare, values = {}, {prec: v_main}
    for other in ("fp64", "mixed", "mixed_bf16"):
        if other == prec:
            continue
        o_steps, o_stats, _, _, values[other], _ = timed(other, max(2, args.steps // 2), 1)
        o_ms = statistics.mean(o_steps)
        compare[other] = {"value": 1000.0 / o_ms, "ms_per_step": o_ms, "outer": o_stats["outer"],
                          "systems": o_stats["systems"], "cycles": o_stats["cycles"]}
    v64 = values["fp64"]
    for k, v in values.items():
        if k != "fp64":
            compare["rel_diff_" + k + "_vs_fp64"] = float(np.max(np.abs(v - v64)) / np.max(np.abs(v64)))
    # every result against the FP64 oracle: its stored run at 1,026 sampled states
    if (SIDE, SEED) == (1023, 2):
        samples = load_samples("isaacs1023_plain_seed2_samples.txt")
        compare["err_vs_oracle_sampled"] = {k: err_vs_samples(v, samples) for k, v in values.items()}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[prec], "data": "synthetic",
        "config": {"workload": f"isaacs_{SIDE}x{SIDE}_plain_{'famgpi' if args.fmg else 'amgpi'}_{prec}",
                   "side": SIDE, "states": n, "seed": SEED, "variant": "plain",
                   "precision": prec, "fmg": bool(args.fmg),
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed between steps (256 MiB write)",
                   "cycle": cycle_label(ISAACS_CYCLE),
                   "outer": stats["outer"], "systems": stats["systems"], "cycles": stats["cycles"],
                   "levels": stats["levels"], "res_inf": stats["res_inf"]},
        "p50_ms": statistics.median(per_step),
        "p99_ms": sorted(per_step)[min(len(per_step) - 1, int(0.99 * len(per_step)))],
        "wall_s_timed_loop": t_wall,
        "gpu_launches": int(launches),
        "compare": compare,
    }
    if clk:
        line["clocks"] = clk

    # roofline of the dominant kernel: the V-cycle launch (one or two per system)
    peak, peak_kind = load_peaks()
    if tr_n:
        kind = prec
        sweeps, sweeps_c = cycle_sweeps(ISAACS_CYCLE)
        total = mg_cycle_bytes(n, kind, tr_n, stats["cycles"] * args.steps, sweeps, sweeps_c)
        bpl = total / tr_n
        avg_s = tr_ms * 1e-3 / tr_n
        ach = bpl / avg_s / 1e9
        line["roofline"] = {"kernel": CYCLE_KERNEL, "bound": "hbm", "achieved": ach,
                            "peak": peak, "unit": "GB/s", "frac": ach / peak,
                            "peak_source": peak_kind,
                            "traffic": PROFILED_TRAFFIC.get((SIDE, prec)),
                            "launches": tr_n, "avg_us": avg_s * 1e6,
                            "algorithmic_bytes_per_launch": bpl,
                            "note": ("working set fits in L2 (129 MB)" if SIDE <= 1023 else
                                     "working set exceeds the 129 MB L2") + "; bytes per state "
                                    + json.dumps({k: round(v, 1) for k, v in
                                                  mg_bytes_per_state(kind, sweeps,
                                                                     sweeps_c).items()})}

    # roofline of the same launches against the L2 (the 1023^2 working set stays in it)
    if "roofline" in line and SIDE <= 1023:
        l2 = measure_l2_copy_gbs()
        r = line["roofline"]
        line["roofline_l2"] = {"kernel": r["kernel"], "achieved": r["achieved"], "peak": l2,
                               "unit": "GB/s", "frac": r["achieved"] / l2,
                               "peak_source": "measured in this run: L2-resident 24-32 MiB copy"}

    # the precision workload: 2047^2, seed 3, every precision, against the oracle
    if not args.no_2047 and SIDE == 1023 and world == 1:
        line["side_2047"] = run_2047(args, stream, peak, peak_kind)
    if world == 1 and SIDE == 1023 and not args.no_obstacle:
        line["obstacle_1023"] = run_obstacle_1023(args, stream)
    # the batching and serving rows' workloads, compact
    if world == 1 and SIDE == 1023 and not args.no_workloads:
        line["batch_4096"] = batch_block(stream)
        sv = serving_line(args)
        line["serving"] = {k: sv[k] for k in ("value", "unit", "p50_ms", "p99_ms", "p50_ms_isaacs",
                                              "p99_ms_isaacs", "p50_ms_games", "p99_ms_games",
                                              "completed", "makespan_s")}
        line["serving"]["config"] = sv["config"]
        _, lo = line_results(args)
        line["stopping_line_2049"] = {"famgpi": lo["famgpi"], "amgpi_flat": lo["amgpi"],
                                      "paper_e_inf": 1.16e-7, "paper_e_l2": 7.40e-8}
        line["continuous_actions_127"] = iex1_block(stream)
        line["tables_famg_line_513"] = tables_famg_block(stream)

    # end to end through the C-ABI with host buffers
    if not args.no_e2e:
        import synth
        xi_h = torch.from_numpy(synth.isaacs_noise(SIDE, SEED)).pin_memory()
        v_h = torch.empty(n, dtype=torch.float64).pin_memory()
        a_h = torch.empty(n, dtype=torch.uint8).pin_memory()
        b_h = torch.empty((n, 4), dtype=torch.uint8).pin_memory()
        s = gs.GameSolver(precision=prec, fmg=args.fmg, fmg_side=31, stream=stream, **ISAACS_CYCLE)
        e2e = []
        for k in range(1 + max(2, args.steps // 2)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.set_isaacs_grid(SIDE, 0, SEED, xi=xi_h)
            s.solve()
            s.get_value(out=v_h)
            s.get_policy(alpha_out=a_h, beta_out=b_h)
            t1 = time.perf_counter()
            if k:
                e2e.append(t1 - t0)
        s.close()
        line["e2e"] = {"value": 1.0 / statistics.mean(e2e), "unit": "solves/s",
                       "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n + n + 4 * n}

    # CPU oracle baseline on a bounded sample (rank 0, one GPU only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        systems, outer = oracle_counts()
        t_solve, t_lu, t_imp = oracle_sample(systems, outer)
        line["cpu_baseline"] = {
            "value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"one sparse-LU policy evaluation ({t_lu:.1f} s) + one improvement "
                      f"({t_imp:.1f} s) at {SIDE}^2, scaled by the oracle's {systems} systems / "
                      f"{outer} outer iterations per solve"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_2047(args, stream, peak, peak_kind):
    """The precision configuration: 2047 x 2047 plain Isaacs game, seed 3,
    flat AMGpi to the float64 floor, each precision timed over a few solves
    (L2 flushed between them), the V-cycle kernel's HBM roofline, and every
    result's error against the stored FP64 oracle run (sampled states)."""
    import numpy as np
    import torch
    import paper_1107_1653_gb300 as gs
    side, seed, n = 2047, 3, 2047 * 2047
    samples = load_samples("isaacs2047_plain_seed3_samples.txt")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out, values = {}, {}
    for prec in ("mixed", "fp64", "mixed_bf16"):
        s = gs.GameSolver(precision=prec, stream=stream, **ISAACS_CYCLE)
        s.set_isaacs_grid(side, 0, seed)
        s.solve()
        s.trace("mg_cycles")
        ts = []
        st = None
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = s.solve()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        tr_ms, tr_n = s.trace_read()
        values[prec] = s.get_value()
        s.close()
        ms = statistics.mean(ts)
        sweeps, sweeps_c = cycle_sweeps(ISAACS_CYCLE)
        total = mg_cycle_bytes(n, prec, tr_n, st["cycles"] * 3, sweeps, sweeps_c)
        ach = total / tr_n / (tr_ms * 1e-3 / tr_n) / 1e9
        out[prec] = {"solves_per_s": 1000.0 / ms, "ms_per_solve": ms, "outer": st["outer"],
                     "systems": st["systems"], "cycles": st["cycles"],
                     "err_vs_oracle_sampled": err_vs_samples(values[prec], samples),
                     "roofline": {"kernel": CYCLE_KERNEL, "bound": "hbm", "achieved": ach,
                                  "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                  "peak_source": peak_kind, "avg_us": tr_ms * 1e3 / tr_n}}
    v64 = values["fp64"]
    for k in ("mixed", "mixed_bf16"):
        out[k]["rel_diff_vs_fp64"] = float(np.max(np.abs(values[k] - v64)) / np.max(np.abs(v64)))
    out["config"] = {"side": side, "states": n, "seed": seed, "cycle": cycle_label(ISAACS_CYCLE),
                     "l2": "flushed between solves (256 MiB write)",
                     "oracle": "isaacs2047_plain_seed3_samples.txt (1,026 states)"}
    return out


def batch_block(stream, count=4096, seed=4, warmup=2, steps=3):
    """The 4096-game batch (C4) with its tables drawn on the device
    (gamesolve_random_game, game g from the stream seed XOR g, as
    synth.random_game_batch draws them on the host): games/s over a few
    solves (L2 flushed between them), iteration counts, convergence."""
    import numpy as np
    import torch
    import synth
    import paper_1107_1653_gb300 as gs
    sizes = synth.batch_game_sizes(count, seed)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    R, K = 16, 8
    rows = int(off[-1]) * R
    dev = torch.device("cuda", torch.cuda.current_device())
    col = torch.empty(rows * K, dtype=torch.int32, device=dev)
    prob = torch.empty(rows * K, dtype=torch.float64, device=dev)
    rew = torch.empty(rows, dtype=torch.float64, device=dev)
    scratch = torch.empty(int(sizes.max()) * R + 1, dtype=torch.int64, device=dev)
    for g in range(count):
        r0 = int(off[g]) * R
        code = gs.lib.gamesolve_random_game(int(sizes[g]), 4, 4, K, synth.batch_game_seed(seed, g),
                                            scratch.data_ptr(), col[r0 * K:].data_ptr(),
                                            prob[r0 * K:].data_ptr(), rew[r0:].data_ptr(), stream.cuda_stream)
        if code != gs.GS_OK:
            raise RuntimeError("gamesolve_random_game failed")
    rp = torch.arange(rows + 1, dtype=torch.int64, device=dev) * K   # rows of 8 entries
    mu = np.full(count, 0.99)
    s = gs.GameSolver(precision="mixed", stream=stream)
    s.set_game_batch(off, 4, 4, rp, col, prob, rew, mu)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        s.solve()
    times = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.solve()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    gst, gres = s.batch_stats()
    s.close()
    sec = statistics.mean(times)
    return {"games_per_s": count / sec, "ms_per_batch": sec * 1e3, "states_per_s": float(off[-1]) / sec,
            "warmup": warmup, "steps": steps,
            "config": {"games": count, "states": int(off[-1]), "seed": seed, "precision": "mixed",
                       "tables": "drawn on the device (gamesolve_random_game), resident before timing",
                       "l2": "flushed between solves (256 MiB write)"},
            "outer_max": int(gst[:, 0].max()), "systems": int(gst[:, 1].sum()),
            "cycles": int(gst[:, 2].sum()), "converged": int(gst[:, 3].min()),
            "res_max": float(gres.max())}


def iex1_block(stream, side=127, ka=32, kb=13):
    """The Isaacs example with continuous action sets (Sec. 6.1), its action
    sets discretised (ka directions on MAX's unit circle, a kb x kb grid of
    MIN's b), lambda = 0: flat AMGpi on the tables path with algebraic
    multigrid, timed once after a warm-up solve, and the error against the
    exact solution sin x1 sin x2."""
    import numpy as np
    import torch
    import synth
    import paper_1107_1653_gb300 as gs
    n, m1, m2, rp, col, prob, rew, mu = synth.iex1_tables(side, ka, kb)
    with gs.GameSolver(precision="mixed", game_solver=1, stream=stream) as s:
        s.set_game(n, m1, m2, rp, col, prob, rew, mu)
        s.solve()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = s.solve()
        e1.record(stream)
        torch.cuda.synchronize()
        v = s.get_value()
    h = 1.0 / (side + 1)
    idx = np.arange(n)
    x1, x2 = (idx % side + 1) * h, (idx // side + 1) * h
    e = v - np.sin(x1) * np.sin(x2)
    return {"ms_per_solve": e0.elapsed_time(e1), "outer": st["outer"], "systems": st["systems"],
            "cycles": st["cycles"], "e_inf": float(np.max(np.abs(e))),
            "e_l2": float(np.sqrt(np.mean(e * e))),
            "config": {"side": side, "max_actions": m1, "min_actions": m2, "rows": int(len(rew)),
                       "precision": "mixed", "game_solver": "algebraic multigrid"}}


def tables_famg_block(stream, points=513):
    """Full multilevel policy iteration for a game given only by its tables
    (algebraic FAMGpi: coarse games by aggregation) against flat AMGpi, both
    on the algebraic-multigrid path, FP64: the Sec. 6.3 game at `points`
    points given as CSR tables; time, MAX iterations on the finest level."""
    import torch
    import synth
    import paper_1107_1653_gb300 as gs
    n, m1, m2, rp, col, prob, rew, mu = synth.two_stop_tables(points)
    out = {}
    for name, fmg in (("famgpi", 1), ("amgpi_flat", 0)):
        with gs.GameSolver(precision="fp64", game_solver=1, fmg=fmg, max_outer=100000,
                           max_inner=100000, stream=stream) as s:
            s.set_game(n, m1, m2, rp, col, prob, rew, mu)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = s.solve()
            e1.record(stream)
            torch.cuda.synchronize()
        out[name] = {"ms": e0.elapsed_time(e1), "outer_finest": st["outer"], "systems_finest": st["systems"],
                     "cycles": st["cycles"], "fmg_levels": st["fmg_levels"], "converged": st["converged"]}
    out["config"] = {"game": "Sec. 6.3 two-sided stopping game as CSR tables", "points": points,
                     "precision": "fp64", "game_solver": "algebraic multigrid"}
    return out


def run_obstacle_1023(args, stream):
    """The obstacle configuration: 1023 x 1023 obstacle Isaacs game, seed 2,
    flat AMGpi against FAMGpi from 31 x 31 (eps_l = 0.01 h_l^2, eps = 0 on the
    finest level), FP64 and mixed, each timed (L2 flushed between solves), and
    every result's error against the stored FP64 oracle run (sampled states)."""
    import torch
    import paper_1107_1653_gb300 as gs
    samples = load_samples("isaacs1023_obstacle_seed2_samples.txt")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    # the plain grid under FAMGpi (its flat solve is the headline), c = 0.1
    plain = load_samples("isaacs1023_plain_seed2_samples.txt")
    for prec in ("fp64", "mixed"):
        s = gs.GameSolver(precision=prec, fmg=1, fmg_side=31, fmg_c=0.1, stream=stream, **ISAACS_CYCLE)
        s.set_isaacs_grid(SIDE, 0, SEED)
        s.solve()
        ts, st = [], None
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = s.solve()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        v = s.get_value()
        s.close()
        ms = statistics.mean(ts)
        out["plain_%s_famg" % prec] = {"ms_per_solve": ms, "solves_per_s": 1000.0 / ms, "outer": st["outer"],
                                       "systems": st["systems"], "cycles": st["cycles"],
                                       "err_vs_oracle_sampled": err_vs_samples(v, plain)}
    for prec in ("fp64", "mixed"):
        for fmg in (0, 1):
            s = gs.GameSolver(precision=prec, fmg=fmg, fmg_side=31, fmg_c=0.01, stream=stream,
                              **ISAACS_CYCLE)
            s.set_isaacs_grid(SIDE, 1, SEED)
            s.solve()
            ts, st = [], None
            for _ in range(2 if not fmg else 3):
                flush.zero_()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = s.solve()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            v = s.get_value()
            s.close()
            ms = statistics.mean(ts)
            out["%s_%s" % (prec, "famg" if fmg else "flat")] = {
                "ms_per_solve": ms, "solves_per_s": 1000.0 / ms, "outer": st["outer"],
                "systems": st["systems"], "cycles": st["cycles"],
                "err_vs_oracle_sampled": err_vs_samples(v, samples)}
    out["config"] = {"side": SIDE, "variant": "obstacle (plain_* entries: the plain grid)", "seed": SEED,
                     "cycle": cycle_label(ISAACS_CYCLE),
                     "famg": "from 31 x 31, eps_l = c h_l^2 (c = 0.01 obstacle, 0.1 plain), eps = 0 on the finest level",
                     "l2": "flushed between solves (256 MiB write)",
                     "oracle": "isaacs1023_obstacle_seed2_samples.txt and isaacs1023_plain_seed2_samples.txt (1,026 states each)"}
    return out


def line_results(args):
    """The two-sided stopping game on a line (Sec. 6.3) at 2049 points: FAMGpi
    (eps_l = 1e-2 h_l^2, eps = 1e-10, as the paper's table) timed over the
    steps, flat AMGpi once; the discretisation errors against the exact
    solution (the paper prints |e|_inf = 1.16e-7, |e|_L2 = 7.40e-8)."""
    import numpy as np
    import torch
    import synth
    import paper_1107_1653_gb300 as gs
    points = 2049
    c, p1, p2, vl, vr = synth.stopping_line(points)
    m = points - 1
    x = np.arange(1, m) / m
    s9, c9 = np.sin(0.09 * np.pi), np.cos(0.09 * np.pi)
    psi = (2 * c9 + np.pi * (0.18 - 1) * s9) / 2
    exact = np.cos(np.pi * x) + np.pi * s9 * x + (psi - c9 - 0.09 * np.pi * s9)
    exact = np.where(x < 0.09, psi, np.where(x > 0.91, -psi, exact))
    stream = torch.cuda.current_stream()
    out = {}
    for name, fmg, steps in (("famgpi", 1, args.steps), ("amgpi", 0, 1)):
        s = gs.GameSolver(fmg=fmg, fmg_c=1e-2, eps=1e-10, max_inner=100000, max_outer=100000,
                          stream=stream)
        s.set_stopping_line(c, p1, p2, vl, vr)
        for _ in range(args.warmup if fmg else 0):
            s.solve()
        ts = []
        for _ in range(steps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = s.solve()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        e = s.get_value() - exact
        s.close()
        out[name] = {"ms": statistics.mean(ts), "outer": st["outer"], "systems": st["systems"],
                     "cycles": st["cycles"], "fmg_levels": st["fmg_levels"],
                     "e_inf": float(np.max(np.abs(e))), "e_l2": float(np.sqrt(np.mean(e * e))),
                     "res_inf": st["res_inf"]}
    return points, out


def run_line(args):
    import torch
    torch.cuda.set_device(0)
    points, out = line_results(args)
    line = {"metric": "two-sided stopping game (Sec. 6.3) solves/s at 2049 points, FAMGpi",
            "value": 1000.0 / out["famgpi"]["ms"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["famgpi"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "stopping_line_2049", "points": points},
            "famgpi": out["famgpi"], "amgpi_flat": out["amgpi"],
            "speedup_famgpi_vs_flat": out["amgpi"]["ms"] / out["famgpi"]["ms"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "mixed_bf16"])
    ap.add_argument("--fmg", type=int, default=0)
    ap.add_argument("--trace-kernel", default="mg_cycles", choices=["mg_cycles", "none"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-2047", action="store_true",
                    help="skip the 2047^2 precision configuration's block")
    ap.add_argument("--no-obstacle", action="store_true",
                    help="skip the 1023^2 obstacle block (flat AMGpi against FAMGpi)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the compact 4096-game batch and serving-stream blocks")
    ap.add_argument("--side", type=int, default=SIDE)
    ap.add_argument("--workload", default="isaacs", choices=["isaacs", "batch", "serving", "line"],
                    help="isaacs: the metric's 1023^2 solve (default); batch: 4096 random "
                         "games; serving: a Poisson request stream; line: the Sec. 6.3 "
                         "stopping game at 2049 points, FAMGpi against flat AMGpi")
    ap.add_argument("--games", type=int, default=4096)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--burst", type=int, default=64)
    ap.add_argument("--slots", type=int, default=2)
    ap.add_argument("--profile", action="store_true",
                    help="run one solve only (for ncu); prints the solve statistics")
    ap.add_argument("--profile-game", type=int, default=0,
                    help="one random-game solve of this many states (for ncu)")
    args = ap.parse_args()
    globals()["SIDE"] = args.side
    if args.profile:
        return run_profile(args)
    if args.profile_game:
        return run_profile_game(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "line":
        return run_line(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
