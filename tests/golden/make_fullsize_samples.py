"""Writes the full-size sampled fixtures of the FP64 oracle.

The GPU parity tests at the workloads' full sizes compare the device solve
with these stored oracle outputs at a seeded sample of states: the oracle
takes minutes to an hour per workload, too long to run beside the GPU.
Calls only oracle/ (and the seeded input generators of synth/).

    python tests/golden/make_fullsize_samples.py isaacs2047_seed3   # ~16 min, ~12 GB
    python tests/golden/make_fullsize_samples.py isaacs1023_seed2   # ~3 min
    python tests/golden/make_fullsize_samples.py obstacle1023
    python tests/golden/make_fullsize_samples.py batch4096

* isaacs2047_seed2, isaacs2047_seed3, isaacs1023_seed2: Algorithm 2 with
  Algorithm 1 inside (sparse LU) on the plain 2047 x 2047 (1023 x 1023) Isaacs
  game, from the default start.
* obstacle1023: the obstacle variant at 1023 x 1023, seed 2.  The oracle runs
  its own FAMGpi (Algorithm 4, from 31 x 31, eps_l = 0.01 h_l^2) with eps = 0
  on the finest level, so the last policy iteration runs until MAX's policy
  is unchanged: the fixed point of Eq. (eq1), which is unique (Sec. 2).
* batch4096: 32 games drawn with a seeded generator from the 4096-game batch
  (n ~ U{256..8192}, seed 4), each solved alone by policy iteration with the
  fixed-point policy evaluation to 1e-14.

Each fixture row holds a state's value, MAX's action, MIN's reply for every
MAX action, and the oracle's gaps (best minus second best) that decide
which policy entries are unique.
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle.fmg import famg_pi  # noqa: E402
from oracle.game import game_from_csr  # noqa: E402
from oracle.isaacs import isaacs_game  # noqa: E402

SAMPLES = 1024
BATCH_GAMES, BATCH_STATES = 32, 64


def sample_states(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct states, the first and last included, in increasing order."""
    rng = np.random.default_rng(seed)
    pick = rng.choice(n, size=min(k, n), replace=False)
    return np.unique(np.concatenate([[0, n - 1], pick]))


def rows(res, idx, prefix=""):
    out = []
    m1 = res.beta.shape[1]
    for x in idx:
        beta = " ".join(str(int(res.beta[x, a])) for a in range(m1))
        gmin = " ".join(f"{res.gap_min[x, a]:.3e}" for a in range(m1))
        out.append(f"{prefix}{x} {res.v[x]:.17e} {int(res.alpha[x])} {beta} "
                   f"{res.gap_max[x]:.3e} {gmin}\n")
    return out


def write(name, header, body):
    with open(os.path.join(HERE, name), "w") as fh:
        for line in header:
            fh.write(f"# {line}\n")
        fh.writelines(body)


def isaacs_plain(side: int, seed: int):
    t0 = time.time()
    res = oracle.policy_iteration(isaacs_game(side, 0, seed=seed))
    idx = sample_states(res.v.size, SAMPLES, side)
    write(f"isaacs{side}_plain_seed{seed}_samples.txt",
          ["FP64 oracle, Algorithm 2 with Algorithm 1 inside (sparse LU), plain Isaacs game",
           f"{side} x {side}, seed {seed}; written by make_fullsize_samples.py isaacs{side}_seed{seed}",
           "columns: state v alpha beta(x,0..m1-1) gap_max gap_min(x,0..m1-1)",
           f"outer {res.outer} systems {res.systems} residual {res.residual:.3e}"],
          [f"vmax {np.max(np.abs(res.v)):.17e}\n"] + rows(res, idx))
    print(f"isaacs{side} seed {seed}: outer {res.outer} systems {res.systems} "
          f"residual {res.residual:.2e} in {time.time() - t0:.0f} s")


def isaacs2047(seed: int):
    isaacs_plain(2047, seed)


def obstacle1023():
    t0 = time.time()
    res, levels = famg_pi(1023, 31, 1, synth.isaacs_noise(1023, 2), c=0.01, eps=0.0)
    idx = sample_states(res.v.size, SAMPLES, 1023)
    write("isaacs1023_obstacle_seed2_samples.txt",
          ["FP64 oracle, FAMGpi (Algorithm 4) from 31 x 31 with eps_l = 0.01 h_l^2 and",
           "eps = 0 on the finest level (policy iteration until alpha is unchanged),",
           "obstacle Isaacs game 1023 x 1023, seed 2; make_fullsize_samples.py obstacle1023",
           "columns: state v alpha beta(x,0..m1-1) gap_max gap_min(x,0..m1-1)",
           f"finest level: outer {res.outer} systems {res.systems} residual {res.residual:.3e}"],
          [f"vmax {np.max(np.abs(res.v)):.17e}\n"] + rows(res, idx))
    print(f"obstacle1023: finest outer {res.outer} systems {res.systems} "
          f"residual {res.residual:.2e} in {time.time() - t0:.0f} s")


def _solve_batch_game(args):
    g, n = args
    rp, col, prob, rew, mu = synth.random_game(int(n), synth.batch_game_seed(4, int(g)))
    game = game_from_csr(int(n), 4, 4, rp, col, prob, rew, mu)
    res = oracle.policy_iteration(game, solver="fixed_point")
    idx = sample_states(int(n), BATCH_STATES, 4096 + int(g))
    head = f"game {g} n {n} vmax {np.max(np.abs(res.v)):.17e} outer {res.outer} " \
           f"systems {res.systems} residual {res.residual:.3e}\n"
    return [head] + rows(res, idx, prefix=f"{g} ")


def batch4096():
    t0 = time.time()
    sizes = synth.batch_game_sizes(4096, 4)
    games = np.sort(np.random.default_rng(4096).choice(4096, BATCH_GAMES, replace=False))
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        parts = pool.map(_solve_batch_game, [(int(g), int(sizes[g])) for g in games])
    write("batch4096_seed4_samples.txt",
          ["FP64 oracle, Algorithm 2 with Algorithm 1 inside (fixed-point policy evaluation",
           "to 1e-14), 32 games of the 4096-game random batch (seed 4) solved alone;",
           "written by make_fullsize_samples.py batch4096",
           "'game' rows: index, size, max |v|, counts; state rows: game state v alpha",
           "beta(x,0..3) gap_max gap_min(x,0..3)"],
          [line for part in parts for line in part])
    print(f"batch4096: {len(games)} games in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    jobs = {"isaacs2047_seed2": lambda: isaacs2047(2), "isaacs2047_seed3": lambda: isaacs2047(3),
            "isaacs1023_seed2": lambda: isaacs_plain(1023, 2),
            "obstacle1023": obstacle1023, "batch4096": batch4096}
    for name in sys.argv[1:] or list(jobs):
        jobs[name]()
