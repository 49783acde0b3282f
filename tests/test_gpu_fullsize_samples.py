"""Parity at the workloads' full sizes on sampled states of stored oracle runs.

The FP64 oracle needs minutes to an hour on these workloads, so its results
are stored at a seeded sample of states (tests/golden/*_samples.txt, written
by tests/golden/make_fullsize_samples.py, which calls only the oracle).  The
GPU solves in the launch configuration the benchmark times (its cycle options
for the Isaacs grids; one persistent launch over the whole 4096-game batch).

Bars: value to 1e-10 relative to max |v*| (float64 path), 1e-9 (mixed and
bfloat16-storage paths); policies bit-exact wherever the oracle's gap exceeds
1e-8.  Beyond the sample, the float64 and mixed solutions of the 2047 x 2047
game agree at every state within the mixed bar.  The 2047 x 2047 game is
checked at seeds 2 and 3.
"""
import os

import numpy as np
import pytest

import synth
from bench import ISAACS_CYCLE as CYCLE

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = {"fp64": 1e-10, "mixed": 1e-9, "mixed_bf16": 1e-9}
SURE = 1e-8


def parse_rows(lines):
    """state rows -> (idx, v, alpha, beta[k, m1], gap_max, gap_min[k, m1])."""
    cols = [ln.split() for ln in lines]
    m1 = (len(cols[0]) - 4) // 2
    idx = np.array([int(c[0]) for c in cols], np.int64)
    v = np.array([float(c[1]) for c in cols])
    alpha = np.array([int(c[2]) for c in cols], np.uint8)
    beta = np.array([[int(x) for x in c[3:3 + m1]] for c in cols], np.uint8)
    gmax = np.array([float(c[3 + m1]) for c in cols])
    gmin = np.array([[float(x) for x in c[4 + m1:4 + 2 * m1]] for c in cols])
    return idx, v, alpha, beta, gmax, gmin


def load_grid_samples(name):
    vmax, body = None, []
    with open(os.path.join(GOLDEN, name)) as fh:
        for ln in fh:
            if ln.startswith("#"):
                continue
            if ln.startswith("vmax"):
                vmax = float(ln.split()[1])
            else:
                body.append(ln)
    return vmax, parse_rows(body)


def check_sample(v, a, b, vmax, sample, tol):
    idx, vs, alpha, beta, gmax, gmin = sample
    err = np.max(np.abs(v[idx] - vs)) / vmax
    assert err <= tol, err
    assert abs(np.max(np.abs(v)) - vmax) / vmax <= tol
    sure_a = gmax > SURE
    assert np.array_equal(a[idx][sure_a], alpha[sure_a])
    sure_b = gmin > SURE
    assert np.array_equal(b.reshape(len(v), -1)[idx][sure_b], beta[sure_b])
    # the sample must decide most policy entries, else it pins little
    assert sure_a.mean() > 0.5 and sure_b.mean() > 0.5
    return err


@pytest.fixture(scope="module", params=[2, 3])
def case2047(request, gs):
    """(seed, stored oracle sample, float64 GPU solve) of the 2047 x 2047 game."""
    seed = request.param
    vmax, sample = load_grid_samples(f"isaacs2047_plain_seed{seed}_samples.txt")
    with gs.GameSolver(precision="fp64", **CYCLE) as s:
        s.set_isaacs_grid(2047, 0, seed)
        st = s.solve()
        v64 = s.get_value()
    return seed, vmax, sample, st, v64


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
def test_isaacs_2047_sampled_parity(gs, case2047, prec):
    seed, vmax, sample, st64, v64 = case2047
    with gs.GameSolver(precision=prec, **CYCLE) as s:
        s.set_isaacs_grid(2047, 0, seed)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    check_sample(v, a, b, vmax, sample, TOL[prec])
    assert st64["converged"] == 1
    # every state, not only the sample: mixed against float64 on the device
    assert np.max(np.abs(v - v64)) / vmax <= TOL[prec]


@pytest.mark.parametrize("prec,fmg", [("fp64", 0), ("mixed", 0), ("mixed", 1), ("mixed_bf16", 1)])
def test_obstacle_1023_sampled_parity(gs, prec, fmg):
    vmax, sample = load_grid_samples("isaacs1023_obstacle_seed2_samples.txt")
    with gs.GameSolver(precision=prec, fmg=fmg, fmg_side=31, fmg_c=0.01, **CYCLE) as s:
        s.set_isaacs_grid(1023, 1, 2)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    check_sample(v, a, b, vmax, sample, TOL[prec])


def load_batch_samples():
    games, rows = {}, []
    with open(os.path.join(GOLDEN, "batch4096_seed4_samples.txt")) as fh:
        for ln in fh:
            if ln.startswith("#"):
                continue
            if ln.startswith("game"):
                f = ln.split()
                games[int(f[1])] = (int(f[3]), float(f[5]))
            else:
                rows.append(ln)
    g_of_row = np.array([int(r.split(None, 1)[0]) for r in rows])
    sample = parse_rows([r.split(None, 1)[1] for r in rows])
    return games, g_of_row, sample


def test_batch4096_sampled_parity(gs):
    games, g_of_row, (idx, vs, alpha, beta, gmax, gmin) = load_batch_samples()
    sizes = synth.batch_game_sizes(4096, 4)
    for g, (n, _) in games.items():
        assert sizes[g] == n
    off, rp, col, prob, rew, mu = synth.random_game_batch(sizes, 4, workers=os.cpu_count() or 1)
    with gs.GameSolver(precision="mixed") as s:
        s.set_game_batch(off, 4, 4, rp, col, prob, rew, mu)
        del rp, col, prob, rew
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
        gst, gres = s.batch_stats()
    assert st["converged"] == 1 and np.all(gst[:, 3] == 1)
    assert gres.max() <= 1e-9
    b = b.reshape(len(v), 4)
    for g, (n, vmax) in games.items():
        rows = g_of_row == g
        x = off[g] + idx[rows]
        err = np.max(np.abs(v[x] - vs[rows])) / vmax
        assert err <= TOL["mixed"], (g, err)
        assert abs(np.max(np.abs(v[off[g]:off[g + 1]])) - vmax) / vmax <= TOL["mixed"], g
        sa = gmax[rows] > SURE
        assert np.array_equal(a[x][sa], alpha[rows][sa]), g
        sb = gmin[rows] > SURE
        assert np.array_equal(b[x][sb], beta[rows][sb]), g
