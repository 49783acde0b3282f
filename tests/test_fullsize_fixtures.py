"""The stored full-size oracle samples (tests/golden/*_samples.txt) on the CPU.

* The writer (make_fullsize_samples.py) and the reader of the GPU parity tests
  round-trip an oracle result exactly, on a game small enough to solve here.
* Batch fixture: the two smallest of its sampled games, solved again by the
  oracle, give the stored rows.
* Every fixture decides most of its policy entries (gaps above 1e-8) and its
  values lie within its stored max |v|.
"""
import importlib.util
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.game import game_from_csr
from oracle.isaacs import default_alpha0, isaacs_game
from test_gpu_fullsize_samples import load_batch_samples, load_grid_samples, parse_rows

HERE = os.path.dirname(os.path.abspath(__file__))


def writer():
    spec = importlib.util.spec_from_file_location(
        "make_fullsize_samples", os.path.join(HERE, "golden", "make_fullsize_samples.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("variant", [0, 1])
def test_rows_round_trip(variant):
    w = writer()
    res = oracle.policy_iteration(isaacs_game(15, variant, seed=3),
                                  alpha0=default_alpha0(15, variant))
    idx = w.sample_states(res.v.size, 40, 7)
    assert idx[0] == 0 and idx[-1] == res.v.size - 1 and np.all(np.diff(idx) > 0)
    i, v, a, b, gmax, gmin = parse_rows(w.rows(res, idx))
    assert np.array_equal(i, idx)
    assert np.array_equal(v, res.v[idx])                     # 17 significant digits
    assert np.array_equal(a, res.alpha[idx])
    assert np.array_equal(b, res.beta[idx])
    assert np.allclose(gmax, res.gap_max[idx], rtol=1e-3, atol=0)
    assert np.allclose(gmin, res.gap_min[idx], rtol=1e-3, atol=0)


def test_batch_fixture_is_the_oracles():
    games, g_of_row, (idx, vs, alpha, beta, gmax, gmin) = load_batch_samples()
    sizes = synth.batch_game_sizes(4096, 4)
    for g in sorted(games, key=lambda g: games[g][0])[:2]:
        n, vmax = games[g]
        assert sizes[g] == n
        rp, col, prob, rew, mu = synth.random_game(n, synth.batch_game_seed(4, g))
        res = oracle.policy_iteration(game_from_csr(n, 4, 4, rp, col, prob, rew, mu),
                                      solver="fixed_point")
        rows = g_of_row == g
        x = idx[rows]
        assert np.array_equal(vs[rows], res.v[x])
        assert float(np.max(np.abs(res.v))) == vmax
        assert np.array_equal(alpha[rows], res.alpha[x])
        assert np.array_equal(beta[rows], res.beta[x])


@pytest.mark.parametrize("name", ["isaacs2047_plain_seed2_samples.txt",
                                  "isaacs2047_plain_seed3_samples.txt",
                                  "isaacs1023_obstacle_seed2_samples.txt"])
def test_grid_fixtures_are_well_formed(name):
    vmax, (idx, v, a, b, gmax, gmin) = load_grid_samples(name)
    side = 2047 if "2047" in name else 1023
    m1 = 5 if "obstacle" in name else 4
    assert len(idx) > 1000 and idx[0] == 0 and idx[-1] == side * side - 1
    assert np.all(np.diff(idx) > 0)
    assert b.shape == (len(idx), m1) and np.all(a < m1) and np.all(b < 4)
    assert np.max(np.abs(v)) <= vmax
    assert (gmax > 1e-8).mean() > 0.5 and (gmin > 1e-8).mean() > 0.5
    if m1 == 5:
        # the obstacle's value is at least the stop reward psi, with equality
        # where MAX stops (Sec. 3.2, Eq. (VI))
        h = 1.0 / (side + 1)
        x1, x2 = (idx % side + 1) * h, (idx // side + 1) * h
        psi = 0.2 - ((x1 - 0.5) ** 2 + (x2 - 0.5) ** 2)
        assert np.all(v >= psi - 1e-15)
        stop = a == 4
        assert stop.any() and np.allclose(v[stop], psi[stop], rtol=0, atol=1e-15)


def test_batch_fixture_is_well_formed():
    games, g_of_row, (idx, vs, alpha, beta, gmax, gmin) = load_batch_samples()
    assert len(games) == 32
    for g, (n, vmax) in games.items():
        rows = g_of_row == g
        assert rows.sum() >= 64 and idx[rows][0] == 0 and idx[rows][-1] == n - 1
        assert np.max(np.abs(vs[rows])) <= vmax <= 1.0 / (1.0 - 0.99)   # |r| <= 1, mu = 0.99
