"""GPU parity of the finite-game path (CSR tables) against the FP64 oracle.

Bars as for the Isaacs path: value to 1e-10 relative (float64) / 1e-9 (mixed),
policies bit-exact wherever the oracle's max-min gap exceeds 1e-8.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.game import game_from_csr

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-9, "mixed_bf16": 1e-9}


def oracle_of(n, m1, m2, rp, col, prob, rew, mu):
    game = game_from_csr(n, m1, m2, rp, col, prob, rew, mu)
    res = oracle.policy_iteration(game, solver="fixed_point" if n > 2000 else "auto")
    return game, res


def check(v, a, b, ref):
    err = np.max(np.abs(v - ref.v)) / max(np.max(np.abs(ref.v)), 1e-300)
    sure_a = ref.gap_max > 1e-8
    assert np.array_equal(a[sure_a], ref.alpha[sure_a])
    sure_b = ref.gap_min > 1e-8
    assert np.array_equal(b.reshape(ref.beta.shape)[sure_b], ref.beta[sure_b])
    return err


def tiny_game(seed, n, m1, m2):
    """Dense random game with some substochastic and some empty (stop) rows."""
    rng = np.random.default_rng(seed)
    R = n * m1 * m2
    rp, col, prob = [0], [], []
    for r in range(R):
        if rng.random() < 0.1:          # a stop row: no successors
            rp.append(len(col))
            continue
        k = rng.integers(1, n + 1)
        cs = np.sort(rng.choice(n, size=k, replace=False))
        p = rng.random(k)
        p /= p.sum()
        if rng.random() < 0.3:
            p *= rng.uniform(0.5, 1.0)
        col.extend(cs.tolist())
        prob.extend(p.tolist())
        rp.append(len(col))
    rew = rng.uniform(-1, 1, R)
    return np.array(rp, np.int64), np.array(col, np.int32), np.array(prob), rew


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,m1,m2", [(1, 1, 1), (2, 2, 2), (4, 2, 2), (5, 3, 2), (7, 8, 8)])
def test_tiny_games(gs, n, m1, m2, prec):
    rp, col, prob, rew = tiny_game(100 * n + m1, n, m1, m2)
    mu = 0.9
    _, ref = oracle_of(n, m1, m2, rp, col, prob, rew, mu)
    with gs.GameSolver(precision=prec) as s:
        s.set_game(n, m1, m2, rp, col, prob, rew, mu)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    assert check(v, a, b, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
@pytest.mark.parametrize("n", [256, 1000, 4096])
def test_random_game(gs, n, prec):
    rp, col, prob, rew, mu = synth.random_game(n, 4 + n)
    _, ref = oracle_of(n, 4, 4, rp, col, prob, rew, mu)
    with gs.GameSolver(precision=prec) as s:
        s.set_game(n, 4, 4, rp, col, prob, rew, mu)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    assert check(v, a, b, ref) <= TOL[prec], st


def test_single_action_closed_form(gs):
    n = 300
    rp, col, prob, rew, mu = synth.random_game(n, 3, m1=1, m2=1, mu=0.95)
    P = np.zeros((n, n))
    for r in range(n):
        for k in range(rp[r], rp[r + 1]):
            P[r, col[k]] += prob[k]
    w = np.linalg.solve(np.eye(n) - mu * P, rew)
    with gs.GameSolver() as s:
        s.set_game(n, 1, 1, rp, col, prob, rew, mu)
        st = s.solve()
        v = s.get_value()
    assert st["outer"] == 1
    assert np.max(np.abs(v - w)) / np.max(np.abs(w)) <= 1e-10


def batch(sizes, seed):
    parts = [synth.random_game(int(n), synth.batch_game_seed(seed, i)) for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rps, cols, probs, rews, mus = [], [], [], [], []
    nnz = 0
    for i, (rp, col, prob, rew, mu) in enumerate(parts):
        rps.append(rp[:-1] + nnz if i < len(parts) - 1 else rp + nnz)
        nnz += rp[-1]
        cols.append(col)
        probs.append(prob)
        rews.append(rew)
        mus.append(mu)
    return (off, np.concatenate(rps), np.concatenate(cols), np.concatenate(probs),
            np.concatenate(rews), np.array(mus)), parts


@pytest.mark.parametrize("prec", ["mixed", "fp64", "mixed_bf16"])
def test_game_batch(gs, prec):
    sizes = synth.batch_game_sizes(24, 4, nmin=256, nmax=1500)
    (off, rp, col, prob, rew, mu), parts = batch(sizes, 4)
    with gs.GameSolver(precision=prec) as s:
        s.set_game_batch(off, 4, 4, rp, col, prob, rew, mu)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
        gst, gres = s.batch_stats()
    assert st["converged"] == 1 and np.all(gst[:, 3] == 1)
    for g, n in enumerate(sizes):
        x0, x1 = off[g], off[g + 1]
        _, ref = oracle_of(int(n), 4, 4, *parts[g])
        assert check(v[x0:x1], a[x0:x1], b[x0:x1], ref) <= TOL[prec], g
        assert gres[g] <= 1e-9


@pytest.mark.parametrize("threads", [256, 512])
def test_game_batch_shapes(gs, threads):
    """Both block shapes of the batch kernel, forced, solve every game."""
    sizes = synth.batch_game_sizes(24, 5, nmin=256, nmax=1500)
    (off, rp, col, prob, rew, mu), parts = batch(sizes, 5)
    with gs.GameSolver(precision="mixed", game_threads=threads) as s:
        s.set_game_batch(off, 4, 4, rp, col, prob, rew, mu)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
        gst, _ = s.batch_stats()
        assert s.batch_shape() == threads
    assert st["converged"] == 1 and np.all(gst[:, 3] == 1)
    for g, n in enumerate(sizes):
        x0, x1 = off[g], off[g + 1]
        _, ref = oracle_of(int(n), 4, 4, *parts[g])
        assert check(v[x0:x1], a[x0:x1], b[x0:x1], ref) <= TOL["mixed"], g


def test_batch_shape_autotuned(gs):
    """A batch of >= 1024 games autotunes its block shape on a sample; the
    result agrees with the other shape's and, on sampled games, the oracle's."""
    sizes = synth.batch_game_sizes(1100, 6, nmin=64, nmax=400)
    (off, rp, col, prob, rew, mu), parts = batch(sizes, 6)
    with gs.GameSolver(precision="mixed") as s:
        s.set_game_batch(off, 4, 4, rp, col, prob, rew, mu)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
        shape = s.batch_shape()
    assert shape in (256, 512)
    assert st["converged"] == 1
    other = 512 if shape == 256 else 256
    with gs.GameSolver(precision="mixed", game_threads=other) as s:
        s.set_game_batch(off, 4, 4, rp, col, prob, rew, mu)
        s.solve()
        w = s.get_value()
    for g in range(len(sizes)):
        x0, x1 = off[g], off[g + 1]
        assert np.max(np.abs(v[x0:x1] - w[x0:x1])) <= 1e-11 * np.max(np.abs(w[x0:x1])), g
    for g in np.random.default_rng(6).choice(len(sizes), 6, replace=False):
        x0, x1 = off[g], off[g + 1]
        _, ref = oracle_of(int(sizes[g]), 4, 4, *parts[g])
        assert check(v[x0:x1], a[x0:x1], b[x0:x1], ref) <= TOL["mixed"], g


def test_game_validation(gs):
    n = 50
    rp, col, prob, rew, mu = synth.random_game(n, 1)
    with gs.GameSolver() as s:
        bad = prob.copy()
        bad[5] = -0.1
        with pytest.raises(gs.GameSolveError) as e:
            s.set_game(n, 4, 4, rp, col, bad, rew, mu)
        assert e.value.status == gs.GS_EINVAL
        badc = col.copy()
        badc[7] = n
        with pytest.raises(gs.GameSolveError):
            s.set_game(n, 4, 4, rp, badc, prob, rew, mu)
        big = prob.copy()
        big[:8] *= 1.5
        with pytest.raises(gs.GameSolveError):
            s.set_game(n, 4, 4, rp, col, big, rew, mu)
        with pytest.raises(gs.GameSolveError):
            s.set_game(n, 4, 4, rp, col, prob, rew, 1.0)
        s.set_game(n, 4, 4, rp, col, prob, rew, mu)   # the valid table is accepted
        assert s.solve()["converged"] == 1


@pytest.mark.parametrize("prec", ["mixed", "fp64", "mixed_bf16"])
@pytest.mark.parametrize("n,blocks", [(5000, 0), (12000, 0), (12000, 8)])
def test_large_game_on_the_grid(gs, n, blocks, prec):
    """Games of >= 4096 states set alone run on a cooperative grid (policy
    iteration on the device, bounded grid barriers); grid_blocks caps it."""
    rp, col, prob, rew, mu = synth.random_game(n, 70 + n)
    _, ref = oracle_of(n, 4, 4, rp, col, prob, rew, mu)
    with gs.GameSolver(precision=prec, grid_blocks=blocks) as s:
        s.set_game(n, 4, 4, rp, col, prob, rew, mu)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    assert check(v, a, b, ref) <= TOL[prec], st
