"""Serving: continuous batching of Isaacs and finite-game requests.

Each result must be the same alone and in the mix: Isaacs values bit for bit
(their kernels' arithmetic does not depend on what else runs), finite games to
1e-12 relative (a grid-wide game's reductions may use a different number of
blocks when the server caps its share of the GPU).  Every result is also
checked against the FP64 oracle: the small mix against full oracle solves,
the full-size requests against stored oracle runs at sampled states
(1023 x 1023 plain and obstacle) or, where no oracle run fits the test's
time, against the oracle's Shapley operator applied to the served value.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.fmg import famg_pi
from oracle.game import game_from_csr
from oracle.isaacs import isaacs_game, default_alpha0

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-9          # value bar of the mixed path, relative to max |v*|
SURE = 1e-8               # policies compared where the oracle's gap exceeds this


def mix():
    reqs = []
    for k, (side, variant) in enumerate(((15, 0), (63, 1), (127, 0), (255, 0), (31, 1), (63, 0),
                                         (127, 1))):
        reqs.append(("isaacs", side, variant, 100 + k))
    for k, n in enumerate((300, 1500, 5000, 9000)):
        reqs.append(("game", n, synth.random_game(n, 500 + k)))
    return reqs


def oracle_result(r):
    """The oracle's solution of a request: policy iteration (obstacle grids via
    the oracle's own FAMGpi, which reaches the same unique fixed point in
    fewer steps; games above 2000 states with the fixed-point evaluation)."""
    if r[0] == "isaacs":
        side, variant, seed = r[1], r[2], r[3]
        if variant == 1 and side >= 31:
            res, _ = famg_pi(side, 15, 1, synth.isaacs_noise(side, seed), c=0.01, eps=0.0)
            return res
        return oracle.policy_iteration(isaacs_game(side, variant, seed=seed),
                                       alpha0=default_alpha0(side, variant))
    n, (rp, col, prob, rew, mu) = r[1], r[2]
    game = game_from_csr(n, 4, 4, rp, col, prob, rew, mu)
    return oracle.policy_iteration(game, solver="auto" if n <= 2000 else "fixed_point")


def check_against_oracle(v, a, b, ref, tag):
    scale = np.max(np.abs(ref.v))
    assert np.max(np.abs(v - ref.v)) <= TOL_MIXED * scale, tag
    sure_a = ref.gap_max > SURE
    assert np.array_equal(a[sure_a], ref.alpha[sure_a]), tag
    m = min(b.shape[1], ref.beta.shape[1], 4)
    sure_b = ref.gap_min[:, :m] > SURE
    assert np.array_equal(b[:, :m][sure_b], ref.beta[:, :m][sure_b]), tag


def alone(gs, r):
    with gs.GameSolver(precision="mixed") as s:
        if r[0] == "isaacs":
            s.set_isaacs_grid(r[1], r[2], r[3])
        else:
            n, (rp, col, prob, rew, mu) = r[1], r[2]
            s.set_game(n, 4, 4, rp, col, prob, rew, mu)
        s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    return v, a, b


def submit(srv, r):
    if r[0] == "isaacs":
        return srv.submit_isaacs(r[1], r[2], r[3])
    n, (rp, col, prob, rew, mu) = r[1], r[2]
    return srv.submit_game(n, 4, 4, rp, col, prob, rew, mu)


def test_results_alone_equal_in_the_mix(gs):
    reqs = mix()
    ref = [alone(gs, r) for r in reqs]
    with gs.GameServer(slots=4, precision="mixed") as srv:
        tickets = [submit(srv, r) for r in reqs]
        infos = [srv.wait(t) for t in tickets]
        out = [srv.result(t) for t in tickets]
    overlap = 0
    for i, (r, (v, a, b), (v0, a0, b0), info) in enumerate(zip(reqs, out, ref, infos)):
        assert info["state"] == 2 and info["status"] == gs.GS_OK
        assert info["t_submit"] <= info["t_start"] <= info["t_end"]
        if r[0] == "isaacs":
            assert np.array_equal(v, v0), i
            assert np.array_equal(a, a0) and np.array_equal(b, b0)
        else:
            assert np.max(np.abs(v - v0)) <= 1e-12 * np.max(np.abs(v0)), i
        check_against_oracle(v, a, b, oracle_result(r), (i, r[:2]))
        for j, other in enumerate(infos):
            if j != i and other["t_start"] < info["t_end"] and info["t_start"] < other["t_end"]:
                overlap += 1
    assert overlap > 0          # the requests' work did overlap


def test_full_size_requests_alone_equal_in_the_mix(gs):
    """The serving workload's largest requests: Isaacs grids up to 1023 x 1023
    (plain and obstacle) and the largest and smallest games of its pool
    (937,562 and 63,437 states, tables borrowed from device memory as the
    benchmark serves them), four slots."""

    import torch
    games = []
    for n, seed in ((937_562, 5007), (63_437, 5000)):
        rp, col, prob, rew, mu = synth.random_game_parallel(n, seed, workers=os.cpu_count() or 1)
        games.append((n, (rp, col, prob, rew, mu)))
    reqs = [("isaacs", 1023, 0, 2), ("isaacs", 1023, 1, 2), ("isaacs", 511, 0, 7),
            ("isaacs", 63, 0, 8)] + [("game", n, t) for n, t in games]
    ref = [alone(gs, r) for r in reqs]
    dev = {n: tuple(torch.from_numpy(x).cuda() for x in t[:4]) + (t[4],) for n, t in games}
    with gs.GameServer(slots=4, precision="mixed") as srv:
        tickets = []
        for r in reqs:
            if r[0] == "isaacs":
                tickets.append(srv.submit_isaacs(r[1], r[2], r[3]))
            else:
                rp, col, prob, rew, mu = dev[r[1]]
                tickets.append(srv.submit_game(r[1], 4, 4, rp, col, prob, rew, mu, borrow=True))
        infos = [srv.wait(t) for t in tickets]
        out = [srv.result(t) for t in tickets]
    torch.cuda.synchronize()
    for i, (r, (v, a, b), (v0, a0, b0), info) in enumerate(zip(reqs, out, ref, infos)):
        assert info["state"] == 2 and info["status"] == gs.GS_OK, i
        assert info["stats"]["converged"] == 1, i
        if r[0] == "isaacs":
            assert np.array_equal(v, v0), i
            assert np.array_equal(a, a0) and np.array_equal(b, b0), i
        else:
            assert np.max(np.abs(v - v0)) <= 1e-12 * np.max(np.abs(v0)), i
    # against the oracle: stored runs at sampled states for the 1023 x 1023
    # grids (seed 2), the oracle's Shapley operator elsewhere
    from test_gpu_fullsize_samples import load_grid_samples, check_sample
    for i, name in ((0, "isaacs1023_plain_seed2_samples.txt"),
                    (1, "isaacs1023_obstacle_seed2_samples.txt")):
        vmax, sample = load_grid_samples(name)
        v, a, b = out[i]
        check_sample(v, a, b, vmax, sample, TOL_MIXED)
    for i in (2, 3):
        side, variant, seed = reqs[i][1:]
        v = out[i][0]
        q = oracle.shapley_q(isaacs_game(side, variant, seed=seed), v)
        assert np.max(np.abs(q.min(axis=2).max(axis=1) - v)) <= 1e-12, i
    n, (rp, col, prob, rew, mu) = games[1]
    v = out[5][0]
    q = oracle.shapley_q(game_from_csr(n, 4, 4, rp, col, prob, rew, mu), v)
    res = np.max(np.abs(q.min(axis=2).max(axis=1) - v))
    # a-posteriori bound of the mu-contraction: |v - v*| <= res / (1 - mu)
    assert res / (1 - mu) <= TOL_MIXED * np.max(np.abs(v)), res


def test_memory_budget_serialises(gs):
    reqs = [("isaacs", 127, 0, 7 + k) for k in range(4)]
    with gs.GameServer(slots=4, mem_budget=1 << 20) as srv:   # below any one request
        tickets = [submit(srv, r) for r in reqs]
        infos = [srv.wait(t) for t in tickets]
        for t in tickets:
            srv.result(t)
    spans = sorted((i["t_start"], i["t_end"]) for i in infos)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0          # admitted one at a time


def test_invalid_requests(gs):
    with gs.GameServer(slots=1) as srv:
        with pytest.raises(gs.GameSolveError):
            srv.submit_isaacs(100)
        rp, col, prob, rew, mu = synth.random_game(50, 2)
        bad = prob.copy()
        bad[3] = -1.0
        t = srv.submit_game(50, 4, 4, rp, col, bad, rew, mu)
        info = srv.wait(t)
        assert info["status"] == gs.GS_EINVAL
        with pytest.raises(gs.GameSolveError):
            srv.result(t)


def test_small_games_batched(gs):
    """Small games (below the grid-wide threshold) that wait together with the
    same kind and action counts are solved as one batch: they share t_start,
    and each result equals the same game solved alone (the batch runs the
    one-block-per-game kernel each would run alone) and the oracle's."""
    drawn = [(n, 900 + k) for k, n in enumerate((200, 350, 800, 1200, 2000, 3000, 640, 999))]
    tables = [(n, synth.random_game(n, 1300 + k)) for k, n in enumerate((260, 500, 1800))]
    with gs.GameServer(slots=1, precision="mixed") as srv:
        t_big = srv.submit_isaacs(1023, 0, 4)     # holds the only slot while the rest queue
        t_drawn = [srv.submit_random_game(n, 4, 4, seed, 0.99) for n, seed in drawn]
        t_tab = [srv.submit_game(n, 4, 4, *tab) for n, tab in tables]
        i_drawn = [srv.wait(t) for t in t_drawn]
        i_tab = [srv.wait(t) for t in t_tab]
        o_drawn = [srv.result(t) for t in t_drawn]
        o_tab = [srv.result(t) for t in t_tab]
        assert srv.wait(t_big)["status"] == gs.GS_OK
        srv.result(t_big)
    assert len({i["t_start"] for i in i_drawn}) == 1
    assert len({i["t_start"] for i in i_tab}) == 1
    for k, ((n, seed), info, (v, a, b)) in enumerate(zip(drawn, i_drawn, o_drawn)):
        assert info["status"] == gs.GS_OK and info["stats"]["converged"] == 1, k
        assert info["stats"]["outer"] >= 1 and info["n"] == n
        with gs.GameSolver(precision="mixed") as s:
            s.set_random_game(n, 4, 4, seed, 0.99)
            st = s.solve()
            a0, b0 = s.get_policy()
            assert np.array_equal(v, s.get_value()), k
            assert np.array_equal(a, a0) and np.array_equal(b, b0), k
            assert info["stats"]["outer"] == st["outer"] and info["stats"]["systems"] == st["systems"]
        if k < 3:
            rp, col, prob, rew, mu = synth.random_game(n, seed)
            check_against_oracle(v, a, b, oracle.policy_iteration(
                game_from_csr(n, 4, 4, rp, col, prob, rew, mu)), ("drawn", k))
    for k, ((n, tab), info, (v, a, b)) in enumerate(zip(tables, i_tab, o_tab)):
        assert info["status"] == gs.GS_OK, k
        v0, a0, b0 = alone(gs, ("game", n, tab))
        assert np.array_equal(v, v0) and np.array_equal(a, a0) and np.array_equal(b, b0), k
        check_against_oracle(v, a, b, oracle_result(("game", n, tab)), ("table", k))


def test_bad_table_in_a_batch_fails_alone(gs):
    """A rejected table among batched games fails only its own request."""
    good = [synth.random_game(n, 1400 + n) for n in (300, 400)]
    bad = list(synth.random_game(350, 1500))
    bad[2] = bad[2].copy()
    bad[2][5] = 1.5                                   # a probability above one
    with gs.GameServer(slots=1, precision="mixed") as srv:
        t_big = srv.submit_isaacs(1023, 0, 5)
        tickets = [srv.submit_game(300, 4, 4, *good[0]), srv.submit_game(350, 4, 4, *bad),
                   srv.submit_game(400, 4, 4, *good[1])]
        infos = [srv.wait(t) for t in tickets]
        srv.wait(t_big)
        srv.result(t_big)
        assert infos[1]["status"] == gs.GS_EINVAL
        for t, info, (n, tab) in ((tickets[0], infos[0], (300, good[0])), (tickets[2], infos[2], (400, good[1]))):
            assert info["status"] == gs.GS_OK
            v, a, b = srv.result(t)
            assert np.array_equal(v, alone(gs, ("game", n, tab))[0])
