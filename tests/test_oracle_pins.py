"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: brute-force
enumeration of all pure stationary policy pairs (Sec. 2 theorem: the value is
attained by pure Markovian stationary strategies), closed forms, the
contraction and monotonicity of the Shapley operator (Sec. 2), the monotone
value sequences of policy iteration (Sec. 4.1-4.2), the a-posteriori bound that
follows from the mu-contraction, O(h) convergence of the Isaacs scheme
(Sec. 3.3) to a manufactured solution, and hand-worked interpolation examples
for FAMGpi (Sec. 5.2).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.game import game_from_csr, shapley_q, _keep_current
from oracle.isaacs import (isaacs_game, isaacs_geometry, stencil_probabilities,
                           default_alpha0, discount)
from oracle.fmg import interp_value, interp_policy, famg_pi, injected_noise

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def tiny_dense_game(seed, n, m1, m2, substochastic=True):
    """Dense p[x, a, b, y] (rows sum to <= 1) and r[x, a, b] for brute force."""
    rng = np.random.default_rng(seed)
    p = rng.random((n, m1, m2, n)) * (rng.random((n, m1, m2, n)) < 0.7)
    p[..., 0] += 1e-3                                  # no empty rows
    p /= p.sum(axis=-1, keepdims=True)
    if substochastic:
        p *= rng.uniform(0.6, 1.0, size=(n, m1, m2, 1)) ** (rng.random((n, m1, m2, 1)) < 0.3)
    r = rng.uniform(-1, 1, size=(n, m1, m2))
    return p, r


def dense_to_game(p, r, mu):
    n, m1, m2, _ = p.shape
    rows = p.reshape(n * m1 * m2, n)
    row_ptr = [0]
    col, prob = [], []
    for row in rows:
        nz = np.nonzero(row)[0]
        col.extend(nz.tolist())
        prob.extend(row[nz].tolist())
        row_ptr.append(len(col))
    return game_from_csr(n, m1, m2, np.array(row_ptr), np.array(col, np.int32),
                         np.array(prob), r.reshape(-1), mu)


def value_of(p, r, mu, alpha, bsel):
    """v^{alpha beta} = (I - mu M)^-1 r^{alpha beta} with M from dense p."""
    n = p.shape[0]
    xs = np.arange(n)
    M = p[xs, alpha, bsel, :]
    return np.linalg.solve(np.eye(n) - mu * M, r[xs, alpha, bsel])


def brute_force(p, r, mu):
    """v* = max_alpha min_beta v^{alpha beta}, componentwise, by enumeration.

    v^{alpha beta} depends on beta only through beta(x, alpha(x)), so MIN's
    choices are enumerated as one action per state.  Returns v* and, per
    alpha, MIN's componentwise-optimal value V^alpha.
    """
    n, m1, m2, _ = p.shape
    V = {}
    for alpha in itertools.product(range(m1), repeat=n):
        vals = np.array([value_of(p, r, mu, np.array(alpha), np.array(b))
                         for b in itertools.product(range(m2), repeat=n)])
        Va = vals.min(axis=0)
        # MDP theory: one stationary beta attains the componentwise minimum.
        assert np.any(np.all(np.abs(vals - Va) <= 1e-12, axis=1))
        V[alpha] = Va
    allV = np.array(list(V.values()))
    vstar = allV.max(axis=0)
    assert np.any(np.all(np.abs(allV - vstar) <= 1e-12, axis=1))
    return vstar, V


def dense_F(p, r, mu, v):
    q = mu * np.einsum("xaby,y->xab", p, v) + r
    return q.min(axis=2).max(axis=1)


# ----------------------------------------------------------------- brute force
@pytest.mark.parametrize("mu", [0.5, 0.9, 0.99])
@pytest.mark.parametrize("n", [2, 3, 4])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pi_matches_brute_force(n, mu, seed):
    p, r = tiny_dense_game(1000 * n + seed, n, 2, 2)
    vstar, V = brute_force(p, r, mu)
    game = dense_to_game(p, r, mu)
    res = oracle.policy_iteration(game)
    assert res.converged
    assert np.max(np.abs(res.v - vstar)) <= 1e-13 * max(1.0, np.max(np.abs(vstar))) * 10
    # the Shapley equation holds at the brute-force value
    assert np.max(np.abs(dense_F(p, r, mu, vstar) - vstar)) <= 1e-12
    # the returned policies are optimal: alpha attains v*, beta is MIN's best reply
    a = res.alpha.astype(int)
    assert np.allclose(V[tuple(a.tolist())], vstar, atol=1e-12)
    b = res.beta[np.arange(n), a].astype(int)
    assert np.allclose(value_of(p, r, mu, a, b), vstar, atol=1e-12)


@pytest.mark.parametrize("m1,m2", [(1, 3), (3, 1), (2, 3)])
def test_pi_matches_brute_force_uneven_actions(m1, m2):
    p, r = tiny_dense_game(77 + m1 * 10 + m2, 3, m1, m2)
    vstar, _ = brute_force(p, r, 0.9)
    res = oracle.policy_iteration(dense_to_game(p, r, 0.9))
    assert np.max(np.abs(res.v - vstar)) <= 1e-12


def test_single_action_closed_form():
    """m1 = m2 = 1: the game is a Markov chain, v = (I - mu P)^-1 r."""
    rng = np.random.default_rng(5)
    n = 40
    p, r = tiny_dense_game(5, n, 1, 1)
    mu = 0.95
    v = np.linalg.solve(np.eye(n) - mu * p[:, 0, 0, :], r[:, 0, 0])
    res = oracle.policy_iteration(dense_to_game(p, r, mu))
    assert res.outer == 1 and res.systems == 1
    assert np.max(np.abs(res.v - v)) <= 1e-12
    del rng


# ----------------------------------------------------------------- operator properties
def _random_game(n=60, seed=3, mu=0.9, k=6):
    rp, col, prob, rew, _ = synth.random_game(n, seed, k=k, mu=mu)
    return game_from_csr(n, 4, 4, rp, col, prob, rew, mu), rew


def _F(game, v):
    return shapley_q(game, v).min(axis=2).max(axis=1)


def test_shapley_monotone_contracting_homogeneous():
    game, _ = _random_game()
    rng = np.random.default_rng(0)
    for _ in range(20):
        v = rng.normal(size=game.n)
        w = v + np.abs(rng.normal(size=game.n))          # w >= v
        assert np.all(_F(game, v) <= _F(game, w) + 1e-15)
        u = rng.normal(size=game.n) * 3
        lhs = np.max(np.abs(_F(game, v) - _F(game, u)))
        assert lhs <= game.mu * np.max(np.abs(v - u)) + 1e-13
        c = rng.normal()
        # rows are stochastic: F(v + c 1) = F(v) + mu c
        assert np.max(np.abs(_F(game, v + c) - _F(game, v) - game.mu * c)) <= 1e-13


@pytest.mark.parametrize("which", ["random", "isaacs", "obstacle"])
def test_contraction_bound_and_fixed_point(which):
    if which == "random":
        game, rew = _random_game(mu=0.97)
    else:
        game = isaacs_game(15, 1 if which == "obstacle" else 0, seed=4)
        rew = game.rew
    a0 = default_alpha0(15, 1) if which == "obstacle" else None
    res = oracle.policy_iteration(game, alpha0=a0)
    assert res.converged
    assert np.max(np.abs(res.v)) <= np.max(np.abs(rew)) / (1 - game.mu) + 1e-12
    assert np.max(np.abs(_F(game, res.v) - res.v)) <= 1e-13


@pytest.mark.parametrize("which", ["random", "isaacs", "obstacle"])
def test_pi_value_sequences_monotone_and_aposteriori(which):
    """Outer values non-decreasing, inner non-increasing (Sec. 4.2); and
    |v - v*| <= |F(v) - v| / (1 - mu) for every intermediate iterate."""
    if which == "random":
        game, _ = _random_game(n=80, seed=11, mu=0.9)
        a0 = None
    else:
        var = 1 if which == "obstacle" else 0
        game = isaacs_game(15, var, seed=6)
        a0 = default_alpha0(15, var)
    res = oracle.policy_iteration(game, alpha0=a0, record=True)
    assert res.converged
    vstar = res.v
    tol = 1e-12
    for k in range(1, len(res.outer_values)):
        assert np.all(res.outer_values[k] >= res.outer_values[k - 1] - tol)
    for inner in res.inner_values:
        for j in range(1, len(inner)):
            assert np.all(inner[j] <= inner[j - 1] + tol)
    for v in res.outer_values:
        bound = np.max(np.abs(_F(game, v) - v)) / (1 - game.mu)
        assert np.max(np.abs(v - vstar)) <= bound + tol


def test_pi_terminates_and_records_counts():
    game, _ = _random_game(n=100, seed=9, mu=0.99)
    res = oracle.policy_iteration(game)
    assert res.converged and 1 <= res.outer <= 50 and res.systems >= res.outer


# ----------------------------------------------------------------- Isaacs scheme
def test_isaacs_stencil_structure():
    side = 9
    game = isaacs_game(side, 1, seed=1)
    h = 1.0 / (side + 1)
    c0 = 2 + h
    # a = +x1 (0), b = -x1 (1): drift (1, 0): upwind weight on +x1
    p = stencil_probabilities(h, 0, 1)
    assert p == pytest.approx(((0.5 + h) / c0, 0.5 / c0, 0.5 / c0, 0.5 / c0, 0.0), abs=0)
    # a = +x2 (2), b = +x1 (0): drift (-1/2, 1/2)
    p = stencil_probabilities(h, 2, 0)
    assert p == pytest.approx((0.5 / c0, (0.5 + h / 2) / c0, (0.5 + h / 2) / c0, 0.5 / c0, 0.0))
    # a == b: zero drift, the spare h/c0 is a self-transition
    p = stencil_probabilities(h, 3, 3)
    assert p == pytest.approx((0.5 / c0,) * 4 + (h / c0,))
    rows = game.prob[:, :4, :, :].sum(axis=-1)
    interior = np.zeros((side, side), bool)
    interior[1:-1, 1:-1] = True
    interior = interior.reshape(-1)
    assert np.allclose(rows[interior], 1.0, atol=1e-15)
    assert np.all(rows[~interior] < 1.0 - 0.2)          # boundary rows lose mass
    assert np.all(game.prob >= 0)
    # stop rows: no successors, reward psi
    _, x1, x2 = isaacs_geometry(side)
    assert np.all(game.succ[:, 4] == -1)
    assert np.allclose(game.rew[:, 4, 0], 0.2 - (x1 - 0.5) ** 2 - (x2 - 0.5) ** 2)
    mu, omm = discount(side)
    assert game.mu == mu and abs((1 - mu) - omm) < 1e-15


def test_isaacs_manufactured_solution_converges_O_h():
    """The scheme (decent)-(centre) is monotone and consistent: O(h) error."""
    errs = []
    for side in (15, 31, 63, 127):
        game = isaacs_game(side, 0, reward="manufactured")
        res = oracle.policy_iteration(game)
        _, x1, x2 = isaacs_geometry(side)
        u = np.sin(np.pi * x1) * np.sin(np.pi * x2)
        errs.append(np.max(np.abs(res.v - u)))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert errs[-1] < 0.02
    assert all(1.6 < q < 2.6 for q in ratios), (errs, ratios)


# ----------------------------------------------------------------- tie rule
def test_keep_current_rule():
    vals = np.array([[1.0, 1.0 + 5e-14, 0.5], [1.0, 2.0, 2.0], [3.0, 1.0, 1.0]])
    cur = np.array([0, 0, 1], np.uint8)
    amax, _ = _keep_current(vals, cur, 1e-13, True)
    assert amax.tolist() == [0, 1, 0]      # within tau: keep; else lowest optimum
    amin, _ = _keep_current(vals, cur, 1e-13, False)
    assert amin.tolist() == [2, 0, 1]


# ----------------------------------------------------------------- FAMGpi pieces
def _golden_rows(name):
    rows = [ln for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    return np.array([[float(t) for t in ln.split()] for ln in rows])


def test_interp_value_hand_example():
    out = interp_value(np.array([1.0]), 1).reshape(3, 3)
    assert np.array_equal(out, _golden_rows("fmg_interp_1to3.txt"))


def test_interp_value_copy_and_second_order():
    errs = []
    for side_c in (7, 15, 31, 63):
        side_f = 2 * side_c + 1
        _, x1c, x2c = isaacs_geometry(side_c)
        _, x1f, x2f = isaacs_geometry(side_f)
        f = lambda a, b: np.sin(np.pi * a) * np.sin(2 * np.pi * b) * np.exp(a)
        out = interp_value(f(x1c, x2c), side_c)
        grid = out.reshape(side_f, side_f)
        assert np.array_equal(grid[1::2, 1::2].reshape(-1), f(x1c, x2c))
        errs.append(np.max(np.abs(out - f(x1f, x2f))))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.3 < q < 4.7 for q in ratios), ratios


def test_interp_policy_hand_example():
    coarse = np.arange(9, dtype=np.uint8)      # 3x3 coarse grid, action = linear index
    out = interp_policy(coarse, 3).reshape(7, 7)
    # coarse points copied
    assert np.array_equal(out[1::2, 1::2].reshape(-1), coarse)
    # worked from the lowest interior member of N(x) (1-based fine (p, q) -> out[q-1, p-1]):
    assert out[0, 0] == 0        # (1,1): N = {(0,0),(1,0),(0,1),(1,1)} -> coarse (1,1)
    assert out[0, 2] == 0        # (3,1): interior members (1,1), (2,1) -> index 0
    assert out[2, 3] == 1        # (4,3): members (2,1), (2,2) -> index 1
    assert out[6, 6] == 8        # (7,7): only (3,3) is interior
    assert out[5, 6] == 8        # (7,6): members (3,3) and boundary (4,3)
    beta = np.stack([coarse, coarse + 10], axis=1)
    assert np.array_equal(interp_policy(beta, 3)[:, 1], out.reshape(-1) + 10)


def test_famg_matches_flat_value():
    """FAMGpi and flat PI reach the same (unique) value, plain and obstacle."""
    for variant in (0, 1):
        xi = synth.isaacs_noise(31, 2)
        res, levels = famg_pi(31, 3, variant, xi, c=0.1, eps=0.0)
        flat = oracle.policy_iteration(isaacs_game(31, variant, xi=xi),
                                       alpha0=default_alpha0(31, variant))
        assert np.max(np.abs(res.v - flat.v)) <= 1e-13
        assert len(levels) == 4


def test_injected_noise_positions():
    xi = np.arange(15 * 15, dtype=float)
    out = injected_noise(xi, 15, 7).reshape(7, 7)
    assert out[0, 0] == xi[1 * 15 + 1] and out[6, 6] == xi[13 * 15 + 13]


# ----------------------------------------------------------------- generators
def test_splitmix64_published_outputs():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as fh:
        want = [int(ln) for ln in fh if ln.strip() and not ln.startswith("#")]
    got = synth.splitmix64(1234567, np.arange(5, dtype=np.uint64))
    assert [int(z) for z in got] == want


def test_random_game_structure():
    n = 300
    rp, col, prob, rew, mu = synth.random_game(n, 17)
    R = n * 16
    assert rp[-1] == R * 8 and mu == 0.99
    c = col.reshape(R, 8)
    assert np.all(np.diff(c, axis=1) > 0)            # distinct, ascending
    assert c.min() >= 0 and c.max() < n
    assert np.allclose(prob.reshape(R, 8).sum(axis=1), 1.0, atol=1e-15)
    assert np.all(prob >= 0) and np.all(np.abs(rew) < 1)
    rp2, col2, prob2, rew2, _ = synth.random_game(n, 17)
    assert np.array_equal(col, col2) and np.array_equal(prob, prob2)
    # roughly uniform successor marginal
    counts = np.bincount(col, minlength=n)
    assert counts.min() > 0.6 * counts.mean() and counts.max() < 1.4 * counts.mean()


# ----------------------------------------------------------------- fixed-point evaluation
@pytest.mark.parametrize("n,seed", [(300, 11), (1000, 12), (2000, 13)])
def test_fixed_point_evaluation_matches_dense_solve(n, seed):
    """The fixed-policy iteration w <- mu M w + r (Eq. (LSPI) as a fixed point)
    stops on its step size; at mu = 0.99 that step bounds the error by
    mu/(1 - mu) times itself, so the result must sit within about 1e-12 of
    the LAPACK solution of the same system.  Random policies, random games."""
    rp, col, prob, rew, mu = synth.random_game(n, seed)
    game = game_from_csr(n, 4, 4, rp, col, prob, rew, mu)
    rng = np.random.default_rng(seed)
    alpha = rng.integers(0, 4, n).astype(np.uint8)
    beta = rng.integers(0, 4, (n, 4)).astype(np.uint8)
    A, r = oracle.policy_system(game, alpha, beta)
    w_dense = oracle.solve_policy_system(A, r, "dense")
    w_fp = oracle.solve_policy_system(A, r, "fixed_point")
    scale = np.max(np.abs(w_dense))
    assert np.max(np.abs(w_fp - w_dense)) <= 1e-12 * scale
    # and the dense solution is the fixed point: w = mu M w + r row by row
    M = (sp_identity(n) - A)
    assert np.max(np.abs(M @ w_dense + r - w_dense)) <= 1e-13 * scale


def sp_identity(n):
    import scipy.sparse as sp
    return sp.identity(n, format="csr")


def test_fixed_point_evaluation_substochastic_rows():
    """Rows that lose mass (stop actions, the Dirichlet boundary) change the
    fixed point: a two-state chain worked by hand.  State 0 moves to 1 with
    p = 1/2 (the rest leaves), state 1 stays with p = 1/4; r = (1, 2),
    mu = 0.8: w1 = 2 / (1 - 0.2) = 2.5, w0 = 1 + 0.4 * 2.5 = 2."""
    game = game_from_csr(2, 1, 1, np.array([0, 1, 2]), np.array([1, 1], np.int32),
                         np.array([0.5, 0.25]), np.array([1.0, 2.0]), 0.8)
    A, r = oracle.policy_system(game, np.zeros(2, np.uint8), np.zeros((2, 1), np.uint8))
    w = oracle.solve_policy_system(A, r, "fixed_point")
    assert abs(w[1] - 2.5) <= 1e-13 and abs(w[0] - 2.0) <= 1e-13


@pytest.mark.parametrize("mu", [0.5, 0.9, 0.99])
@pytest.mark.parametrize("n", [2, 3, 4])
def test_pi_with_fixed_point_evaluation_matches_brute_force(n, mu):
    """Whole policy iteration with the fixed-point policy evaluation (the one
    used for random games above 2000 states) against enumeration."""
    p, r = tiny_dense_game(5000 * n + int(100 * mu), n, 2, 2)
    vstar, V = brute_force(p, r, mu)
    res = oracle.policy_iteration(dense_to_game(p, r, mu), solver="fixed_point")
    assert res.converged
    # stopping on a 1e-14 step at mu = 0.99 leaves at most ~1e-12 relative
    assert np.max(np.abs(res.v - vstar)) <= 2e-12 * max(1.0, np.max(np.abs(vstar)))
    a = res.alpha.astype(int)
    assert np.allclose(V[tuple(a.tolist())], vstar, atol=1e-11)


# ----------------------------------------------------------------- gaps and rewards
def test_gap_hand_example():
    """Best minus second best over the last axis: for MAX the two largest,
    for MIN the two smallest; a tie gives 0; one action gives inf."""
    from oracle.game import _gap
    vals = np.array([[3.0, 1.0, 2.0], [5.0, 5.0, 0.0], [-1.0, 4.0, 0.5]])
    assert _gap(vals, True).tolist() == [1.0, 0.0, 3.5]
    assert _gap(vals, False).tolist() == [1.0, 5.0, 1.5]
    assert np.all(np.isinf(_gap(np.zeros((4, 1)), True)))
    # the PI result's gaps are those of F(v; x, a) over a and F(v; x, a, b) over b
    p, r = tiny_dense_game(31, 3, 2, 2)
    res = oracle.policy_iteration(dense_to_game(p, r, 0.9))
    q = 0.9 * np.einsum("xaby,y->xab", p, res.v) + r
    fa = q.min(axis=2)
    assert np.allclose(res.gap_max, np.abs(fa[:, 0] - fa[:, 1]), atol=1e-15)
    assert np.allclose(res.gap_min, np.abs(q[:, :, 0] - q[:, :, 1]), atol=1e-15)


def test_config_reward_hand_values():
    """r(x, a, b) = sin(pi x1) sin(pi x2) + 0.1 (a - b) + xi at hand-computed
    points: x = (1/2, 1/4), a = 3, b = 1, xi = 0.01 gives sqrt(2)/2 + 0.21;
    x = (1/6, 1/2), a = b = 2, xi = -0.05 gives 1/2 - 0.05."""
    from oracle.isaacs import config_reward
    assert abs(config_reward(0.5, 0.25, 3, 1, 0.01) - (np.sqrt(2) / 2 + 0.21)) <= 2e-16
    assert abs(config_reward(1 / 6, 0.5, 2, 2, -0.05) - 0.45) <= 2e-16
    assert abs(config_reward(0.5, 0.5, 0, 3, 0.0) - 0.7) <= 2e-16
    # the oracle's game carries (1 - mu) r with 1 - mu = h^2 / (1 + h^2)
    g = isaacs_game(3, 0, xi=np.zeros(9))
    h = 0.25
    x = 4                                       # centre point (1/2, 1/2)
    assert abs(g.rew[x, 1, 3] - h * h / (1 + h * h) * (1.0 - 0.2)) <= 1e-17


# ----------------------------------------------------------------- table generators
def _rows_as_sets(game):
    """{(x, a, b): (sorted successor/probability pairs, reward)} of a Game."""
    out = {}
    n, m1, m2 = game.n, game.m1, game.m2
    for x in range(n):
        for a in range(m1):
            for b in range(m2):
                pairs = sorted((int(y), float(p)) for y, p in zip(game.succ[x, a, b], game.prob[x, a, b])
                               if y >= 0 and p != 0.0)
                out[(x, a, b)] = (pairs, float(game.rew[x, a, b]))
    return out


@pytest.mark.parametrize("side,variant", [(3, 0), (7, 0), (7, 1)])
def test_isaacs_tables_are_the_oracles_game(side, variant):
    """synth's CSR tables of the Isaacs workload (input of the finite-game path)
    describe the same game as the oracle's own generator."""
    n, m1, m2, rp, col, prob, rew, mu = synth.isaacs_tables(side, variant, 5)
    ours = _rows_as_sets(game_from_csr(n, m1, m2, rp, col, prob, rew, mu))
    ref_game = isaacs_game(side, variant, seed=5)
    ref = _rows_as_sets(ref_game)
    assert abs(mu - ref_game.mu) <= 1e-16
    for key in ref:
        (pa, ra), (pb, rb) = ours[key], ref[key]
        assert [y for y, _ in pa] == [y for y, _ in pb], key
        assert np.allclose([p for _, p in pa], [p for _, p in pb], rtol=0, atol=1e-16), key
        assert abs(ra - rb) <= 1e-16 + 1e-15 * abs(rb), key


def test_two_stop_tables_are_the_oracles_game():
    from oracle.stopping1d import two_stop_game
    n, m1, m2, rp, col, prob, rew, mu = synth.two_stop_tables(17)
    ours = _rows_as_sets(game_from_csr(n, m1, m2, rp, col, prob, rew, mu))
    ref_game = two_stop_game(17)
    ref = _rows_as_sets(ref_game)
    assert mu == ref_game.mu == 1.0
    for key in ref:
        (pa, ra), (pb, rb) = ours[key], ref[key]
        assert pa == pb, key
        assert abs(ra - rb) <= 1e-15, key


# ----------------------------------------------------------------- Isaacs example with continuous actions
def test_iex1_tables_are_the_oracles_game():
    """synth's tables of the Sec. 6.1 example with discretised action sets
    (Eq. (Iex1d)) describe the oracle's game row by row."""
    from oracle.iex1 import iex1_game
    n, m1, m2, rp, col, prob, rew, mu = synth.iex1_tables(5, 4, 3)
    ours = _rows_as_sets(game_from_csr(n, m1, m2, rp, col, prob, rew, mu))
    ref_game = iex1_game(5, 4, 3)
    ref = _rows_as_sets(ref_game)
    assert mu == ref_game.mu == 1.0
    for key in ref:
        (pa, ra), (pb, rb) = ours[key], ref[key]
        assert [y for y, _ in pa] == [y for y, _ in pb], key
        assert np.allclose([p for _, p in pa], [p for _, p in pb], rtol=0, atol=1e-16), key
        assert abs(ra - rb) <= 1e-16 + 1e-14 * abs(rb), key


def test_iex1_rows_are_stochastic_up_to_the_boundary():
    """Every (a, b) row sums to one when all four neighbours are interior and
    to less near the boundary (Sec. 6.1's remark), with non-negative weights."""
    from oracle.iex1 import iex1_game
    g = iex1_game(7, 8, 5)
    tot = g.prob.sum(axis=-1)
    interior = (g.succ >= 0).all(axis=-1)
    assert np.all(g.prob >= 0)
    assert np.allclose(tot[interior], 1.0, atol=1e-15)
    assert np.all(tot[~interior] < 1.0)


def test_iex1_converges_to_the_exact_solution():
    """The discrete value approaches the paper's exact solution sin x1 sin x2
    as the grid and the action sets refine (Sec. 6.1); policy iteration needs
    a handful of MAX steps, as the paper's Table 1 reports (3 outer steps)."""
    from oracle.iex1 import iex1_game, exact_value
    errs = []
    for side, Ka, Kb in ((7, 8, 5), (15, 16, 9), (15, 32, 13)):
        res = oracle.policy_iteration(iex1_game(side, Ka, Kb))
        assert res.converged and res.outer <= 5
        h = 1.0 / (side + 1)
        idx = np.arange(side * side)
        u = exact_value((idx % side + 1) * h, (idx // side + 1) * h)
        errs.append(np.max(np.abs(res.v - u)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 3e-4, errs


@pytest.mark.parametrize("k", [1, 3, 8])
def test_random_game_recipe(k):
    """synth.random_game follows its documented counter-based recipe, which
    the device generator (gamesolve_random_game) restates: row rho's
    successors are the ranks picked by draws rho*17 + t (t < k), stepped past
    the earlier picks; its probabilities the normalised -log1p(-u) of draws
    rho*17 + 8 + t (pairwise sum for k = 8, left to right otherwise, the last
    one set to one minus the others); its reward 2u - 1 of draw rho*17 + 16.
    Recomputed here row by row in plain Python from synth.uniform01."""
    import math
    n, seed, m1, m2 = 37, 1234567, 2, 3
    rp, col, prob, rew, _ = synth.random_game(n, seed, m1=m1, m2=m2, k=k)
    assert np.array_equal(rp, np.arange(n * m1 * m2 + 1) * k)
    for rho in range(n * m1 * m2):
        base = rho * 17
        u = [float(x) for x in synth.uniform01(seed, np.arange(base, base + 17, dtype=np.uint64))]
        picks, taken = [], []
        for t in range(k):
            idx = min(int(u[t] * (n - t)), n - t - 1)
            for p in sorted(taken):
                if idx >= p:
                    idx += 1
            picks.append(idx)
            taken.append(idx)
        e = [-math.log1p(-u[8 + t]) for t in range(k)]
        if k == 8:
            tot = ((e[0] + e[1]) + (e[2] + e[3])) + ((e[4] + e[5]) + (e[6] + e[7]))
        else:
            tot = 0.0
            for x in e:
                tot += x
        p = [x / tot for x in e]
        if k > 1:
            head = 0.0
            for x in p[:-1]:
                head += x
            p[-1] = max(1.0 - head, 0.0)
        else:
            p = [1.0]
        order = sorted(range(k), key=lambda t: picks[t])
        assert list(col[rho * k:(rho + 1) * k]) == [picks[t] for t in order]
        assert np.allclose(prob[rho * k:(rho + 1) * k], [p[t] for t in order], rtol=0, atol=4e-16)
        assert rew[rho] == u[16] * 2.0 - 1.0
