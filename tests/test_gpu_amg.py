"""Algebraic multigrid for finite games given as CSR tables (options.game_solver
= 1; Sec. 4.3): strength of connection, C/F splitting (PMIS, or PMIS with the
Ruge-Stueben second pass), direct interpolation, Galerkin coarse operators,
V-cycles with C/F relaxation, rebuilt for every policy-fixed system.

Checked against the FP64 oracle on structured games given as tables: the
Isaacs workload (a 2-D grid) and the Sec. 6.3 stopping game on a line
(undiscounted, mu = 1), value to 1e-10 (float64) / 1e-9 (mixed), policies
where the oracle's gap exceeds 1e-8; the cycles per system stay bounded as
the grid grows.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.game import game_from_csr
from oracle.isaacs import default_alpha0

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-9}
_ORACLE = {}


def oracle_of(key, tables, alpha0=None):
    if key not in _ORACLE:
        n, m1, m2, rp, col, prob, rew, mu = tables
        game = game_from_csr(n, m1, m2, rp, col, prob, rew, mu)
        _ORACLE[key] = oracle.policy_iteration(game, alpha0=alpha0)
    return _ORACLE[key]


def solve_tables(gs, tables, **opts):
    n, m1, m2, rp, col, prob, rew, mu = tables
    with gs.GameSolver(game_solver=1, **opts) as s:
        s.set_game(n, m1, m2, rp, col, prob, rew, mu)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    return v, a, b, st


def check(v, a, b, ref, tol):
    scale = max(np.max(np.abs(ref.v)), 1e-300)
    assert np.max(np.abs(v - ref.v)) <= tol * scale, np.max(np.abs(v - ref.v)) / scale
    sure = ref.gap_max > 1e-8
    assert np.array_equal(a[sure], ref.alpha[sure])
    m = min(b.shape[1], ref.beta.shape[1])
    sure_b = ref.gap_min[:, :m] > 1e-8
    assert np.array_equal(b[:, :m][sure_b], ref.beta[:, :m][sure_b])


@pytest.mark.parametrize("coarsening", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("side", [15, 63])
def test_isaacs_as_tables_matches_oracle(gs, side, prec, coarsening):
    tables = synth.isaacs_tables(side, 0, 3)
    ref = oracle_of(("isaacs", side), tables)
    v, a, b, st = solve_tables(gs, tables, precision=prec, amg_coarsening=coarsening)
    assert st["converged"] == 1 and st["levels"] >= 2
    check(v, a, b, ref, TOL[prec])


def test_isaacs_obstacle_as_tables_matches_oracle(gs):
    side = 31
    tables = synth.isaacs_tables(side, 1, 4)
    ref = oracle_of(("obstacle", side), tables, alpha0=default_alpha0(side, 1))
    v, a, b, st = solve_tables(gs, tables, precision="mixed")
    assert st["converged"] == 1
    check(v, a, b, ref, TOL["mixed"])


@pytest.mark.parametrize("points", [65, 513, 2049])
def test_stopping_line_as_tables_matches_oracle(gs, points):
    """The undiscounted chain of Sec. 6.3 (mu = 1): the paper's own AMGpi
    example with a genuinely one-dimensional hierarchy."""
    tables = synth.two_stop_tables(points)
    ref = oracle_of(("line", points), tables)
    v, a, b, st = solve_tables(gs, tables, precision="fp64", amg_coarsening=1,
                               max_outer=100000, max_inner=100000)
    assert st["converged"] == 1
    check(v, a, b, ref, 1e-10)


def test_cycles_per_system_bounded(gs):
    """Cycles per linear system stay bounded as the grid grows (the paper's
    tables report size-independent counts): PMIS splitting with extended+i
    interpolation, the default."""
    per = []
    for side in (63, 127, 255, 511):
        tables = synth.isaacs_tables(side, 0, 2)
        _, _, _, st = solve_tables(gs, tables, precision="mixed", pi_rtol=0.0)
        assert st["converged"] == 1
        per.append(st["cycles"] / st["systems"])
    assert max(per) <= 2.5 * per[0] + 2, per


def test_amg_rejects_undiscounted_without_it(gs):
    n, m1, m2, rp, col, prob, rew, mu = synth.two_stop_tables(17)
    with gs.GameSolver() as s:
        with pytest.raises(gs.GameSolveError) as e:
            s.set_game(n, m1, m2, rp, col, prob, rew, mu)
        assert e.value.status == gs.GS_EINVAL


@pytest.mark.parametrize("points", [513, 2049])
def test_algebraic_famg_on_the_stopping_line(gs, points):
    """Full multilevel policy iteration for a game given only by its tables
    (options.fmg with game_solver 1): coarse games by aggregation, AMGpi from
    the coarsest up.  It reaches the oracle's value (the fixed point is
    unique), and the finest level needs far fewer MAX iterations than flat
    AMGpi (the paper's FAMGpi effect, Sec. 6.3, without a PDE)."""
    tables = synth.two_stop_tables(points)
    ref = oracle_of(("line", points), tables)
    kw = dict(precision="fp64", max_outer=100000, max_inner=100000)
    v, a, b, st = solve_tables(gs, tables, fmg=1, **kw)
    assert st["converged"] == 1 and st["fmg_levels"] >= 3
    check(v, a, b, ref, 1e-10)
    _, _, _, flat = solve_tables(gs, tables, fmg=0, **kw)
    assert st["outer"] * 4 <= flat["outer"], (st, flat)


def test_algebraic_famg_on_the_obstacle_grid(gs):
    side = 63
    tables = synth.isaacs_tables(side, 1, 4)
    ref = oracle_of(("obstacle", side), tables, alpha0=default_alpha0(side, 1))
    v, a, b, st = solve_tables(gs, tables, fmg=1, precision="mixed")
    assert st["converged"] == 1 and st["fmg_levels"] >= 2
    check(v, a, b, ref, TOL["mixed"])
    n, m1, m2, rp, col, prob, rew, mu = tables
    with gs.GameSolver(game_solver=1, fmg=1, precision="mixed") as s:
        s.set_game(n, m1, m2, rp, col, prob, rew, mu)
        s.solve()
        lv = s.level_stats()
    assert lv[-1][0] == n and all(lv[k][0] < lv[k + 1][0] for k in range(len(lv) - 1))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("side", [15, 31])
def test_continuous_action_isaacs_matches_oracle(gs, side, prec):
    """The Isaacs example of Sec. 6.1 with continuous action sets (NEXT-3),
    read as fine discretisations of them (16 directions on MAX's unit circle,
    a 9 x 9 grid of MIN's b), undiscounted (lambda = 0): the tables path with
    algebraic multigrid against the oracle's own generator and policy
    iteration."""
    from oracle.iex1 import iex1_game
    key = ("iex1", side)
    if key not in _ORACLE:
        _ORACLE[key] = oracle.policy_iteration(iex1_game(side, 16, 9))
    ref = _ORACLE[key]
    v, a, b, st = solve_tables(gs, synth.iex1_tables(side, 16, 9), precision=prec)
    assert st["converged"] == 1 and st["outer"] == ref.outer
    check(v, a, b, ref, TOL[prec])


def test_continuous_action_isaacs_algebraic_famg(gs):
    """Algebraic FAMGpi on the continuous-action example (63 x 63, mu = 1):
    its aggregated coarse games average up to 16 x 81 rows whose successors
    can all fall in one aggregate (a probability one ulp above 1 before the
    clamp); it reaches the fixed point of flat AMGpi."""
    tables = synth.iex1_tables(63, 16, 9)
    v0, _, _, st0 = solve_tables(gs, tables, precision="mixed")
    v1, _, _, st1 = solve_tables(gs, tables, precision="mixed", fmg=1)
    assert st0["converged"] == 1 and st1["converged"] == 1
    assert np.max(np.abs(v1 - v0)) <= 1e-9 * np.max(np.abs(v0))


def test_continuous_action_isaacs_approaches_the_exact_solution(gs):
    """On finer grids (and a finer MIN grid) the GPU value approaches the
    paper's exact solution sin x1 sin x2 (Sec. 6.1)."""
    from oracle.iex1 import exact_value
    errs = []
    for side, Ka, Kb in ((31, 16, 9), (63, 32, 13)):
        v, _, _, st = solve_tables(gs, synth.iex1_tables(side, Ka, Kb), precision="mixed")
        assert st["converged"] == 1
        h = 1.0 / (side + 1)
        idx = np.arange(side * side)
        errs.append(np.max(np.abs(v - exact_value((idx % side + 1) * h, (idx // side + 1) * h))))
    assert errs[1] < errs[0] < 3e-4, errs
