"""Oracle pins on the stopping game with two optimal stoppings (Sec. 6.3,
Eq. (exVI2stop)): the game with a closed-form solution whose discretisation
errors the paper prints for every grid from 9 to 2049 points."""
import os

import numpy as np
import pytest

import oracle
from oracle import stopping1d as s1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "two_stop_errors.txt")


def printed_errors():
    rows = []
    with open(GOLDEN) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                p, einf, el2 = ln.split()
                rows.append((int(p), float(einf), float(el2)))
    return rows


def half_unit_of_last_digit(printed: float) -> float:
    """Half a unit in the third significant digit of a value printed as d.dde-XX."""
    return 0.5 * 10.0 ** (np.floor(np.log10(printed)) - 2)


def solve(points, warm=True):
    game = s1.two_stop_game(points)
    a0, b0 = s1.continuous_policies(points) if warm else (None, None)
    return game, oracle.policy_iteration(game, alpha0=a0, beta0=b0)


def test_exact_solution_solves_the_equation():
    """The closed form as transcribed: 0.5 v'' + r = 0 between the free
    boundaries, v = psi_2 / psi_1 and v' = 0 (smooth fit) at 0.09 / 0.91."""
    h = 1e-4
    x = np.linspace(0.1, 0.9, 81)
    v2 = (s1.exact_value(x + h) - 2 * s1.exact_value(x) + s1.exact_value(x - h)) / h ** 2
    assert np.max(np.abs(0.5 * v2 + s1.reward(x))) < 1e-5
    mid = lambda t: np.cos(np.pi * t) + np.pi * np.sin(0.09 * np.pi) * t + s1._C
    assert mid(0.09) == pytest.approx(s1.PSI_BAR, abs=1e-15)
    assert mid(0.91) == pytest.approx(-s1.PSI_BAR, abs=1e-15)
    for xb in (0.09, 0.91):
        assert abs((mid(xb + h) - mid(xb - h)) / (2 * h)) < 1e-7
    assert s1.PSI_BAR == pytest.approx(0.6, abs=0.01)      # "about 0.6"


def test_game_rows():
    game = s1.two_stop_game(9)
    n = game.n
    assert (game.m1, game.m2, n, game.mu) == (2, 2, 7, 1.0)
    rowsum = game.prob.sum(axis=-1)
    assert np.all(rowsum[:, :, s1.STOP] == 0) and np.all(rowsum[:, s1.STOP, :] == 0)
    cont = rowsum[:, s1.CONTINUE, s1.CONTINUE]
    assert np.all(cont[1:-1] == 1.0) and cont[0] == 0.5 and cont[-1] == 0.5


@pytest.mark.parametrize("points,e_inf,e_l2", printed_errors())
def test_printed_discretisation_errors(points, e_inf, e_l2):
    """The oracle's fixed point reproduces the paper's printed error norms to
    the digits printed (this pins the discretisation reading and the
    undiscounted stop-row policy iteration together)."""
    _, res = solve(points)
    assert res.converged and res.residual <= 1e-15
    got_inf, got_l2 = s1.error_norms(points, res.v)
    assert abs(got_inf - e_inf) <= half_unit_of_last_digit(e_inf), got_inf
    assert abs(got_l2 - e_l2) <= half_unit_of_last_digit(e_l2), got_l2


@pytest.mark.parametrize("points", [17, 33, 65])
def test_cold_start_reaches_the_same_fixed_point(points):
    """From the default policies (MAX stops everywhere) policy iteration takes
    many more steps (of the order of the grid's diameter, as the paper's flat
    AMGpi table shows) but ends at the same value: the fixed point is unique."""
    _, warm = solve(points)
    _, cold = solve(points, warm=False)
    assert cold.converged
    assert np.max(np.abs(cold.v - warm.v)) <= 1e-14
    assert cold.outer > warm.outer


def test_discrete_stopping_regions():
    """Away from the free boundaries the discrete optimal policies are the
    exact game's: MAX stops right of 0.91, MIN left of 0.09."""
    points = 257
    _, res = solve(points)
    x = s1.grid(points)
    h = 1.0 / (points - 1)
    a_ref, b_ref = s1.continuous_policies(points)
    far = (np.abs(x - 0.09) > 2 * h) & (np.abs(x - 0.91) > 2 * h)
    assert np.array_equal(res.alpha[far], a_ref[far])
    b_at_alpha = res.beta[np.arange(len(x)), res.alpha]
    assert np.array_equal(b_at_alpha[far], b_ref[far, 0])


def test_synthetic_line_data_is_the_oracle_game():
    """The C-ABI's arrays (synth.stopping_line) describe the oracle's game."""
    import synth
    points = 33
    c, p1, p2, vl, vr = synth.stopping_line(points)
    game = s1.two_stop_game(points)
    n = game.n
    assert len(c) == n
    assert np.allclose(game.rew[:, s1.STOP, s1.CONTINUE], p1, rtol=0, atol=1e-15)
    assert np.allclose(game.rew[:, s1.CONTINUE, s1.STOP], p2, rtol=0, atol=1e-15)
    cont = c.copy()
    cont[0] += 0.5 * vl
    cont[-1] += 0.5 * vr
    assert np.allclose(game.rew[:, s1.CONTINUE, s1.CONTINUE], cont, rtol=0, atol=1e-15)
