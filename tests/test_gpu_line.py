"""The two-sided stopping game on a line (Sec. 6.3) on the device, against
the oracle and the paper's printed errors.

Flat AMGpi from the default policies must follow the oracle's policy
iteration (same value, same MAX/MIN iteration counts: both solve every
system exactly); FAMGpi (Algorithm 4) must reach the same unique fixed point,
whose distance to the exact solution the paper prints for every grid from 9
to 2049 points (tests/golden/two_stop_errors.txt)."""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import stopping1d as s1

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "two_stop_errors.txt")


def printed():
    rows = []
    with open(GOLDEN) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                p, ei, el = ln.split()
                rows.append((int(p), float(ei), float(el)))
    return rows


def gpu_solve(gs, points, fmg, **opts):
    c, p1, p2, vl, vr = synth.stopping_line(points)
    with gs.GameSolver(fmg=fmg, fmg_c=1e-2, **opts) as s:
        s.set_stopping_line(c, p1, p2, vl, vr)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    return v, a, b, st


@pytest.mark.parametrize("points", [9, 17, 33, 65, 129, 2049])
def test_flat_amgpi_follows_the_oracle(gs, points):
    """(2049 points: two states per thread of the block.)"""
    game = s1.two_stop_game(points)
    ref = oracle.policy_iteration(game)
    v, a, b, st = gpu_solve(gs, points, fmg=0)
    assert st["converged"] == 1
    assert np.max(np.abs(v - ref.v)) <= 1e-12
    assert (st["outer"], st["systems"]) == (ref.outer, ref.systems)
    sure = ref.gap_max > 1e-8
    assert np.array_equal(a[sure], ref.alpha[sure])


@pytest.mark.parametrize("points,e_inf,e_l2", printed())
def test_famgpi_reaches_the_printed_errors(gs, points, e_inf, e_l2):
    v, a, b, st = gpu_solve(gs, points, fmg=1, eps=1e-10)
    assert st["converged"] == 1
    a0, b0 = s1.continuous_policies(points)
    ref = oracle.policy_iteration(s1.two_stop_game(points), alpha0=a0, beta0=b0)
    assert np.max(np.abs(v - ref.v)) <= 1e-10 * np.max(np.abs(ref.v))
    got_inf, got_l2 = s1.error_norms(points, v)
    half = lambda x: 0.5 * 10.0 ** (np.floor(np.log10(x)) - 2)
    assert abs(got_inf - e_inf) <= half(e_inf) and abs(got_l2 - e_l2) <= half(e_l2)


def test_famgpi_is_far_cheaper_than_flat(gs):
    """The paper's point for this game (Sec. 6.3): flat AMGpi needs MAX policy
    iterations of the order of the grid's diameter (each moves MAX's stopping
    boundary by about one point), FAMGpi a few per grid.  (With MIN's inner
    loop started from its best reply, the inner loops take one or two systems
    each, not the hundreds of the paper's table.)"""
    points = 257
    _, _, _, flat = gpu_solve(gs, points, fmg=0)
    _, _, _, fmg = gpu_solve(gs, points, fmg=1, eps=1e-10)
    assert flat["outer"] >= 50 and fmg["fmg_levels"] == 8
    assert fmg["systems"] * 4 < flat["systems"]


def test_line_validation(gs):
    c, p1, p2, vl, vr = synth.stopping_line(9)
    with gs.GameSolver() as s:
        with pytest.raises(gs.GameSolveError):
            s.set_stopping_line(c[:6], p1[:6], p2[:6], vl, vr)      # n = 6 is not 2^k - 1
        bad = p1.copy()
        bad[3] = 1.0                                                # psi1 > psi2
        with pytest.raises(gs.GameSolveError):
            s.set_stopping_line(c, bad, p2, vl, vr)
        s.set_stopping_line(c, p1, p2, vl, vr)
        assert s.solve()["converged"] == 1
