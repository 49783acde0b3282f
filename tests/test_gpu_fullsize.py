"""Full-size parity on the 1023 x 1023 Isaacs workload (the benchmark's), seed 2.

The FP64 oracle solves the same game with sparse LU (a few minutes on one
core); the GPU runs in the launch configuration bench.py times.  Checked:
the value (1e-10 relative FP64 path, 1e-9 mixed paths), the policies where
the oracle's max-min gap exceeds 1e-8, and, from the oracle's own Shapley
operator at every state, that the GPU value is a fixed point of Eq. (eq1).
"""
import numpy as np
import pytest

import oracle
from bench import ISAACS_CYCLE
from oracle.isaacs import isaacs_game

pytestmark = pytest.mark.gpu

SIDE, SEED = 1023, 2


@pytest.fixture(scope="module")
def reference():
    game = isaacs_game(SIDE, 0, seed=SEED)
    return game, oracle.policy_iteration(game)


@pytest.mark.parametrize("prec,fmg,cycle", [("fp64", 0, {}), ("mixed", 0, {}), ("mixed", 1, {}),
                                            ("mixed_bf16", 0, {}), ("mixed", 0, ISAACS_CYCLE),
                                            ("fp64", 0, ISAACS_CYCLE)])
def test_isaacs_1023_parity(gs, reference, prec, fmg, cycle):
    """The default V(1,1) cycles and the benchmark's cycle options."""
    game, ref = reference
    with gs.GameSolver(precision=prec, fmg=fmg, fmg_side=31, **cycle) as s:
        s.set_isaacs_grid(SIDE, 0, SEED)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    err = np.max(np.abs(v - ref.v)) / np.max(np.abs(ref.v))
    assert err <= (1e-10 if prec == "fp64" else 1e-9), (err, st)
    sure_a = ref.gap_max > 1e-8
    assert np.array_equal(a[sure_a], ref.alpha[sure_a])
    sure_b = ref.gap_min > 1e-8
    assert np.array_equal(b[sure_b], ref.beta[sure_b])
    # the oracle's Shapley operator at every state: F(v) = v up to rounding and
    # the keep-current tie tolerance
    q = oracle.shapley_q(game, v)
    fv = q.min(axis=2).max(axis=1)
    assert np.max(np.abs(fv - v)) <= 1e-12
