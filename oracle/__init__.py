"""Plain FP64 CPU oracle for policy iteration on discounted zero-sum games.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path; both take their seeded inputs from ``synth``.

What it computes (Akian & Detournay, "Multigrid methods for two-player
zero-sum stochastic games"):

* the Shapley operator F(v; x, a, b), F(v; x, a), F(v; x) of Eq. (eq1) and
  Eq. (ILPI), Sec. 2;
* the policy-fixed linear system (I - mu M^{alpha beta}) v = r^{alpha beta}
  of Eq. (LSPI), Sec. 4.2, solved directly (dense or sparse LU) or by the
  fixed-policy fixed-point iteration for random games;
* Hoffman-Karp / Puri policy iteration, Algorithm 2 with Algorithm 1 as its
  inner loop (Sec. 4.1-4.2), with the stopping rule of Sec. 5.1;
* the finite-difference Isaacs game of Sec. 3.3, schemes (decent)-(centre),
  scaled to the Shapley form as in Sec. 6.1, Eq. (Iex1d), and its obstacle
  (optimal-stopping) variant of Sec. 3.2 / Sec. 6.2;
* the full multilevel policy iteration FAMGpi, Algorithm 4 (Sec. 5.2), with
  the value interpolation I and the strategy interpolation U;
* the undiscounted stopping game with two optimal stoppings of Sec. 6.3,
  Eq. (exVI2stop), and its closed-form solution (``stopping1d``).

Parity pins (tests/test_oracle_*.py): brute-force enumeration of all pure
stationary policy pairs on tiny games, the closed form (I - mu P)^-1 r for
single-action games, the contraction bound, monotonicity and
additive homogeneity of F, monotone PI value sequences, the a-posteriori
error bound, O(h) convergence to a manufactured Isaacs solution, and the
paper's printed discretisation errors of the Sec. 6.3 game on every grid from
9 to 2049 points.
"""
from .game import (Game, shapley_q, improve, policy_system, solve_policy_system,
                   policy_iteration, PIResult, tie_tolerance, game_from_csr)
from .isaacs import isaacs_game, isaacs_geometry
from .fmg import interp_value, interp_policy, famg_pi
from . import stopping1d

__all__ = [
    "Game", "shapley_q", "improve", "policy_system", "solve_policy_system",
    "policy_iteration", "PIResult", "tie_tolerance", "game_from_csr",
    "isaacs_game", "isaacs_geometry", "interp_value", "interp_policy", "famg_pi",
    "stopping1d",
]
