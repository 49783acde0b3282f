"""Full multilevel policy iteration FAMGpi, Algorithm 4 (Sec. 5.2) - oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Grids: level l has side_l = 2 side_{l+1} + 1 interior points per direction and
step h_l = 2 h_{l-1}; the coarse point (I, J) (1-based) is the fine point
(2I, 2J), so X_l is a subset of X_{l-1}.

* Value interpolation I^{l-1}_l: a fine point that is also a coarse point
  keeps its value; any other fine point x takes the mean of v^l(y) over
  N(x) = { y : |x - y|_2 <= h_l }.  Reading: y ranges over the coarse grid
  points including the boundary ones, which carry the Dirichlet value 0.
* Strategy interpolation U^{l-1}_l: coarse points keep their action; a new
  fine point takes "an arbitrary" action a_0.  Reading: a_0 is the action of
  the interior coarse point of N(x) with the lowest row-major index (for
  beta, the same point's beta(., a) for every a).
* Per-level reward noise: level l's game uses the finest grid's noise at the
  points of X_l (the noise is a function on X_0 restricted to X_l).
"""
from __future__ import annotations

import numpy as np

from .game import policy_iteration
from .isaacs import isaacs_game, default_alpha0


def _neighbours(side_c: int):
    """N(x) for every fine point, as candidate arrays over a 3x3 window.

    Returns (p, q, P, Q, member, interior): the fine 1-based positions and,
    each [n_f, 9], the coarse 1-based
    positions (P, Q) of the window around (p // 2, q // 2), whether each is in
    N(x), and whether it is an interior coarse point.  Membership is decided
    exactly in units of the fine step: a coarse point sits at fine 1-based
    position (2P, 2Q) and belongs to N(x) for the fine point (p, q) when
    (p - 2P)^2 + (q - 2Q)^2 <= 4, i.e. |x - y|_2 <= h_l.  Every coarse point
    within that distance lies in the window, boundary points (P or Q equal
    to 0 or side_c + 1) included.
    """
    side_f = 2 * side_c + 1
    x = np.arange(side_f * side_f)
    p = x % side_f + 1
    q = x // side_f + 1
    off = np.array([-1, 0, 1])
    P = (p // 2)[:, None, None] + off[None, None, :]
    Q = (q // 2)[:, None, None] + off[None, :, None]
    P, Q = np.broadcast_arrays(P, Q)
    P = P.reshape(-1, 9)
    Q = Q.reshape(-1, 9)
    member = ((p[:, None] - 2 * P) ** 2 + (q[:, None] - 2 * Q) ** 2 <= 4)
    member &= (P >= 0) & (P <= side_c + 1) & (Q >= 0) & (Q <= side_c + 1)
    interior = member & (P >= 1) & (P <= side_c) & (Q >= 1) & (Q <= side_c)
    return p, q, P, Q, member, interior


def interp_value(v_c: np.ndarray, side_c: int) -> np.ndarray:
    """I^{l-1}_l v (Sec. 5.2): copy on X_l, mean over N(x) elsewhere."""
    v_c = np.asarray(v_c, dtype=np.float64)
    p, q, P, Q, member, interior = _neighbours(side_c)
    cidx = np.where(interior, (Q - 1) * side_c + (P - 1), 0)
    vals = np.where(interior, v_c[cidx], 0.0)          # boundary members carry 0
    mean = (vals * member).sum(axis=1) / member.sum(axis=1)
    on_coarse = (p % 2 == 0) & (q % 2 == 0)
    copy = v_c[np.where(on_coarse, (q // 2 - 1) * side_c + (p // 2 - 1), 0)]
    return np.where(on_coarse, copy, mean)


def interp_policy(pol_c: np.ndarray, side_c: int) -> np.ndarray:
    """U^{l-1}_l for alpha ([n_c]) or beta ([n_c, m1]) (Sec. 5.2)."""
    pol_c = np.asarray(pol_c)
    p, q, P, Q, member, interior = _neighbours(side_c)
    big = side_c * side_c
    lin = np.where(interior, (Q - 1) * side_c + (P - 1), big)
    src = lin.min(axis=1)                                # lowest interior member
    on_coarse = (p % 2 == 0) & (q % 2 == 0)
    src = np.where(on_coarse, (q // 2 - 1) * side_c + (p // 2 - 1), src)
    return pol_c[src].copy()


def level_sides(side_fine: int, side_coarse: int):
    """Sides from coarsest to finest: side_coarse, 2 side_coarse + 1, ..., side_fine."""
    sides = [side_fine]
    while sides[-1] > side_coarse:
        s = sides[-1]
        if s % 2 == 0:
            raise ValueError("sides must be 2^k - 1")
        sides.append((s - 1) // 2)
    if sides[-1] != side_coarse:
        raise ValueError("side_coarse not on the hierarchy of side_fine")
    return sides[::-1]


def injected_noise(xi_fine: np.ndarray, side_fine: int, side: int) -> np.ndarray:
    """Noise on the grid of ``side`` taken at the same points of the finest grid."""
    step = (side_fine + 1) // (side + 1)
    g = np.asarray(xi_fine).reshape(side_fine, side_fine)
    return g[step - 1::step, step - 1::step].reshape(-1).copy()


def famg_pi(side_fine: int, side_coarse: int, variant: int, xi_fine: np.ndarray,
            c: float, eps: float, solver: str = "auto", **game_kw):
    """FAMGpi, Algorithm 4: AMGpi-style PI per level to eps_l = c h_l^2, then up.

    Returns (PIResult on the finest level, list of per-level PIResults).
    """
    sides = level_sides(side_fine, side_coarse)
    alpha0 = default_alpha0(sides[0], variant)
    beta0 = None
    v0 = None
    per_level = []
    for li, side in enumerate(sides):
        xi = injected_noise(xi_fine, side_fine, side)
        game = isaacs_game(side, variant, xi=xi, **game_kw)
        h = 1.0 / (side + 1)
        last = li == len(sides) - 1
        res = policy_iteration(game, alpha0, beta0, v0, eps=eps if last else c * h * h,
                               solver=solver)
        per_level.append(res)
        if last:
            return res, per_level
        v0 = interp_value(res.v, side)
        alpha0 = interp_policy(res.alpha, side)
        beta0 = interp_policy(res.beta, side)
