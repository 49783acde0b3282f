"""Finite-difference Isaacs game on the unit square (oracle generator).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The workload discretises

    max_a min_b ( 1/2 Lap v + beta(a,b) . grad v ) / c0 - v + r(x,a,b) = 0   on ]0,1[^2,
    v = 0 on the boundary,

with the schemes of Sec. 3.3: upwind first derivatives, Eq. (decent), and
centred second derivatives, Eq. (centre), on the interior grid of
side x side points, h = 1/(side+1), scaled to the Shapley form of Eq. (eq1)
the way Sec. 6.1 turns the Isaacs example into Eq. (Iex1d): multiply by h^2,
normalise by c0 and add v to both sides.  Readings (each also listed in the
design notes):

* actions a, b in {0,1,2,3} index the directions e_0 = +x1, e_1 = -x1,
  e_2 = +x2, e_3 = -x2, and the drift is beta(a,b) = (e_a - e_b)/2, so
  |beta|_1 is 1 when a != b and 0 when a == b;
* one normaliser c0 = 2 + h for every (a, b): the pair a == b carries the
  spare h/c0 as a self-transition, so every row sums to one before the
  boundary truncation;
* transition probabilities p(x + h e_i) = (1/2 + h max(beta_i, 0)) / c0 and
  p(x - h e_i) = (1/2 + h max(-beta_i, 0)) / c0, as in Eq. (Iex1pr);
  neighbours on the boundary are dropped (Dirichlet v = 0, Sec. 3.3), which
  leaves the boundary rows substochastic as Sec. 6.1 notes;
* discount mu = 1/(1 + h^2) ("literal"; mu_mode="exact" gives the exact
  scaling c0/(c0 + h^2)), and the discrete reward is (1 - mu) r(x, a, b)
  with 1 - mu evaluated as h^2/(1 + h^2) (resp. h^2/(c0 + h^2));
* r(x, a, b) = sin(pi x1) sin(pi x2) + 0.1 (a - b) + xi(x) with xi the
  per-state noise from ``synth.isaacs_noise``;
* obstacle variant (Sec. 3.2, Eq. (VI); discrete form of Sec. 6.2): MAX gets
  a fifth action a = 4, "stop", with no successors and reward
  psi(x) = 0.2 - |x - (0.5, 0.5)|^2, so v = max(psi, ...).
"""
from __future__ import annotations

import numpy as np

from .game import Game

DIRECTIONS = ((1, 0), (-1, 0), (0, 1), (0, -1))   # e_0..e_3 as (d i1, d i2)
STOP = 4


def isaacs_geometry(side: int):
    """(h, x1, x2) for the interior points in row-major order x = i2*side + i1."""
    h = 1.0 / (side + 1)
    idx = np.arange(side * side)
    i1 = idx % side
    i2 = idx // side
    return h, (i1 + 1) * h, (i2 + 1) * h


def discount(side: int, mu_mode: str = "literal"):
    """(mu, 1 - mu) of the scaled scheme, 1 - mu evaluated without cancellation."""
    h = 1.0 / (side + 1)
    c0 = 2.0 + h
    if mu_mode == "literal":
        return 1.0 / (1.0 + h * h), (h * h) / (1.0 + h * h)
    if mu_mode == "exact":
        return c0 / (c0 + h * h), (h * h) / (c0 + h * h)
    raise ValueError(mu_mode)


def drift(a: int, b: int):
    """beta(a, b) = (e_a - e_b) / 2 as a pair of floats."""
    ea, eb = DIRECTIONS[a], DIRECTIONS[b]
    return 0.5 * (ea[0] - eb[0]), 0.5 * (ea[1] - eb[1])


def stencil_probabilities(h: float, a: int, b: int):
    """p for the slots (+x1, -x1, +x2, -x2, self) of the pair (a, b)."""
    c0 = 2.0 + h
    b1, b2 = drift(a, b)
    return ((0.5 + h * max(b1, 0.0)) / c0,
            (0.5 + h * max(-b1, 0.0)) / c0,
            (0.5 + h * max(b2, 0.0)) / c0,
            (0.5 + h * max(-b2, 0.0)) / c0,
            (h / c0) if a == b else 0.0)


def config_reward(x1, x2, a, b, xi):
    """r(x, a, b) = sin(pi x1) sin(pi x2) + 0.1 (a - b) + xi(x)."""
    return np.sin(np.pi * x1) * np.sin(np.pi * x2) + 0.1 * (a - b) + xi


def manufactured_reward(x1, x2, a, b):
    """Reward whose continuous game has the value u = sin(pi x1) sin(pi x2).

    With L_ab u = 1/2 Lap u + beta(a,b) . grad u and the continuous-limit
    normaliser c = 2, r = u - L_ab u / 2 + 0.1 (a - b) makes u solve
    max_a min_b (L_ab v / 2 - v + r) = 0, because max_a min_b 0.1 (a - b) = 0.
    """
    u = np.sin(np.pi * x1) * np.sin(np.pi * x2)
    ux1 = np.pi * np.cos(np.pi * x1) * np.sin(np.pi * x2)
    ux2 = np.pi * np.sin(np.pi * x1) * np.cos(np.pi * x2)
    lap = -2.0 * np.pi ** 2 * u
    b1, b2 = drift(a, b)
    L = 0.5 * lap + b1 * ux1 + b2 * ux2
    return u - L / 2.0 + 0.1 * (a - b)


def obstacle(x1, x2):
    """psi(x) = 0.2 - |x - (0.5, 0.5)|^2."""
    return 0.2 - ((x1 - 0.5) ** 2 + (x2 - 0.5) ** 2)


def isaacs_game(side: int, variant: int = 0, xi=None, seed: int = 1,
                reward: str = "config", mu_mode: str = "literal") -> Game:
    """The Isaacs game as an explicit finite game (slots +x1, -x1, +x2, -x2, self).

    variant 0: plain, m1 = m2 = 4.  variant 1: obstacle, m1 = 5 (a = 4 stops).
    ``xi`` is the per-state noise (default ``synth.isaacs_noise(side, seed)``).
    """
    if xi is None:
        import synth
        xi = synth.isaacs_noise(side, seed)
    n = side * side
    h, x1, x2 = isaacs_geometry(side)
    mu, one_minus_mu = discount(side, mu_mode)
    m1 = 5 if variant == 1 else 4
    m2 = 4
    K = 5
    idx = np.arange(n)
    i1, i2 = idx % side, idx // side
    neigh = np.empty((n, K), dtype=np.int64)
    for s, (d1, d2) in enumerate(DIRECTIONS):
        j1, j2 = i1 + d1, i2 + d2
        inside = (j1 >= 0) & (j1 < side) & (j2 >= 0) & (j2 < side)
        neigh[:, s] = np.where(inside, j2 * side + j1, -1)
    neigh[:, 4] = idx
    succ = -np.ones((n, m1, m2, K), dtype=np.int64)
    prob = np.zeros((n, m1, m2, K), dtype=np.float64)
    rew = np.zeros((n, m1, m2), dtype=np.float64)
    for a in range(4):
        for b in range(4):
            p = stencil_probabilities(h, a, b)
            for s in range(K):
                if p[s] == 0.0:
                    continue
                succ[:, a, b, s] = neigh[:, s]
                prob[:, a, b, s] = np.where(neigh[:, s] >= 0, p[s], 0.0)
            if reward == "config":
                r = config_reward(x1, x2, a, b, xi)
            elif reward == "manufactured":
                r = manufactured_reward(x1, x2, a, b)
            else:
                raise ValueError(reward)
            rew[:, a, b] = one_minus_mu * r
    if variant == 1:
        rew[:, STOP, :] = obstacle(x1, x2)[:, None]
    return Game(succ, prob, rew, mu)


def default_alpha0(side: int, variant: int) -> np.ndarray:
    """Initial MAX policy: action 0, or "stop everywhere" for the obstacle (Sec. 6.2)."""
    return np.full(side * side, STOP if variant == 1 else 0, dtype=np.uint8)
