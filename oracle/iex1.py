"""The Isaacs example of Sec. 6.1 (Eq. (Iex1)) with fine discretisations of its
continuous action sets (oracle generator).

TEST INFRASTRUCTURE ONLY (see the package docstring).

On the unit square, v = sin x1 sin x2 on the boundary and

    max_{|a|_2 <= 1} min_{b in R^2} ( Lap v + (a - b) . grad v - lambda v
                                       + |b|^2 / 2 + f(x) ) = 0,

with f = -(Lap u + |grad u|_2 - |grad u|^2 / 2 - lambda u) for u = sin x1 sin x2,
so that u is the exact value (the maximum over the unit ball of a . g is |g|,
the minimum over b of |b|^2/2 - b . g is -|g|^2/2).  The paper discretises it
with the upwind scheme of Eq. (Iex1d): on the interior grid (h = 1/(side+1)),
with d = a - b and c = 4 + h |d_1| + h |d_2|, the transition to the east
neighbour has probability (1 + h max(d_1, 0)) / c, to the west
(1 + h max(-d_1, 0)) / c, to the north and south likewise with d_2; the
reward is h^2 (|b|^2/2 + f(x)) / c, and a neighbour on the boundary leaves the
state space, its probability times the boundary value psi_1 moving into the
reward; lambda = 0 (as in the paper's tests) gives mu = 1.

The paper does not say how it takes the max and min over the continuous sets.
Reading (fine discretisation): MAX's actions are Ka points of the unit circle,
a_k = (cos 2 pi k/Ka, sin 2 pi k/Ka) (a linear function of a is maximised on
the boundary of the ball); MIN's actions are the Kb x Kb points of a uniform
grid over [lo, hi]^2, b index = j1 * Kb + j2 for b = (lo + j1 s, lo + j2 s).
"""
from __future__ import annotations

import numpy as np

from .game import Game


def exact_value(x1, x2):
    """u(x) = sin x1 sin x2, the exact value of Eq. (Iex1)."""
    return np.sin(x1) * np.sin(x2)


def source(x1, x2, lam: float = 0.0):
    """f = -(Lap u + |grad u|_2 - |grad u|_2^2 / 2 - lam u) for u = sin x1 sin x2."""
    u = np.sin(x1) * np.sin(x2)
    g1 = np.cos(x1) * np.sin(x2)
    g2 = np.sin(x1) * np.cos(x2)
    ng = np.sqrt(g1 * g1 + g2 * g2)
    return -(-2.0 * u + ng - 0.5 * ng * ng - lam * u)


def max_actions(Ka: int):
    """MAX's actions: Ka points of the unit circle, as an array [Ka, 2]."""
    t = 2.0 * np.pi * np.arange(Ka) / Ka
    return np.stack([np.cos(t), np.sin(t)], axis=1)


def min_actions(Kb: int, lo: float, hi: float):
    """MIN's actions: the Kb x Kb grid over [lo, hi]^2, index j1 * Kb + j2."""
    g = lo + (hi - lo) * np.arange(Kb) / (Kb - 1)
    b1, b2 = np.meshgrid(g, g, indexing="ij")
    return np.stack([b1.reshape(-1), b2.reshape(-1)], axis=1)


def iex1_game(side: int, Ka: int, Kb: int, lo: float = -0.25, hi: float = 1.25) -> Game:
    """The discretised game (Eq. (Iex1d), lambda = 0) with the action sets above.

    States x = i2 * side + i1 with coordinates ((i1+1) h, (i2+1) h); successor
    slots east, west, north, south (-1 where the neighbour is on the boundary).
    """
    h = 1.0 / (side + 1)
    n = side * side
    A = max_actions(Ka)
    B = min_actions(Kb, lo, hi)
    m1, m2 = len(A), len(B)
    idx = np.arange(n)
    i1, i2 = idx % side, idx // side
    x1, x2 = (i1 + 1) * h, (i2 + 1) * h
    f = source(x1, x2)
    steps = ((1, 0), (-1, 0), (0, 1), (0, -1))
    succ = -np.ones((n, m1, m2, 4), np.int64)
    prob = np.zeros((n, m1, m2, 4))
    rew = np.zeros((n, m1, m2))
    d1 = A[:, None, 0] - B[None, :, 0]            # [m1, m2]
    d2 = A[:, None, 1] - B[None, :, 1]
    c = 4.0 + h * np.abs(d1) + h * np.abs(d2)
    pk = [(1.0 + h * np.maximum(d1, 0.0)) / c, (1.0 + h * np.maximum(-d1, 0.0)) / c,
          (1.0 + h * np.maximum(d2, 0.0)) / c, (1.0 + h * np.maximum(-d2, 0.0)) / c]
    bb = 0.5 * (B[:, 0] ** 2 + B[:, 1] ** 2)      # [m2]
    rew[:] = (h * h / c)[None, :, :] * (bb[None, None, :] + f[:, None, None])
    for s, (s1, s2) in enumerate(steps):
        j1, j2 = i1 + s1, i2 + s2
        inside = (j1 >= 0) & (j1 < side) & (j2 >= 0) & (j2 < side)
        nb = np.where(inside, j2 * side + j1, -1)
        psi = np.sin((j1 + 1) * h) * np.sin((j2 + 1) * h)          # boundary value
        succ[:, :, :, s] = nb[:, None, None]
        prob[:, :, :, s] = np.where(inside[:, None, None], pk[s][None, :, :], 0.0)
        rew += np.where(inside, 0.0, psi)[:, None, None] * pk[s][None, :, :]
    return Game(succ, prob, rew, 1.0)
