"""The stopping game with two optimal stoppings, Sec. 6.3, Eq. (exVI2stop) (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

On X = [0, 1] either player may stop the diffusion dX = dW: if MAX stops
first it receives psi_1, if MIN stops (also when both stop at once) MAX
receives psi_2, and until then MAX earns the running reward
r(x) = 0.5 pi^2 cos(pi x).  The value solves
    max{psi_1 - v, min{psi_2 - v, 0.5 v'' + r}} = 0,
with psi_1 = -psi_bar, psi_2 = psi_bar and
psi_bar = (2 cos(0.09 pi) + pi (0.18 - 1) sin(0.09 pi)) / 2 (about 0.6).  The
paper gives the exact solution: psi_2 left of 0.09, psi_1 right of 0.91 and
cos(pi x) + pi sin(0.09 pi) x + c in between, c = psi_bar - cos(0.09 pi)
- 0.09 pi sin(0.09 pi) (smooth fit at both free boundaries).

Discretisation (the reading that reproduces the paper's tables, Sec. 6.3):
a grid of m + 1 points x_i = i h, h = 1/m; the states are the m - 1 interior
points; the end points hold the stop values v(0) = psi_2 and v(1) = psi_1.
Actions are 0 = stop and 1 = continue for both players, so the game has
m1 = m2 = 2 and, per state x,
  * (a, b = 0): MIN stops, a stop row with reward psi_2;
  * (a = 0, b = 1): MAX stops, a stop row with reward psi_1;
  * (a = 1, b = 1): both continue; the central difference of 0.5 v'' gives
    v(x) = v(x - h)/2 + v(x + h)/2 + h^2 r(x), undiscounted (mu = 1); an end
    point's value moves into the reward and its probability leaves the
    state space.
Every pair of policies stops the chain or lets it reach an end point with
probability one, so every policy-fixed system (Eq. (LSPI)) is nonsingular.
"""
from __future__ import annotations

import numpy as np

from .game import Game

STOP, CONTINUE = 0, 1
_C9 = np.cos(0.09 * np.pi)
_S9 = np.sin(0.09 * np.pi)
PSI_BAR = (2.0 * _C9 + np.pi * (0.18 - 1.0) * _S9) / 2.0
_C = PSI_BAR - _C9 - 0.09 * np.pi * _S9


def reward(x):
    """Running reward r(x) = 0.5 pi^2 cos(pi x) of Eq. (exVI2stop)."""
    return 0.5 * np.pi ** 2 * np.cos(np.pi * np.asarray(x, np.float64))


def exact_value(x):
    """The paper's exact (viscosity) solution of Eq. (exVI2stop)."""
    x = np.asarray(x, np.float64)
    v = np.cos(np.pi * x) + np.pi * _S9 * x + _C
    v = np.where(x < 0.09, PSI_BAR, v)
    return np.where(x > 1.0 - 0.09, -PSI_BAR, v)


def grid(points: int):
    """Interior points x_1..x_{m-1} of the grid with `points` = m + 1 points."""
    m = points - 1
    return np.arange(1, m) / m


def two_stop_game(points: int) -> Game:
    """The discretised game on a grid of `points` points (2^k + 1 in the paper)."""
    if points < 3:
        raise ValueError("need at least 3 grid points")
    m = points - 1
    h = 1.0 / m
    n = m - 1
    x = grid(points)
    succ = -np.ones((n, 2, 2, 2), np.int64)
    prob = np.zeros((n, 2, 2, 2))
    rew = np.zeros((n, 2, 2))
    rew[:, :, STOP] = PSI_BAR                 # MIN stops (wins a simultaneous stop)
    rew[:, STOP, CONTINUE] = -PSI_BAR         # MAX stops alone
    cont = h * h * reward(x)
    for i in range(n):
        k = 0
        for j, end_value in ((i - 1, PSI_BAR), (i + 1, -PSI_BAR)):
            if 0 <= j < n:
                succ[i, CONTINUE, CONTINUE, k] = j
                prob[i, CONTINUE, CONTINUE, k] = 0.5
                k += 1
            else:
                cont[i] += 0.5 * end_value
    rew[:, CONTINUE, CONTINUE] = cont
    return Game(succ=succ, prob=prob, rew=rew, mu=1.0)


def continuous_policies(points: int):
    """The exact game's optimal stopping regions on the grid: MAX stops right of
    0.91, MIN left of 0.09 (alpha, and beta(x, a) for both a)."""
    x = grid(points)
    alpha = np.where(x > 1.0 - 0.09, STOP, CONTINUE).astype(np.uint8)
    b = np.where(x < 0.09, STOP, CONTINUE).astype(np.uint8)
    return alpha, np.stack([b, b], axis=1)


def error_norms(points: int, v):
    """|e|_inf and the root mean square of e = v - exact over the interior points."""
    e = np.asarray(v) - exact_value(grid(points))
    return float(np.max(np.abs(e))), float(np.sqrt(np.mean(e * e)))
