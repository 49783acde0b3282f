"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module draws random numbers and lays them out; it holds none of the
solver's arithmetic (no Shapley operator, no policy iteration, no multigrid).
Both sides of every parity test take their inputs from here, or, for the
Isaacs per-state noise that the C-ABI can also generate from a seed, each side
implements the same counter-based generator (SplitMix64) from its published
definition and the tests check that the two agree bit for bit.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the i-th output (i = 0, 1, ...) of the stream with
seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15 mod 2^64), where mix is the
variant-13 finaliser of MurmurHash3 with shifts (30, 27, 31).  A double in
[0, 1) takes the top 53 bits: (z >> 11) * 2^-53.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = float(2.0 ** -53)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Outputs number ``counters`` (0-based, uint64 array) of the stream ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    z = splitmix64(seed, counters)
    return (z >> np.uint64(11)).astype(np.float64) * _TWO_M53


def isaacs_noise(side: int, seed: int) -> np.ndarray:
    """Per-state reward noise xi(x) ~ U(-0.05, 0.05) of the Isaacs workload.

    One draw per interior grid point, in row-major state order
    x = i2 * side + i1 (i1 along the first coordinate), drawn from the stream
    ``seed``: xi = 0.1 * u - 0.05 with u the x-th uniform.  Returned as a
    float64 array of length side*side.
    """
    n = side * side
    u = uniform01(seed, np.arange(n, dtype=np.uint64))
    return u * 0.1 - 0.05


DRAWS_PER_ROW = 17  # 8 successor draws, 8 exponential draws, 1 reward draw


def random_game(n: int, seed: int, m1: int = 4, m2: int = 4, k: int = 8,
                mu: float = 0.99, rows=None):
    """A random finite discounted game in the C-ABI's CSR layout.

    Rows are indexed (x * m1 + a) * m2 + b.  Each row has ``k`` distinct
    successors drawn uniformly from {0..n-1} (the state itself allowed),
    with Dirichlet(1) probabilities (normalised Exp(1) draws, the last drawn
    entry set to one minus the others) and a reward U(-1, 1).  Within a row
    the successors are stored in increasing column order.

    Row rho uses counters rho*17 .. rho*17+16 of the stream ``seed``: draws
    0..k-1 pick the successors (sampling without replacement by rank
    adjustment), draws 8..8+k-1 the exponentials, draw 16 the reward.

    Returns (row_ptr int64[R+1], col int32[R*k], prob float64[R*k],
    reward float64[R], mu) with R = n*m1*m2.  ``rows=(r0, r1)`` draws only
    those rows (the same values as the whole game's), with row_ptr from 0.
    """
    if not (1 <= k <= 8) or k > n:
        raise ValueError("need 1 <= k <= min(8, n)")
    r0, r1 = (0, n * m1 * m2) if rows is None else rows
    R = r1 - r0
    base = np.arange(r0, r1, dtype=np.uint64) * np.uint64(DRAWS_PER_ROW)
    picks = np.empty((R, k), dtype=np.int64)
    for t in range(k):
        u = uniform01(seed, base + np.uint64(t))
        idx = np.minimum((u * (n - t)).astype(np.int64), n - t - 1)
        if t:
            prev = np.sort(picks[:, :t], axis=1)
            for s in range(t):          # shift past each earlier pick, ascending
                idx = idx + (idx >= prev[:, s])
        picks[:, t] = idx
    e = np.empty((R, k), dtype=np.float64)
    for t in range(k):
        u = uniform01(seed, base + np.uint64(8 + t))
        e[:, t] = -np.log1p(-u)
    tot = e.sum(axis=1, keepdims=True)
    p = e / tot
    if k > 1:
        p[:, k - 1] = np.maximum(1.0 - p[:, : k - 1].sum(axis=1), 0.0)
    else:
        p[:, 0] = 1.0
    reward = uniform01(seed, base + np.uint64(16)) * 2.0 - 1.0
    order = np.argsort(picks, axis=1, kind="stable")
    col = np.take_along_axis(picks, order, axis=1).astype(np.int32)
    prob = np.take_along_axis(p, order, axis=1)
    row_ptr = np.arange(R + 1, dtype=np.int64) * k
    return row_ptr, col.reshape(-1), prob.reshape(-1), reward, float(mu)


def batch_game_sizes(count: int, seed: int, nmin: int = 256, nmax: int = 8192) -> np.ndarray:
    """Sizes n_i ~ U{nmin..nmax} of a batch of random games (stream ``seed``)."""
    u = uniform01(seed, np.arange(count, dtype=np.uint64))
    return nmin + np.minimum((u * (nmax - nmin + 1)).astype(np.int64), nmax - nmin)


def batch_game_seed(seed: int, i: int) -> int:
    """Stream of game i of a batch: SplitMix64 seeded with seed XOR i."""
    return (seed ^ i) & 0xFFFFFFFFFFFFFFFF


def _batch_part(args):
    """Worker: games [g0, g1) of a batch (module level so a spawn pool can run it)."""
    sizes, seed, g0, g1, m1, m2, k, mu = args
    out = []
    for g in range(g0, g1):
        _, col, prob, rew, _ = random_game(int(sizes[g]), batch_game_seed(seed, g), m1, m2, k, mu)
        out.append((col, prob, rew))
    return g0, out


def random_game_batch(sizes, seed: int, m1: int = 4, m2: int = 4, k: int = 8,
                      mu: float = 0.99, workers: int = 0):
    """A batch of random games (game g from the stream seed XOR g) in the
    concatenated CSR layout of gamesolve_set_game_batch.

    Returns (state_offsets, row_ptr, col, prob, reward, mu_per_game).  With
    workers > 1 the games are drawn by a spawn-context process pool; the
    result is identical to the serial one.
    """
    import multiprocessing as mp
    sizes = np.asarray(sizes, dtype=np.int64)
    count = len(sizes)
    R = sizes * m1 * m2
    row_off = np.concatenate([[0], np.cumsum(R)]).astype(np.int64)
    total_rows = int(row_off[-1])
    col = np.empty(total_rows * k, np.int32)
    prob = np.empty(total_rows * k, np.float64)
    reward = np.empty(total_rows, np.float64)

    def place(g, parts):
        for j, (c, p, r) in enumerate(parts):
            a, b = row_off[g + j], row_off[g + j + 1]
            col[a * k:b * k] = c
            prob[a * k:b * k] = p
            reward[a:b] = r

    chunk = max(1, count // max(1, 4 * max(1, workers)))
    tasks = [(sizes, seed, g, min(count, g + chunk), m1, m2, k, mu) for g in range(0, count, chunk)]
    if workers and workers > 1 and count > 1:
        with mp.get_context("spawn").Pool(workers) as pool:
            for g0, parts in pool.imap_unordered(_batch_part, tasks):
                place(g0, parts)
    else:
        for t in tasks:
            g0, parts = _batch_part(t)
            place(g0, parts)
    row_ptr = np.arange(total_rows + 1, dtype=np.int64) * k
    st_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return st_off, row_ptr, col, prob, reward, np.full(count, float(mu))


def _rows_part(args):
    n, seed, r0, r1, m1, m2, k, mu = args
    _, col, prob, rew, _ = random_game(n, seed, m1, m2, k, mu, rows=(r0, r1))
    return r0, col, prob, rew


def random_game_parallel(n: int, seed: int, m1: int = 4, m2: int = 4, k: int = 8,
                         mu: float = 0.99, workers: int = 0):
    """random_game drawn by row ranges in a spawn-context process pool (same result)."""
    import multiprocessing as mp
    R = n * m1 * m2
    if not workers or workers < 2:
        return random_game(n, seed, m1, m2, k, mu)
    col = np.empty(R * k, np.int32)
    prob = np.empty(R * k, np.float64)
    reward = np.empty(R, np.float64)
    step = max(1, -(-R // (4 * workers)))
    tasks = [(n, seed, r, min(R, r + step), m1, m2, k, mu) for r in range(0, R, step)]
    with mp.get_context("spawn").Pool(workers) as pool:
        for r0, c, p, rw in pool.imap_unordered(_rows_part, tasks):
            col[r0 * k:r0 * k + len(c)] = c
            prob[r0 * k:r0 * k + len(p)] = p
            reward[r0:r0 + len(rw)] = rw
    return np.arange(R + 1, dtype=np.int64) * k, col, prob, reward, float(mu)


def stopping_line(points: int):
    """Data of the two-sided stopping game of Sec. 6.3 on a grid of `points`
    points over [0, 1] (h = 1/(points-1)), in the C-ABI's form for the n =
    points - 2 interior points: the continuation reward c = h^2 r(x) with
    r(x) = 0.5 pi^2 cos(pi x), MAX's stop value psi1 = -psi_bar and MIN's
    psi2 = psi_bar, psi_bar = (2 cos(0.09 pi) + pi (0.18 - 1) sin(0.09 pi)) / 2,
    and the end values v(0) = psi2, v(1) = psi1.

    Returns (c, psi1, psi2, v_left, v_right).  (Deterministic problem data;
    the game itself is solved elsewhere.)
    """
    m = points - 1
    h = 1.0 / m
    x = np.arange(1, m) * h
    psi_bar = (2.0 * np.cos(0.09 * np.pi) + np.pi * (0.18 - 1.0) * np.sin(0.09 * np.pi)) / 2.0
    c = h * h * 0.5 * np.pi ** 2 * np.cos(np.pi * x)
    n = m - 1
    return c, np.full(n, -psi_bar), np.full(n, psi_bar), float(psi_bar), float(-psi_bar)


def isaacs_tables(side: int, variant: int, seed: int):
    """The finite-difference Isaacs workload written out as explicit CSR
    transition tables (the C-ABI's gamesolve_set_game layout), so that the
    general finite-game path can be run on it.  Problem data only: the grid,
    the upwind stencil probabilities and the rewards of the workload's
    definition (interior side x side, h = 1/(side+1), directions
    0:+x1 1:-x1 2:+x2 3:-x2, drift (e_a - e_b)/2, normaliser 2 + h, neighbours
    on the boundary dropped, mu = 1/(1+h^2), reward (1 - mu)(sin pi x1 sin pi x2
    + 0.1(a - b) + xi) with xi from isaacs_noise; variant 1 adds MAX's stop
    action a = 4 with no successors and reward 0.2 - |x - (1/2,1/2)|^2).

    Returns (n, m1, m2, row_ptr, col, prob, reward, mu); row (x*m1 + a)*m2 + b.
    """
    h = 1.0 / (side + 1)
    c0 = 2.0 + h
    mu = 1.0 / (1.0 + h * h)
    kappa = (h * h) / (1.0 + h * h)
    n = side * side
    m1, m2 = (5 if variant == 1 else 4), 4
    xi = isaacs_noise(side, seed)
    steps = ((1, 0), (-1, 0), (0, 1), (0, -1))
    row_ptr = [0]
    cols, probs, rews = [], [], []
    for x in range(n):
        i1, i2 = x % side, x // side
        x1, x2 = (i1 + 1) * h, (i2 + 1) * h
        base = np.sin(np.pi * x1) * np.sin(np.pi * x2) + xi[x]
        for a in range(m1):
            for b in range(m2):
                if a == 4:
                    rews.append(0.2 - ((x1 - 0.5) ** 2 + (x2 - 0.5) ** 2))
                    row_ptr.append(len(cols))
                    continue
                d1 = 0.5 * (steps[a][0] - steps[b][0])
                d2 = 0.5 * (steps[a][1] - steps[b][1])
                for (s1, s2), drift in (((1, 0), d1), ((-1, 0), -d1), ((0, 1), d2), ((0, -1), -d2)):
                    j1, j2 = i1 + s1, i2 + s2
                    if 0 <= j1 < side and 0 <= j2 < side:
                        cols.append(j2 * side + j1)
                        probs.append((0.5 + h * max(drift, 0.0)) / c0)
                if a == b:
                    cols.append(x)
                    probs.append(h / c0)
                rews.append(kappa * (base + 0.1 * (a - b)))
                row_ptr.append(len(cols))
    return (n, m1, m2, np.array(row_ptr, np.int64), np.array(cols, np.int32),
            np.array(probs, np.float64), np.array(rews, np.float64), mu)


def two_stop_tables(points: int):
    """The two-sided stopping game of Sec. 6.3 on `points` grid points as
    explicit CSR tables (gamesolve_set_game layout, undiscounted: mu = 1):
    n = points - 2 interior states, actions 0 = stop, 1 = continue for both
    players; (a, b = 0): MIN stops, reward psi_bar; (a = 0, b = 1): MAX stops,
    reward -psi_bar; (1, 1): both continue to the two neighbours with
    probability 1/2 each, reward h^2 r(x) plus half of an end point's stop
    value where a neighbour is an end point (v(0) = psi_bar, v(1) = -psi_bar).

    Returns (n, m1, m2, row_ptr, col, prob, reward, mu)."""
    c, psi1, psi2, v_left, v_right = stopping_line(points)
    n = points - 2
    row_ptr = [0]
    cols, probs, rews = [], [], []
    for x in range(n):
        for a in range(2):
            for b in range(2):
                if b == 0:
                    rews.append(psi2[x])
                elif a == 0:
                    rews.append(psi1[x])
                else:
                    r = c[x]
                    for j, end in ((x - 1, v_left), (x + 1, v_right)):
                        if 0 <= j < n:
                            cols.append(j)
                            probs.append(0.5)
                        else:
                            r += 0.5 * end
                    rews.append(r)
                row_ptr.append(len(cols))
    return (n, 2, 2, np.array(row_ptr, np.int64), np.array(cols, np.int32),
            np.array(probs, np.float64), np.array(rews, np.float64), 1.0)


def iex1_tables(side: int, Ka: int, Kb: int, lo: float = -0.25, hi: float = 1.25):
    """The Isaacs example of Sec. 6.1 (Eq. (Iex1d), lambda = 0, so mu = 1) with
    finite action sets, as CSR tables (gamesolve_set_game layout).  Problem
    data only.  h = 1/(side+1); MAX's actions a_k = (cos 2 pi k/Ka, sin 2 pi
    k/Ka); MIN's actions the Kb x Kb grid over [lo, hi]^2 (index j1 * Kb + j2).
    With d = a - b and c = 4 + h|d1| + h|d2|, the moves east / west / north /
    south have probabilities (1 + h max(d1,0))/c, (1 + h max(-d1,0))/c,
    (1 + h max(d2,0))/c, (1 + h max(-d2,0))/c; a move onto the boundary leaves
    the state space and its probability times sin x1 sin x2 there joins the
    reward h^2 (|b|^2/2 + f(x))/c, f = 2u - |grad u| + |grad u|^2/2 for
    u = sin x1 sin x2.  Rows hold the interior moves in the order east, west,
    north, south.

    Returns (n, m1, m2, row_ptr, col, prob, reward, mu)."""
    h = 1.0 / (side + 1)
    n = side * side
    t = 2.0 * np.pi * np.arange(Ka) / Ka
    a1, a2 = np.cos(t), np.sin(t)
    g = lo + (hi - lo) * np.arange(Kb) / (Kb - 1)
    b1 = np.repeat(g, Kb)
    b2 = np.tile(g, Kb)
    m1, m2 = Ka, Kb * Kb
    d1 = a1[:, None] - b1[None, :]
    d2 = a2[:, None] - b2[None, :]
    c = 4.0 + h * (np.abs(d1) + np.abs(d2))
    moves = [((1, 0), (1.0 + h * np.maximum(d1, 0.0)) / c), ((-1, 0), (1.0 + h * np.maximum(-d1, 0.0)) / c),
             ((0, 1), (1.0 + h * np.maximum(d2, 0.0)) / c), ((0, -1), (1.0 + h * np.maximum(-d2, 0.0)) / c)]
    x = np.arange(n)
    i1, i2 = x % side, x // side
    x1, x2 = (i1 + 1) * h, (i2 + 1) * h
    u = np.sin(x1) * np.sin(x2)
    gn = np.sqrt((np.cos(x1) * np.sin(x2)) ** 2 + (np.sin(x1) * np.cos(x2)) ** 2)
    f = 2.0 * u - gn + 0.5 * gn * gn
    half_b2 = 0.5 * (b1 * b1 + b2 * b2)
    reward = (h * h / c)[None] * (half_b2[None, None, :] + f[:, None, None])     # [n, m1, m2]
    cols, probs, count = [], [], np.zeros(n, np.int64)
    for (s1, s2), p in moves:
        j1, j2 = i1 + s1, i2 + s2
        inside = (j1 >= 0) & (j1 < side) & (j2 >= 0) & (j2 < side)
        psi = np.sin((j1 + 1) * h) * np.sin((j2 + 1) * h)
        reward += np.where(inside, 0.0, psi)[:, None, None] * p[None]
        cols.append(np.where(inside, j2 * side + j1, -1))
        probs.append(p)
        count += inside
    # rows in (x, a, b) order, each with its interior moves
    k_of = count                                             # moves per row of state x
    row_len = np.repeat(k_of, m1 * m2)
    row_ptr = np.concatenate([[0], np.cumsum(row_len)]).astype(np.int64)
    col = np.empty(int(row_ptr[-1]), np.int32)
    prob = np.empty(int(row_ptr[-1]), np.float64)
    pos = row_ptr[:-1].reshape(n, m1, m2).copy()
    for cset, p in zip(cols, probs):
        ok = cset >= 0
        xs = np.nonzero(ok)[0]
        if len(xs) == 0:
            continue
        dst = pos[xs]                                        # [k, m1, m2]
        col[dst.reshape(-1)] = np.repeat(cset[xs], m1 * m2)
        prob[dst.reshape(-1)] = np.broadcast_to(p[None], (len(xs), m1, m2)).reshape(-1)
        pos[xs] += 1
    return (n, m1, m2, row_ptr, col, prob, reward.reshape(-1), 1.0)
