"""Finite discounted zero-sum games and Hoffman-Karp policy iteration (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

A game is stored densely per (x, a, b): up to K successors with their
probabilities (unused slots have successor -1 and probability 0) and the
reward r(x, a, b).  All arithmetic is float64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass
class Game:
    """(n, m1, m2, p(.|x,a,b), r(x,a,b), mu) of Sec. 2.

    succ[x, a, b, k] is the k-th successor y of row (x, a, b) or -1;
    prob[x, a, b, k] is p(y | x, a, b) for that successor.  Rows may be
    substochastic (sum p < 1): the missing mass leaves the state space
    (Dirichlet boundary of Sec. 3.3, or a stop action of Sec. 3.2).
    """
    succ: np.ndarray
    prob: np.ndarray
    rew: np.ndarray
    mu: float

    @property
    def n(self):
        return self.succ.shape[0]

    @property
    def m1(self):
        return self.succ.shape[1]

    @property
    def m2(self):
        return self.succ.shape[2]


def game_from_csr(n, m1, m2, row_ptr, col, prob, reward, mu) -> Game:
    """Converts the C-ABI's CSR layout (row (x*m1+a)*m2+b) to a dense Game."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    R = n * m1 * m2
    lens = np.diff(row_ptr)
    K = int(lens.max()) if R else 0
    K = max(K, 1)
    succ = -np.ones((R, K), dtype=np.int64)
    pr = np.zeros((R, K), dtype=np.float64)
    for k in range(K):
        has = lens > k
        idx = row_ptr[:-1][has] + k
        succ[has, k] = np.asarray(col, dtype=np.int64)[idx]
        pr[has, k] = np.asarray(prob, dtype=np.float64)[idx]
    return Game(succ.reshape(n, m1, m2, K), pr.reshape(n, m1, m2, K),
                np.asarray(reward, dtype=np.float64).reshape(n, m1, m2), float(mu))


def shapley_q(game: Game, v: np.ndarray) -> np.ndarray:
    """Q[x, a, b] = F(v; x, a, b) = sum_y mu p(y|x,a,b) v(y) + r(x,a,b), Eq. (ILPI)."""
    vpad = np.append(np.asarray(v, dtype=np.float64), 0.0)   # index -1 reads 0
    gathered = vpad[game.succ]                                 # v(y) per successor slot
    return (game.mu * game.prob * gathered).sum(axis=-1) + game.rew


def tie_tolerance(v: np.ndarray) -> float:
    """Improvement threshold tau = 1e-13 * max(1, |v|_inf) of the keep-current rule."""
    return 1e-13 * max(1.0, float(np.max(np.abs(v))) if v.size else 1.0)


def _keep_current(vals: np.ndarray, cur: np.ndarray, tau: float, maximise: bool):
    """argmax/argmin over the last axis with the keep-current tie rule.

    The current action is kept unless another action is better by more than
    tau; otherwise the lowest index attaining the exact optimum is taken.
    (The paper's argmax/argmin of Eq. (eq1) are sets; this picks one element.)
    """
    best = vals.max(axis=-1) if maximise else vals.min(axis=-1)
    curval = np.take_along_axis(vals, cur[..., None].astype(np.int64), axis=-1)[..., 0]
    first = np.argmax(vals == best[..., None], axis=-1)
    worse = (best - curval > tau) if maximise else (curval - best > tau)
    return np.where(worse, first, cur).astype(np.uint8), best


def _gap(vals: np.ndarray, maximise: bool) -> np.ndarray:
    """Best minus second-best value over the last axis (inf with one action)."""
    if vals.shape[-1] < 2:
        return np.full(vals.shape[:-1], np.inf)
    s = np.sort(vals, axis=-1)
    return (s[..., -1] - s[..., -2]) if maximise else (s[..., 1] - s[..., 0])


def improve(game: Game, v: np.ndarray, alpha: np.ndarray, beta: np.ndarray):
    """One full policy improvement at value v (Alg. 2 step 2 with the MIN reply).

    For every x and a: beta'(x, a) in argmin_b F(v; x, a, b); then
    alpha'(x) in argmax_a F(v; x, a) with F(v; x, a) = min_b F(v; x, a, b)
    (Eq. (ILPI)), both with the keep-current rule.  Returns
    (alpha', beta', Fv) where Fv[x] = F(v; x) of Eq. (eq1).
    """
    tau = tie_tolerance(v)
    q = shapley_q(game, v)
    beta_new, fa = _keep_current(q, beta, tau, maximise=False)
    alpha_new, fv = _keep_current(fa, alpha, tau, maximise=True)
    return alpha_new, beta_new, fv


def improve_min(game: Game, w: np.ndarray, alpha: np.ndarray, beta: np.ndarray):
    """Inner improvement of Alg. 1 step 2 at fixed alpha: beta(x, alpha(x)) only."""
    tau = tie_tolerance(w)
    q = shapley_q(game, w)
    n = game.n
    qa = q[np.arange(n), alpha]                      # F(w; x, alpha(x), b) over b
    ba = beta[np.arange(n), alpha]
    ba_new, _ = _keep_current(qa, ba, tau, maximise=False)
    beta_new = beta.copy()
    beta_new[np.arange(n), alpha] = ba_new
    return beta_new


def policy_system(game: Game, alpha: np.ndarray, beta: np.ndarray):
    """(A, r) with A = I - mu M^{alpha beta} and r = r^{alpha beta}, Eq. (LSPI).

    M_{x,y} = p(y | x, alpha(x), beta(x, alpha(x))); duplicate successors of a
    row are summed.  A is returned as a scipy CSR matrix.
    """
    n = game.n
    xs = np.arange(n)
    a = alpha.astype(np.int64)
    b = beta[xs, a].astype(np.int64)
    succ = game.succ[xs, a, b]                # [n, K]
    prob = game.prob[xs, a, b]
    rows = np.repeat(xs, succ.shape[1])
    cols = succ.reshape(-1)
    vals = prob.reshape(-1)
    keep = cols >= 0
    M = sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n, n))
    A = (sp.identity(n, format="csr") - game.mu * M).tocsr()
    r = game.rew[xs, a, b].copy()
    return A, r


def solve_policy_system(A, r, method: str = "auto", tol: float = 1e-14,
                        max_sweeps: int = 200000):
    """Solves A w = r for the policy-fixed system of Eq. (LSPI).

    * "dense": LAPACK LU (numpy.linalg.solve), n <= a few thousand;
    * "lu": sparse LU (SuperLU) followed by two steps of iterative
      refinement with float64 residuals;
    * "fixed_point": w <- (I - A) w + r, i.e. w <- mu M w + r, the
      fixed-policy value iteration, a mu-contraction in the sup-norm; stops
      when |w - (mu M w + r)|_inf <= tol * max(1, |w|_inf).
    """
    n = A.shape[0]
    if method == "auto":
        method = "dense" if n <= 2000 else "lu"
    if method == "dense":
        return np.linalg.solve(A.toarray(), r)
    if method == "lu":
        lu = spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A")
        w = lu.solve(r)
        for _ in range(2):
            w = w + lu.solve(r - A @ w)
        return w
    if method == "fixed_point":
        B = (sp.identity(n, format="csr") - A).tocsr()      # = mu M
        w = r.copy()
        for _ in range(max_sweeps):
            w_next = B @ w + r
            if np.max(np.abs(w_next - w)) <= tol * max(1.0, np.max(np.abs(w_next))):
                return w_next
            w = w_next
        raise RuntimeError("fixed-point solve did not reach tolerance")
    raise ValueError(method)


@dataclass
class PIResult:
    v: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    outer: int                       # MAX policy iterations k
    systems: int                     # linear systems solved (sum of #j)
    residual: float                  # |F(v) - v|_inf at the final v
    converged: bool
    gap_max: np.ndarray = None       # best minus second-best F(v; x, a) over a
    gap_min: np.ndarray = None       # same over b, for every (x, a)
    outer_values: list = field(default_factory=list)   # v after each outer step
    inner_values: list = field(default_factory=list)   # per outer step, the inner w's


def policy_iteration(game: Game, alpha0=None, beta0=None, v0=None, eps: float = 0.0,
                     max_outer: int = 10000, max_inner: int = 10000,
                     solver: str = "auto", record: bool = False) -> PIResult:
    """Hoffman-Karp / Puri policy iteration, Algorithm 2 with Algorithm 1 inside.

    alpha <- alpha0 (default all 0).  v <- v0 (default 0).  The first inner
    loop starts from beta0 when given (a warm start, as FAMGpi passes it),
    else from MIN's best reply beta(x, a) in argmin_b F(v; x, a, b).

    Inner loop (Alg. 1, alpha fixed): solve (I - mu M^{alpha beta}) w =
    r^{alpha beta}; beta'(x, alpha(x)) in argmin_b F(w; x, alpha(x), b); stop
    when beta is unchanged.  Then v <- w and the outer step (Alg. 2 step 2):
    beta(x, a) in argmin_b F(v; x, a, b) for every a, alpha'(x) in
    argmax_a F(v; x, a); stop when |F(v) - v|_inf <= eps (Sec. 5.1) or alpha is
    unchanged; otherwise alpha <- alpha' and repeat.  The returned policies are
    the final improvement's (greedy with respect to the returned v).
    """
    n, m1, m2 = game.n, game.m1, game.m2
    alpha = np.zeros(n, np.uint8) if alpha0 is None else np.asarray(alpha0, np.uint8).copy()
    v = np.zeros(n) if v0 is None else np.asarray(v0, np.float64).copy()
    if beta0 is None:
        q = shapley_q(game, v)
        beta, _ = _keep_current(q, np.zeros((n, m1), np.uint8), tie_tolerance(v), False)
    else:
        beta = np.asarray(beta0, np.uint8).reshape(n, m1).copy()
    outer = systems = 0
    outer_values, inner_values = [], []
    converged = False
    while True:
        inner = []
        for _ in range(max_inner):
            A, r = policy_system(game, alpha, beta)
            w = solve_policy_system(A, r, solver)
            systems += 1
            if record:
                inner.append(w.copy())
            beta_new = improve_min(game, w, alpha, beta)
            if np.array_equal(beta_new, beta):
                break
            beta = beta_new
        v = w
        outer += 1
        if record:
            outer_values.append(v.copy())
            inner_values.append(inner)
        alpha_new, beta, fv = improve(game, v, alpha, beta)
        residual = float(np.max(np.abs(fv - v))) if n else 0.0
        if residual <= eps or np.array_equal(alpha_new, alpha):
            alpha = alpha_new
            converged = True
            break
        alpha = alpha_new
        if outer >= max_outer:
            break
    q = shapley_q(game, v)
    fa = q.min(axis=-1)
    res = PIResult(v=v, alpha=alpha, beta=beta, outer=outer, systems=systems,
                   residual=residual, converged=converged,
                   gap_max=_gap(fa, True), gap_min=_gap(q, False),
                   outer_values=outer_values, inner_values=inner_values)
    return res
