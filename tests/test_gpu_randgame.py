"""Random games drawn on the device (gamesolve_random_game / set_random_game).

The device generator and synth.random_game implement the same counter-based
recipe from the SplitMix64 definition: successors and rewards must agree bit
for bit, probabilities to a few units in the last place (each side takes
log1p from its own maths library).  Games set from a seed are solved and
compared with the FP64 oracle run on synth's tables of the same seed.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.game import game_from_csr

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-9}


@pytest.mark.parametrize("n,m1,m2,k,seed", [(50, 4, 4, 8, 3), (1, 2, 3, 1, 9), (8, 3, 2, 8, 11),
                                            (5, 4, 4, 3, 12345), (40000, 4, 4, 8, 77),
                                            (1000, 7, 2, 5, (1 << 64) - 5)])
def test_device_tables_match_synth(gs, n, m1, m2, k, seed):
    rp, col, prob, rew, _ = gs.random_game(n, m1, m2, seed, k=k)
    rp0, col0, prob0, rew0, _ = synth.random_game(n, seed, m1=m1, m2=m2, k=k)
    assert np.array_equal(rp, rp0)
    assert np.array_equal(col, col0)
    assert np.array_equal(rew, rew0)
    assert np.max(np.abs(prob - prob0)) <= 4 * np.finfo(np.float64).eps
    # every row a distribution over distinct successors in increasing order
    c = col.reshape(-1, k)
    assert np.all(np.diff(c, axis=1) > 0) and c.min() >= 0 and c.max() < n
    s = prob.reshape(-1, k).sum(axis=1)
    assert np.all(np.abs(s - 1.0) <= 1e-14) and prob.min() >= 0.0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,seed", [(300, 21), (1500, 22), (5000, 23)])
def test_set_random_game_against_oracle(gs, n, seed, prec):
    rp, col, prob, rew, mu = synth.random_game(n, seed)
    ref = oracle.policy_iteration(game_from_csr(n, 4, 4, rp, col, prob, rew, mu),
                                  solver="auto" if n <= 2000 else "fixed_point")
    with gs.GameSolver(precision=prec) as s:
        s.set_random_game(n, 4, 4, seed, mu)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    assert np.max(np.abs(v - ref.v)) <= TOL[prec] * np.max(np.abs(ref.v))
    sure = ref.gap_max > 1e-8
    assert np.array_equal(a[sure], ref.alpha[sure])
    # the same game given as the device-drawn table
    tab = gs.random_game(n, 4, 4, seed)
    with gs.GameSolver(precision=prec) as s:
        s.set_game(n, 4, 4, *tab)
        s.solve()
        assert np.array_equal(s.get_value(), v)


def test_random_game_rejects(gs):
    import torch
    rp = torch.empty(4 * 4 * 10 + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(4 * 4 * 10 * 8, dtype=torch.int32, device="cuda")
    prob = torch.empty(4 * 4 * 10 * 8, dtype=torch.float64, device="cuda")
    rew = torch.empty(4 * 4 * 10, dtype=torch.float64, device="cuda")
    ptrs = [rp.data_ptr(), col.data_ptr(), prob.data_ptr(), rew.data_ptr()]
    for n, m1, m2, k in ((0, 4, 4, 8), (10, 0, 4, 8), (10, 65, 4, 8), (10, 4, 256, 8), (10, 4, 4, 9),
                         (5, 4, 4, 6), (10, 4, 4, 0)):
        assert gs.lib.gamesolve_random_game(n, m1, m2, k, 1, *ptrs, None) == gs.GS_EINVAL
    host = np.empty(4 * 4 * 10 + 1, np.int64)
    assert gs.lib.gamesolve_random_game(10, 4, 4, 8, 1, host.ctypes.data, *ptrs[1:], None) == gs.GS_EINVAL
    assert b"device memory" in gs.lib.gamesolve_last_error()
    with gs.GameSolver() as s:
        assert gs.lib.gamesolve_set_random_game(s.h, 10, 4, 4, 8, 1, 1.0) == gs.GS_EINVAL
        assert gs.lib.gamesolve_set_random_game(s.h, 10, 4, 4, 8, 1, 0.0) == gs.GS_EINVAL
    torch.cuda.synchronize()
