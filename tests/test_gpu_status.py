"""Failure statuses through the C-ABI: iteration caps and bounded waits.

* A policy evaluation that reaches max_cycles before the float64 floor has
  not evaluated the policy, so no decision of Algorithm 1 or 2 may rest on
  it: the solve ends with GS_ENOTCONV (stats.converged = 0), on the Isaacs
  path, for a single large game (grid-wide) and for a batch of games.
* Every cooperative kernel synchronises through a grid barrier whose waits
  give up after a limit.  The self-test leaves one block away from the
  barrier with a 2 ms limit: the call must return GS_ETIMEOUT (no hang, no
  trap), and the GPU must stay usable for a following solve.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_isaacs_policy_solve_cycle_cap_is_not_converged(gs):
    side = 255
    n = side * side
    rng = np.random.default_rng(3)
    alpha = rng.integers(0, 4, n).astype(np.uint8)
    beta = rng.integers(0, 4, (n, 4)).astype(np.uint8)
    for prec in ("fp64", "mixed"):
        with gs.GameSolver(precision=prec, max_cycles=1) as s:
            s.set_isaacs_grid(side, 0, 1)
            w, st = s.policy_solve(alpha, beta, allow_notconv=True)
        assert st["status"] == gs.GS_ENOTCONV and st["converged"] == 0, st
        assert st["cycles"] == 1 and st["res_inf"] > 1e-12
        with gs.GameSolver(precision=prec) as s:   # the default cap reaches the floor
            s.set_isaacs_grid(side, 0, 1)
            w, st = s.policy_solve(alpha, beta)
        assert st["status"] == gs.GS_OK and st["converged"] == 1


@pytest.mark.parametrize("fmg", [0, 1])
def test_isaacs_solve_cycle_cap_is_not_converged(gs, fmg):
    with gs.GameSolver(precision="mixed", max_cycles=1, fmg=fmg, fmg_side=15) as s:
        s.set_isaacs_grid(127, 0, 1)
        st = gs.gs_solve_stats()
        code = gs.lib.gamesolve_solve(s.h, ctypes.byref(st))
        v = s.get_value()
    assert code == gs.GS_ENOTCONV and st.converged == 0
    assert np.all(np.isfinite(v))


@pytest.mark.parametrize("n", [600, 6000])
def test_game_cycle_cap_is_not_converged(gs, n):
    """n = 600 runs in one thread block, n = 6000 on the whole grid."""
    rp, col, prob, rew, mu = synth.random_game(n, 21)
    for cap, want in ((1, gs.GS_ENOTCONV), (200, gs.GS_OK)):
        with gs.GameSolver(precision="mixed", max_cycles=cap) as s:
            s.set_game(n, 4, 4, rp, col, prob, rew, mu)
            st = gs.gs_solve_stats()
            code = gs.lib.gamesolve_solve(s.h, ctypes.byref(st))
        assert code == want, (cap, code, st.cycles)
        assert st.converged == (1 if want == gs.GS_OK else 0)


def test_barrier_wait_gives_up_and_the_gpu_stays_usable(gs):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    passed = ctypes.c_int32(-1)
    # every block arrives: all rounds complete
    code = gs.lib.gamesolve_selftest_barrier(64, -1, 2_000_000, 5, stream, ctypes.byref(passed))
    assert code == gs.GS_OK and passed.value == 64 * 5
    # block 7 never arrives: the first wait of the others gives up after 2 ms
    code = gs.lib.gamesolve_selftest_barrier(64, 7, 2_000_000, 5, stream, ctypes.byref(passed))
    assert code == gs.GS_ETIMEOUT, gs.lib.gamesolve_last_error()
    assert passed.value == 0
    torch.cuda.synchronize()
    # the context is intact: a fresh solver solves
    with gs.GameSolver(precision="mixed") as s:
        s.set_isaacs_grid(63, 0, 1)
        st = s.solve()
    assert st["converged"] == 1
