"""The allocation-free policy solve against the allocating one.

gamesolve_isaacs_policy_solve_static serves callers that cannot let a
library allocate device memory (their device memory belongs to their own
allocator, or cudaMalloc/cudaFree and the synchronisation they can imply are
not acceptable where they call from): it takes its scratch from one static
device array instead.  Its result must match gamesolve_policy_solve, which
allocates a solver's hierarchy, on the same system, call after call (the
array keeps the previous call's contents, so the second call checks that
everything that must start from zero is cleared).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-9, "mixed_bf16": 1e-9}   # the value tolerances of the parity tests


def _static_solve(gs, torch, side, variant, seed, alpha_d, beta_d, w_d, precision):
    st = gs.gs_solve_stats()
    stream = torch.cuda.current_stream().cuda_stream
    code = gs.lib.gamesolve_isaacs_policy_solve_static(
        side, variant, seed, None, alpha_d.data_ptr(), beta_d.data_ptr(), None, w_d.data_ptr(),
        gs.PRECISIONS[precision], stream, ctypes.byref(st))
    torch.cuda.synchronize()
    return code, st


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_bf16"])
@pytest.mark.parametrize("side,variant", [(127, 0), (63, 1), (127, 1)])
def test_static_solve_matches_allocating_solve(gs, side, variant, precision):
    import torch
    rng = np.random.default_rng(side + variant)
    n, m1 = side * side, 5 if variant else 4
    seed = 9
    for call in range(2):
        alpha = rng.integers(0, m1, size=n).astype(np.uint8)
        beta = rng.integers(0, 4, size=(n, m1)).astype(np.uint8)
        with gs.GameSolver(precision=precision) as s:
            s.set_isaacs_grid(side, variant, seed)
            w_ref, _ = s.policy_solve(alpha, beta)
        alpha_d = torch.from_numpy(alpha).cuda()
        beta_d = torch.from_numpy(beta).cuda()
        w_d = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        code, st = _static_solve(gs, torch, side, variant, seed, alpha_d, beta_d, w_d, precision)
        assert code == gs.GS_OK, gs.lib.gamesolve_last_error()
        w = w_d.cpu().numpy()
        err = np.max(np.abs(w - w_ref)) / np.max(np.abs(w_ref))
        assert err <= TOL[precision], (call, err, st.cycles)


def test_static_solve_rejects_oversize_and_host_memory(gs):
    import torch
    side = 255
    n = side * side
    a = torch.zeros(n, dtype=torch.uint8, device="cuda")
    b = torch.zeros((n, 4), dtype=torch.uint8, device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    code, _ = _static_solve(gs, torch, side, 0, 1, a, b, w, "fp64")
    assert code == gs.GS_EINVAL and b"at most 127" in gs.lib.gamesolve_last_error()
    side = 15
    n = side * side
    a_h = np.zeros(n, np.uint8)
    b_d = torch.zeros((n, 4), dtype=torch.uint8, device="cuda")
    w_d = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = gs.gs_solve_stats()
    code = gs.lib.gamesolve_isaacs_policy_solve_static(
        side, 0, 1, None, a_h.ctypes.data, b_d.data_ptr(), None, w_d.data_ptr(), 0, None,
        ctypes.byref(st))
    assert code == gs.GS_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("side,variant", [(15, 0), (31, 1)])
def test_static_solve_matches_oracle_and_allocates_nothing(gs, side, variant, precision):
    """Against the oracle's direct solve of the same policy-fixed system
    (Eq. (LSPI)), and with the device's free memory unchanged across the
    call: the entry point takes its scratch from the static array only."""
    import torch
    import oracle
    from oracle.isaacs import isaacs_game
    rng = np.random.default_rng(side)
    n, m1 = side * side, 5 if variant else 4
    seed = 4
    alpha = rng.integers(0, m1, size=n).astype(np.uint8)
    beta = rng.integers(0, 4, size=(n, m1)).astype(np.uint8)
    A, r = oracle.policy_system(isaacs_game(side, variant, seed=seed), alpha, beta)
    w_ref = oracle.solve_policy_system(A, r, "dense")
    alpha_d = torch.from_numpy(alpha).cuda()
    beta_d = torch.from_numpy(beta).cuda()
    w_d = torch.zeros(n, dtype=torch.float64, device="cuda")
    code, _ = _static_solve(gs, torch, side, variant, seed, alpha_d, beta_d, w_d, precision)
    assert code == gs.GS_OK
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        code, st = _static_solve(gs, torch, side, variant, seed, alpha_d, beta_d, w_d, precision)
        assert code == gs.GS_OK and st.converged == 1
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    w = w_d.cpu().numpy()
    assert np.max(np.abs(w - w_ref)) <= 1e-10 * np.max(np.abs(w_ref))
