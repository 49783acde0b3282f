"""GPU parity of the Isaacs path against the FP64 oracle, through the C-ABI.

Bars: value to 1e-10 relative max-norm (FP64 path) and 1e-9 (mixed path);
policies bit-exact wherever the oracle's max-min gap exceeds 1e-8; integer
work (noise generation, interpolated policies) bit-exact.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.isaacs import isaacs_game, default_alpha0
from oracle.fmg import famg_pi, interp_value, interp_policy

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-9, "mixed_bf16": 1e-9}
_CACHE = {}


def oracle_solve(side, variant, seed):
    key = (side, variant, seed)
    if key not in _CACHE:
        game = isaacs_game(side, variant, seed=seed)
        _CACHE[key] = (game, oracle.policy_iteration(game, alpha0=default_alpha0(side, variant)))
    return _CACHE[key]


def rel_err(v, ref):
    return np.max(np.abs(v - ref)) / max(np.max(np.abs(ref)), 1e-300)


def check_policies(alpha, beta, ref, m1):
    sure_a = ref.gap_max > 1e-8
    assert np.array_equal(alpha[sure_a], ref.alpha[sure_a])
    sure_b = ref.gap_min[:, :4] > 1e-8
    assert np.array_equal(beta[:, :4][sure_b], ref.beta[:, :4][sure_b])
    assert beta.shape == (len(alpha), m1)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
@pytest.mark.parametrize("side", [1, 3, 7, 15, 63, 255])
def test_solve_parity_plain(gs, side, prec):
    game, ref = oracle_solve(side, 0, 1)
    with gs.GameSolver(precision=prec) as s:
        s.set_isaacs_grid(side, 0, 1)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    assert rel_err(v, ref.v) <= TOL[prec], (rel_err(v, ref.v), st)
    check_policies(a, b, ref, 4)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
@pytest.mark.parametrize("side", [15, 63])
def test_solve_parity_obstacle(gs, side, prec):
    game, ref = oracle_solve(side, 1, 2)
    with gs.GameSolver(precision=prec) as s:
        s.set_isaacs_grid(side, 1, 2)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    assert rel_err(v, ref.v) <= TOL[prec]
    check_policies(a, b, ref, 5)


def test_noise_generators_agree(gs):
    """The CUDA SplitMix64 stream and synth's give bit-identical solves."""
    side, seed = 63, 12345
    out = []
    for xi in (None, synth.isaacs_noise(side, seed)):
        with gs.GameSolver() as s:
            s.set_isaacs_grid(side, 0, seed, xi=xi)
            s.solve()
            out.append(s.get_value())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("side", [63, 255])
def test_improve_parity(gs, side):
    """One policy improvement (Eq. (eq1)/(ILPI)) at a perturbed value."""
    game, ref = oracle_solve(side, 0, 1)
    rng = np.random.default_rng(side)
    v = ref.v + 1e-3 * rng.standard_normal(ref.v.shape)
    alpha0 = rng.integers(0, 4, size=game.n).astype(np.uint8)
    beta0 = rng.integers(0, 4, size=(game.n, 4)).astype(np.uint8)
    a_ref, b_ref, fv_ref = oracle.improve(game, v, alpha0, beta0)
    q = oracle.shapley_q(game, v)
    with gs.GameSolver() as s:
        s.set_isaacs_grid(side, 0, 1)
        s.set_initial(alpha0=alpha0, beta0=beta0)
        a, b, fv = s.improve(v)
    assert np.max(np.abs(fv - fv_ref)) <= 1e-14
    fa = q.min(axis=2)
    srt = np.sort(fa, axis=1)
    sure_a = srt[:, -1] - srt[:, -2] > 1e-8
    assert np.array_equal(a[sure_a], a_ref[sure_a])
    sb = np.sort(q, axis=2)
    sure_b = sb[:, :, 1] - sb[:, :, 0] > 1e-8
    assert np.array_equal(b[sure_b], b_ref[sure_b])


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
@pytest.mark.parametrize("side", [7, 63, 255])
def test_policy_solve_parity(gs, side, prec):
    """The multigrid solve of Eq. (LSPI) for fixed policies vs a direct solve."""
    game, _ = oracle_solve(side, 0, 1)
    rng = np.random.default_rng(7)
    alpha = rng.integers(0, 4, size=game.n).astype(np.uint8)
    beta = rng.integers(0, 4, size=(game.n, 4)).astype(np.uint8)
    A, r = oracle.policy_system(game, alpha, beta)
    w_ref = oracle.solve_policy_system(A, r)
    with gs.GameSolver(precision=prec) as s:
        s.set_isaacs_grid(side, 0, 1)
        w, st = s.policy_solve(alpha, beta)
    assert rel_err(w, w_ref) <= TOL[prec] / 10, (rel_err(w, w_ref), st)


def test_bf16_storage_takes_effect(gs):
    """bfloat16 weights change the V-cycle's iterates (not bit-identical to the
    float32-weight path) but not the float64 answer they refine."""
    side = 255
    rng = np.random.default_rng(5)
    alpha = rng.integers(0, 4, size=side * side).astype(np.uint8)
    beta = rng.integers(0, 4, size=(side * side, 4)).astype(np.uint8)
    out = {}
    for prec in ("mixed", "mixed_bf16"):
        with gs.GameSolver(precision=prec) as s:
            s.set_isaacs_grid(side, 0, 1)
            out[prec] = s.policy_solve(alpha, beta)
    (w32, st32), (w16, st16) = out["mixed"], out["mixed_bf16"]
    assert not np.array_equal(w32, w16)
    assert rel_err(w16, w32) <= 1e-12, (st32, st16)


@pytest.mark.parametrize("variant", [0, 1])
def test_fmg_parity(gs, variant):
    """FAMGpi (Algorithm 4) from side 15 to 127 reaches the oracle's value."""
    side, seed = 127, 3
    _, ref = oracle_solve(side, variant, seed)
    with gs.GameSolver(fmg=1, fmg_side=15, fmg_c=0.1 if variant == 0 else 0.01) as s:
        s.set_isaacs_grid(side, variant, seed)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["fmg_levels"] == 4 and st["converged"] == 1
    assert rel_err(v, ref.v) <= 1e-10
    check_policies(a, b, ref, 5 if variant else 4)


def test_status_codes(gs):
    with gs.GameSolver() as s:
        with pytest.raises(gs.GameSolveError) as e:
            s.solve()
        assert e.value.status == gs.GS_ESTATE
        with pytest.raises(gs.GameSolveError) as e:
            s.set_isaacs_grid(10, 0, 1)
        assert e.value.status == gs.GS_EINVAL
        s.set_isaacs_grid(15, 0, 1)
        with pytest.raises(gs.GameSolveError) as e:
            s.set_initial(alpha0=np.full(225, 7, np.uint8))
        assert e.value.status == gs.GS_EINVAL
    with gs.GameSolver(max_outer=1, max_inner=1) as s:
        s.set_isaacs_grid(63, 0, 1)
        st = gs.gs_solve_stats()
        code = gs.lib.gamesolve_solve(s.h, gs.ctypes.byref(st))
        assert code == gs.GS_ENOTCONV and st.outer == 1
    with gs.GameSolver(mem_budget=1 << 16) as s:
        with pytest.raises(gs.GameSolveError) as e:
            s.set_isaacs_grid(255, 0, 1)
        assert e.value.status == gs.GS_ENOMEM


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
@pytest.mark.parametrize("tail_side", [1, 7, 15, 31, 63])
def test_vcycle_count_size_independent(gs, prec, tail_side):
    """AMG cycles per system stay bounded as the grid grows (the paper's tables
    report 3-5 W-cycles per system at every size), whatever the split between
    grid-wide and single-block levels.  Rounding the coarse operators to
    bfloat16 (8 significant bits) perturbs the preconditioner, not the float64
    residual it drives down, so it may cost a few more cycles."""
    rng = np.random.default_rng(11)
    for side in (63, 255, 1023):
        n = side * side
        alpha = rng.integers(0, 4, size=n).astype(np.uint8)
        beta = rng.integers(0, 4, size=(n, 4)).astype(np.uint8)
        with gs.GameSolver(precision=prec, tail_side=tail_side) as s:
            s.set_isaacs_grid(side, 0, 1)
            _, st = s.policy_solve(alpha, beta)
        assert st["cycles"] <= (20 if prec == "mixed_bf16" else 14), (side, st)
        assert st["res_inf"] < 1e-14


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("side,variant", [(15, 0), (63, 0), (255, 0), (63, 1)])
def test_wcycle_solve_parity(gs, side, variant, prec):
    """W-cycles (Algorithm 3 with gamma = 2, the paper's own cycle) reach the
    oracle's value and policies like V-cycles."""
    _, ref = oracle_solve(side, variant, 1)
    with gs.GameSolver(precision=prec, cycle_gamma=2) as s:
        s.set_isaacs_grid(side, variant, 1)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    assert rel_err(v, ref.v) <= TOL[prec], (rel_err(v, ref.v), st)
    check_policies(a, b, ref, 5 if variant else 4)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
@pytest.mark.parametrize("sweeps", [(1, 2, 0, 1), (1, 2, 1, 0), (1, 2, 1, 1), (2, 1, 0, 2)])
@pytest.mark.parametrize("side,variant,tail", [(63, 0, 15), (255, 0, 31), (255, 0, 63), (63, 1, 31)])
def test_coarse_sweeps_solve_parity(gs, side, variant, tail, sweeps, prec):
    """Other sweep counts on the coarse levels than on the finest (Algorithm 3
    leaves nu1, nu2 free per level) reach the oracle's value and policies, on
    the grid-wide levels and on the single-block tail."""
    nu1, nu2, c1, c2 = sweeps
    _, ref = oracle_solve(side, variant, 1)
    with gs.GameSolver(precision=prec, nu1=nu1, nu2=nu2, nu1_coarse=c1, nu2_coarse=c2,
                       tail_side=tail) as s:
        s.set_isaacs_grid(side, variant, 1)
        st = s.solve()
        v = s.get_value()
        a, b = s.get_policy()
    assert st["converged"] == 1
    assert rel_err(v, ref.v) <= TOL[prec], (rel_err(v, ref.v), st)
    check_policies(a, b, ref, 5 if variant else 4)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("tail_side", [1, 15, 31, 63])
def test_wcycle_needs_no_more_cycles_than_vcycle(gs, prec, tail_side):
    """A W-cycle visits every coarse level twice per visit of the level above:
    per system it needs at most as many cycles as a V-cycle, at every split
    between grid-wide and single-block levels, and it solves the same system."""
    rng = np.random.default_rng(13)
    side = 255
    alpha = rng.integers(0, 4, size=side * side).astype(np.uint8)
    beta = rng.integers(0, 4, size=(side * side, 4)).astype(np.uint8)
    out = {}
    for gamma in (1, 2):
        with gs.GameSolver(precision=prec, tail_side=tail_side, cycle_gamma=gamma) as s:
            s.set_isaacs_grid(side, 0, 1)
            out[gamma] = s.policy_solve(alpha, beta)
    (wv, stv), (ww, stw) = out[1], out[2]
    assert stw["cycles"] <= stv["cycles"], (stv, stw)
    assert stw["res_inf"] < 1e-14
    assert rel_err(ww, wv) <= 1e-12


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("side_c", [1, 7, 31, 63])
def test_fmg_interpolation_matches_oracle(gs, side_c, variant):
    """FAMGpi's interpolations I (value) and U (strategies) of Sec. 5.2, run
    by the CUDA kernel the solver uses, against the oracle's: policies bit for
    bit, values to 1e-15 (a mean of 2 or 4 numbers, summed in another order)."""
    rng = np.random.default_rng(100 * side_c + variant)
    n, m1 = side_c * side_c, 5 if variant else 4
    v = rng.standard_normal(n)
    alpha = rng.integers(0, m1, n).astype(np.uint8)
    beta = rng.integers(0, 4, (n, m1)).astype(np.uint8)
    vf, af, bf = gs.fmg_interpolate(side_c, variant, v, alpha, beta)
    v_ref = interp_value(v, side_c)
    assert np.max(np.abs(vf - v_ref)) <= 1e-15 * np.max(np.abs(v_ref))
    assert np.array_equal(af, interp_policy(alpha, side_c))
    assert np.array_equal(bf, interp_policy(beta, side_c))


@pytest.mark.parametrize("variant", [0, 1])
def test_fmg_level_counts_match_oracle(gs, variant):
    """FAMGpi from side 15 to 127 (Algorithm 4), every policy evaluation to the
    float64 floor (pi_rtol = 0): per level, the MAX iterations and the linear
    systems solved are the oracle's, so the GPU follows the same path of
    policies on every level, not only to the same fixed point."""
    side, seed = 127, 3
    c = 0.1 if variant == 0 else 0.01
    xi = synth.isaacs_noise(side, seed)
    _, per_level = famg_pi(side, 15, variant, xi, c=c, eps=0.0)
    want = [(s, r.outer, r.systems) for s, r in zip((15, 31, 63, 127), per_level)]
    for prec in ("fp64", "mixed"):
        with gs.GameSolver(precision=prec, fmg=1, fmg_side=15, fmg_c=c, pi_rtol=0.0,
                           setup_reuse=0.0) as s:
            s.set_isaacs_grid(side, variant, seed)
            st = s.solve()
            got = s.level_stats()
        assert st["converged"] == 1
        assert got == want, (prec, got, want)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
@pytest.mark.parametrize("side,variant,cyc", [(63, 0, (1, 1)), (255, 1, (1, 2)), (1023, 0, (1, 2)),
                                              (255, 0, (2, 1)), (2047, 1, (1, 2))])
def test_tiled_cycles_match_per_colour_kernel(gs, side, variant, cyc, prec):
    """The tiled V-cycle kernel (default) and the one-phase-per-colour kernel
    run the same arithmetic per point: the same policy-fixed solve reaches the
    same value (to rounding of a different contraction order) in the same
    number of cycles."""
    rng = np.random.default_rng(side + variant)
    n, m1 = side * side, 5 if variant else 4
    alpha = rng.integers(0, m1, n).astype(np.uint8)
    beta = rng.integers(0, 4, (n, m1)).astype(np.uint8)
    out = {}
    for ck in (0, 1):
        with gs.GameSolver(precision=prec, cycle_kernel=ck, nu1=cyc[0], nu2=cyc[1]) as s:
            s.set_isaacs_grid(side, variant, 3)
            out[ck] = s.policy_solve(alpha, beta)
    (w0, s0), (w1, s1) = out[0], out[1]
    assert s0["cycles"] == s1["cycles"], (s0, s1)
    assert rel_err(w0, w1) <= 1e-13
