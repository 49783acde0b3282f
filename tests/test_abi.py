"""The C-ABI library loads and exports every entry point include/gamesolve.h
declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "gamesolve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gamesolve_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def gs():
    if not os.path.exists(os.path.join(ROOT, "paper_1107_1653_gb300", "libgamesolve.so")):
        pytest.skip("library not built")
    import paper_1107_1653_gb300 as pkg
    return pkg


def test_every_declared_symbol_is_exported(gs):
    names = declared()
    assert len(names) >= 13
    for name in names:
        assert hasattr(gs.lib, name), name
    assert sorted(gs.exported_symbols()) == names


def test_struct_layouts_match_header(gs):
    # gs_options: 152 bytes, the stream pointer at 88; gs_solve_stats: 48 bytes
    assert ctypes.sizeof(gs.gs_options) == 152 and gs.gs_options.stream.offset == 88
    assert gs.gs_options.game_solver.offset == 136 and gs.gs_options.amg_theta.offset == 144
    assert gs.gs_options.grid_blocks.offset == 112
    assert gs.gs_options.cycle_gamma.offset == 116
    assert gs.gs_options.nu1_coarse.offset == 120 and gs.gs_options.nu2_coarse.offset == 124
    assert gs.gs_options.game_threads.offset == 128
    assert gs.gs_options.cycle_kernel.offset == 132
    assert gs.gs_options.pi_rtol.offset == 96
    assert ctypes.sizeof(gs.gs_solve_stats) == 48


def test_host_side_checks_without_gpu(gs):
    o = gs.default_options()
    assert o.precision == gs.GS_PREC_FP64 and o.nu1 == 1 and o.nu2 == 1 and o.cycle_gamma == 1
    assert o.nu1_coarse == -1 and o.nu2_coarse == -1 and o.game_threads == 0
    assert gs.lib.gamesolve_strerror(gs.GS_ENOTCONV).startswith(b"iteration caps")
    # NULL out-pointer and invalid options are rejected before any CUDA call
    assert gs.lib.gamesolve_create(None, None) == gs.GS_EINVAL
    h = ctypes.c_void_p()
    for kw in ({"coarse_max": 0}, {"nu1_coarse": -2}, {"nu1_coarse": 0, "nu2_coarse": 0},
               {"game_threads": 384}, {"cycle_kernel": 2}, {"game_solver": 2},
               {"amg_coarsening": 2}, {"amg_theta": 1.0}):
        bad = gs.default_options(**kw)
        assert gs.lib.gamesolve_create(ctypes.byref(h), ctypes.byref(bad)) == gs.GS_EINVAL, kw
    assert gs.lib.gamesolve_solve(None, None) == gs.GS_EINVAL
    gs.lib.gamesolve_destroy(None)


def test_barrier_selftest_rejects_bad_arguments_without_gpu(gs):
    # checked before any CUDA call: no blocks, a limit outside 1 us .. 100 ms,
    # an absent block outside the launch
    f = gs.lib.gamesolve_selftest_barrier
    assert f(0, -1, 10**6, 1, None, None) == gs.GS_EINVAL
    assert f(4, -1, 10, 1, None, None) == gs.GS_EINVAL
    assert f(4, -1, 10**9, 1, None, None) == gs.GS_EINVAL
    assert f(4, 4, 10**6, 1, None, None) == gs.GS_EINVAL
