"""Python binding of libgamesolve (include/gamesolve.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; this module only
converts arguments.  Importing it loads the in-tree shared library and fails
loudly if it has not been built (``paper_1107_1653_gb300.build.build()``).
Arrays may be numpy arrays (host) or torch tensors (host or CUDA); outputs
are numpy arrays unless a preallocated ``out`` tensor is given.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgamesolve.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1107_1653_gb300.build.build()")
lib = ctypes.CDLL(LIB_PATH)

GS_OK, GS_EINVAL, GS_ENOMEM, GS_ENOTCONV, GS_ETIMEOUT, GS_ECUDA, GS_ESTATE = range(7)
GS_PREC_FP64, GS_PREC_MIXED, GS_PREC_MIXED_BF16 = range(3)
KERNEL_CLASSES = {"none": 0, "improve": 1, "mg_setup": 2, "mg_cycles": 3}
PRECISIONS = {"fp64": GS_PREC_FP64, "mixed": GS_PREC_MIXED, "mixed_bf16": GS_PREC_MIXED_BF16}


class gs_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32), ("eps", ctypes.c_double),
        ("max_outer", ctypes.c_int32), ("max_inner", ctypes.c_int32),
        ("nu1", ctypes.c_int32), ("nu2", ctypes.c_int32),
        ("max_cycles", ctypes.c_int32), ("lin_tol", ctypes.c_double),
        ("coarse_max", ctypes.c_int32), ("fmg", ctypes.c_int32),
        ("fmg_side", ctypes.c_int32), ("fmg_c", ctypes.c_double),
        ("mu_mode", ctypes.c_int32), ("tail_side", ctypes.c_int32),
        ("mem_budget", ctypes.c_uint64), ("stream", ctypes.c_void_p),
        ("pi_rtol", ctypes.c_double), ("setup_reuse", ctypes.c_double),
        ("grid_blocks", ctypes.c_int32), ("cycle_gamma", ctypes.c_int32),
        ("nu1_coarse", ctypes.c_int32), ("nu2_coarse", ctypes.c_int32),
        ("game_threads", ctypes.c_int32),
        ("cycle_kernel", ctypes.c_int32),
        ("game_solver", ctypes.c_int32), ("amg_coarsening", ctypes.c_int32),
        ("amg_theta", ctypes.c_double),
    ]


class gs_solve_stats(ctypes.Structure):
    _fields_ = [
        ("outer", ctypes.c_int32), ("systems", ctypes.c_int32),
        ("cycles", ctypes.c_int32), ("levels", ctypes.c_int32),
        ("res_inf", ctypes.c_double), ("res_l2", ctypes.c_double),
        ("seconds", ctypes.c_double), ("converged", ctypes.c_int32),
        ("fmg_levels", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gs_request(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("side", ctypes.c_int32), ("variant", ctypes.c_int32),
        ("m1", ctypes.c_int32), ("m2", ctypes.c_int32), ("seed", ctypes.c_uint64),
        ("n", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
        ("prob", ctypes.c_void_p), ("reward", ctypes.c_void_p), ("mu", ctypes.c_double),
        ("flags", ctypes.c_int32), ("k", ctypes.c_int32),
    ]


GS_REQ_BORROW = 1


class gs_ticket_info(ctypes.Structure):
    _fields_ = [
        ("state", ctypes.c_int32), ("status", ctypes.c_int32),
        ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_end", ctypes.c_double),
        ("n", ctypes.c_int64), ("stats", gs_solve_stats),
    ]


_P = ctypes.c_void_p
_S = ctypes.c_int
_SIGS = {
    "gamesolve_default_options": (None, [ctypes.POINTER(gs_options)]),
    "gamesolve_create": (_S, [ctypes.POINTER(_P), ctypes.POINTER(gs_options)]),
    "gamesolve_set_game": (_S, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P,
                                ctypes.c_double]),
    "gamesolve_set_game_batch": (_S, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                      _P, _P, _P, _P]),
    "gamesolve_get_batch_stats": (_S, [_P, _P, _P]),
    "gamesolve_random_game": (_S, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_uint64, _P, _P, _P, _P, _P]),
    "gamesolve_set_random_game": (_S, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_uint64, ctypes.c_double]),
    "gamesolve_get_batch_shape": (_S, [_P, _P]),
    "gamesolve_set_stopping_line": (_S, [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_double,
                                         ctypes.c_double]),
    "gamesolve_set_isaacs_grid": (_S, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _P]),
    "gamesolve_set_initial": (_S, [_P, _P, _P, _P]),
    "gamesolve_solve": (_S, [_P, ctypes.POINTER(gs_solve_stats)]),
    "gamesolve_get_value": (_S, [_P, _P, ctypes.c_int64]),
    "gamesolve_get_policy": (_S, [_P, _P, _P]),
    "gamesolve_improve": (_S, [_P, _P, _P, _P, _P]),
    "gamesolve_policy_solve": (_S, [_P, _P, _P, _P, _P, ctypes.POINTER(gs_solve_stats)]),
    "gamesolve_isaacs_policy_solve_static": (_S, [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                                  _P, _P, _P, _P, _P, ctypes.c_int32, _P,
                                                  ctypes.POINTER(gs_solve_stats)]),
    "gamesolve_fmg_interpolate": (_S, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P, _P,
                                       _P]),
    "gamesolve_get_level_stats": (_S, [_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "gamesolve_selftest_barrier": (_S, [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.c_int32, _P, ctypes.POINTER(ctypes.c_int32)]),
    "gamesolve_trace": (_S, [_P, ctypes.c_int32]),
    "gamesolve_trace_read": (_S, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "gamesolve_kernel_launches": (ctypes.c_uint64, []),
    "gamesolve_server_create": (_S, [ctypes.POINTER(_P), ctypes.POINTER(gs_options), ctypes.c_int32,
                                     ctypes.c_uint64]),
    "gamesolve_server_submit": (_S, [_P, ctypes.POINTER(gs_request), ctypes.POINTER(ctypes.c_int64)]),
    "gamesolve_server_poll": (_S, [_P, ctypes.c_int64, ctypes.POINTER(gs_ticket_info)]),
    "gamesolve_server_wait": (_S, [_P, ctypes.c_int64, ctypes.POINTER(gs_ticket_info)]),
    "gamesolve_server_result": (_S, [_P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P]),
    "gamesolve_server_destroy": (None, [_P]),
    "gamesolve_destroy": (None, [_P]),
    "gamesolve_strerror": (ctypes.c_char_p, [_S]),
    "gamesolve_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args
    globals()[_name] = _fn


class GameSolveError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib.gamesolve_strerror(status).decode()
        detail = lib.gamesolve_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")


def _check(st, where, allow=(GS_OK,)):
    if st not in allow:
        raise GameSolveError(st, where)
    return st


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None stays NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def _as(a, dtype):
    if a is None or not isinstance(a, np.ndarray) and not isinstance(a, (list, tuple)):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


def default_options(**kw) -> gs_options:
    o = gs_options()
    lib.gamesolve_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream
        setattr(o, k, v)
    return o


class GameSolver:
    """Owns one gs_solver.  Keyword arguments override gs_options fields."""

    def __init__(self, **opts):
        self.opts = default_options(**opts)
        h = _P()
        _check(lib.gamesolve_create(ctypes.byref(h), ctypes.byref(self.opts)), "gamesolve_create")
        self.h = h
        self.n = 0
        self.m1 = 0

    def close(self):
        if getattr(self, "h", None):
            lib.gamesolve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_isaacs_grid(self, side, variant=0, seed=1, xi=None):
        xi = _as(xi, np.float64)
        _check(lib.gamesolve_set_isaacs_grid(self.h, side, variant, seed, _ptr(xi)),
               "gamesolve_set_isaacs_grid")
        self.n = side * side
        self.m1 = 5 if variant == 1 else 4

    def set_game(self, n, m1, m2, row_ptr, col, prob, reward, mu):
        row_ptr, col = _as(row_ptr, np.int64), _as(col, np.int32)
        prob, reward = _as(prob, np.float64), _as(reward, np.float64)
        _check(lib.gamesolve_set_game(self.h, n, m1, m2, _ptr(row_ptr), _ptr(col), _ptr(prob),
                                      _ptr(reward), mu), "gamesolve_set_game")
        self.n, self.m1, self.count = n, m1, 1

    def set_random_game(self, n, m1, m2, seed, mu, k=8):
        """The random game of random_game(n, m1, m2, seed, k), drawn on the device."""
        _check(lib.gamesolve_set_random_game(self.h, n, m1, m2, k, seed, mu),
               "gamesolve_set_random_game")
        self.n, self.m1, self.count = n, m1, 1

    def set_stopping_line(self, c, psi1, psi2, v_left, v_right):
        c, psi1, psi2 = _as(c, np.float64), _as(psi1, np.float64), _as(psi2, np.float64)
        n = len(c)
        _check(lib.gamesolve_set_stopping_line(self.h, n, _ptr(c), _ptr(psi1), _ptr(psi2),
                                               float(v_left), float(v_right)),
               "gamesolve_set_stopping_line")
        self.n, self.m1, self.count = n, 2, 1

    def set_game_batch(self, state_offsets, m1, m2, row_ptr, col, prob, reward, mu):
        off = _as(state_offsets, np.int64)
        row_ptr, col = _as(row_ptr, np.int64), _as(col, np.int32)
        prob, reward, mu = _as(prob, np.float64), _as(reward, np.float64), _as(mu, np.float64)
        count = len(off) - 1
        _check(lib.gamesolve_set_game_batch(self.h, count, m1, m2, _ptr(off), _ptr(row_ptr),
                                            _ptr(col), _ptr(prob), _ptr(reward), _ptr(mu)),
               "gamesolve_set_game_batch")
        self.n, self.m1, self.count = int(off[-1]), m1, count

    def batch_stats(self):
        st = np.empty((self.count, 4), np.int32)
        res = np.empty(self.count, np.float64)
        _check(lib.gamesolve_get_batch_stats(self.h, _ptr(st), _ptr(res)),
               "gamesolve_get_batch_stats")
        return st, res

    def batch_shape(self):
        t = ctypes.c_int32()
        _check(lib.gamesolve_get_batch_shape(self.h, ctypes.byref(t)), "gamesolve_get_batch_shape")
        return t.value

    def set_initial(self, v0=None, alpha0=None, beta0=None):
        v0, alpha0, beta0 = _as(v0, np.float64), _as(alpha0, np.uint8), _as(beta0, np.uint8)
        _check(lib.gamesolve_set_initial(self.h, _ptr(v0), _ptr(alpha0), _ptr(beta0)),
               "gamesolve_set_initial")

    def solve(self, allow_notconv=False):
        st = gs_solve_stats()
        allow = (GS_OK, GS_ENOTCONV) if allow_notconv else (GS_OK,)
        _check(lib.gamesolve_solve(self.h, ctypes.byref(st)), "gamesolve_solve", allow)
        return st.as_dict()

    def get_value(self, out=None):
        out = np.empty(self.n, np.float64) if out is None else out
        _check(lib.gamesolve_get_value(self.h, _ptr(out), self.n), "gamesolve_get_value")
        return out

    def get_policy(self, alpha_out=None, beta_out=None):
        a = np.empty(self.n, np.uint8) if alpha_out is None else alpha_out
        b = np.empty((self.n, self.m1), np.uint8) if beta_out is None else beta_out
        _check(lib.gamesolve_get_policy(self.h, _ptr(a), _ptr(b)), "gamesolve_get_policy")
        return a, b

    def improve(self, v):
        v = _as(v, np.float64)
        a = np.empty(self.n, np.uint8)
        b = np.empty((self.n, self.m1), np.uint8)
        fv = np.empty(self.n, np.float64)
        _check(lib.gamesolve_improve(self.h, _ptr(v), _ptr(a), _ptr(b), _ptr(fv)),
               "gamesolve_improve")
        return a, b, fv

    def trace(self, kernel_class):
        cls = KERNEL_CLASSES[kernel_class] if isinstance(kernel_class, str) else kernel_class
        _check(lib.gamesolve_trace(self.h, cls), "gamesolve_trace")

    def trace_read(self):
        ms = ctypes.c_double()
        cnt = ctypes.c_int64()
        _check(lib.gamesolve_trace_read(self.h, ctypes.byref(ms), ctypes.byref(cnt)),
               "gamesolve_trace_read")
        return ms.value, cnt.value

    def level_stats(self):
        """Per FAMGpi level (coarsest first): (side, MAX iterations, linear systems)."""
        out = np.zeros((32, 3), np.int32)
        nl = ctypes.c_int32()
        _check(lib.gamesolve_get_level_stats(self.h, _ptr(out), 32, ctypes.byref(nl)),
               "gamesolve_get_level_stats")
        return [tuple(int(x) for x in row) for row in out[:nl.value]]

    def policy_solve(self, alpha, beta, w0=None, allow_notconv=False):
        alpha, beta, w0 = _as(alpha, np.uint8), _as(beta, np.uint8), _as(w0, np.float64)
        w = np.empty(self.n, np.float64)
        st = gs_solve_stats()
        allow = (GS_OK, GS_ENOTCONV) if allow_notconv else (GS_OK,)
        code = _check(lib.gamesolve_policy_solve(self.h, _ptr(alpha), _ptr(beta), _ptr(w0),
                                                 _ptr(w), ctypes.byref(st)),
                      "gamesolve_policy_solve", allow)
        d = st.as_dict()
        d["status"] = code
        return w, d


class GameServer:
    """Owns one gs_server (continuous batching of solve requests)."""

    def __init__(self, slots=2, mem_budget=0, **opts):
        self.opts = default_options(**opts)
        h = _P()
        _check(lib.gamesolve_server_create(ctypes.byref(h), ctypes.byref(self.opts), slots,
                                           mem_budget), "gamesolve_server_create")
        self.h = h
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            lib.gamesolve_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit_isaacs(self, side, variant=0, seed=1):
        r = gs_request(kind=1, side=side, variant=variant, seed=seed)
        t = ctypes.c_int64()
        _check(lib.gamesolve_server_submit(self.h, ctypes.byref(r), ctypes.byref(t)),
               "gamesolve_server_submit")
        self._keep[t.value] = (side * side, 5 if variant == 1 else 4)
        return t.value

    def submit_game(self, n, m1, m2, row_ptr, col, prob, reward, mu, borrow=False):
        """borrow=True: the arrays (host or CUDA) are read when the request runs
        and must stay alive and unchanged until it is done."""
        row_ptr, col = _as(row_ptr, np.int64), _as(col, np.int32)
        prob, reward = _as(prob, np.float64), _as(reward, np.float64)
        r = gs_request(kind=2, n=n, m1=m1, m2=m2, row_ptr=_ptr(row_ptr), col=_ptr(col),
                       prob=_ptr(prob), reward=_ptr(reward), mu=mu,
                       flags=GS_REQ_BORROW if borrow else 0)
        t = ctypes.c_int64()
        _check(lib.gamesolve_server_submit(self.h, ctypes.byref(r), ctypes.byref(t)),
               "gamesolve_server_submit")
        self._keep[t.value] = (n, m1)
        return t.value

    def submit_random_game(self, n, m1, m2, seed, mu, k=8):
        """A random game given by its seed: its table is drawn on the device when
        the request runs (gamesolve_set_random_game)."""
        r = gs_request(kind=3, n=n, m1=m1, m2=m2, seed=seed, mu=mu, k=k)
        t = ctypes.c_int64()
        _check(lib.gamesolve_server_submit(self.h, ctypes.byref(r), ctypes.byref(t)),
               "gamesolve_server_submit")
        self._keep[t.value] = (n, m1)
        return t.value

    @staticmethod
    def _info(info):
        d = {k: getattr(info, k) for k, _ in gs_ticket_info._fields_ if k != "stats"}
        d["stats"] = info.stats.as_dict()
        return d

    def poll(self, ticket):
        info = gs_ticket_info()
        _check(lib.gamesolve_server_poll(self.h, ticket, ctypes.byref(info)), "gamesolve_server_poll")
        return self._info(info)

    def wait(self, ticket):
        info = gs_ticket_info()
        _check(lib.gamesolve_server_wait(self.h, ticket, ctypes.byref(info)), "gamesolve_server_wait")
        return self._info(info)

    def result(self, ticket):
        n, m1 = self._keep.pop(ticket)
        v = np.empty(n, np.float64)
        a = np.empty(n, np.uint8)
        b = np.empty((n, m1), np.uint8)
        _check(lib.gamesolve_server_result(self.h, ticket, _ptr(v), n, _ptr(a), _ptr(b)),
               "gamesolve_server_result", (GS_OK, GS_ENOTCONV))
        return v, a, b


def fmg_interpolate(side_c, variant, v_c, alpha_c, beta_c):
    """FAMGpi's value and strategy interpolations (Sec. 5.2) to side 2 side_c + 1."""
    m1 = 5 if variant == 1 else 4
    v_c, alpha_c = _as(v_c, np.float64), _as(alpha_c, np.uint8)
    beta_c = _as(beta_c, np.uint8)
    sf = 2 * side_c + 1
    v = np.empty(sf * sf, np.float64)
    a = np.empty(sf * sf, np.uint8)
    b = np.empty((sf * sf, m1), np.uint8)
    _check(lib.gamesolve_fmg_interpolate(side_c, variant, _ptr(v_c), _ptr(alpha_c), _ptr(beta_c),
                                         _ptr(v), _ptr(a), _ptr(b), None),
           "gamesolve_fmg_interpolate")
    return v, a, b


def random_game(n, m1, m2, seed, k=8, mu=0.99):
    """The random game of gamesolve_random_game, drawn on the current CUDA device
    and returned as host arrays (row_ptr, col, prob, reward, mu) in the layout of
    GameSolver.set_game."""
    import torch
    rows = n * m1 * m2
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.empty(rows + 1, dtype=torch.int64, device=dev)
    col = torch.empty(rows * k, dtype=torch.int32, device=dev)
    prob = torch.empty(rows * k, dtype=torch.float64, device=dev)
    rew = torch.empty(rows, dtype=torch.float64, device=dev)
    _check(lib.gamesolve_random_game(n, m1, m2, k, seed, rp.data_ptr(), col.data_ptr(), prob.data_ptr(),
                                     rew.data_ptr(), torch.cuda.current_stream().cuda_stream),
           "gamesolve_random_game")
    torch.cuda.synchronize()
    return rp.cpu().numpy(), col.cpu().numpy(), prob.cpu().numpy(), rew.cpu().numpy(), float(mu)


def exported_symbols():
    """Names of the C-ABI functions this binding resolves from the library."""
    return sorted(_SIGS)
