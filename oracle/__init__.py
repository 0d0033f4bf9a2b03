"""ctypes front-end of the CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg import this package.  The CUDA library and its Python binding
never do: the two implementations share no code.

The oracle restates the F3R solver of "A Nested Krylov Method Using
Half-Precision Arithmetic" (Sec. 4.2, Table 1, Algorithm 1, Eqs. 4-5) with
per-operation rounding; see f3r_oracle.cpp for the readings it takes.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

F64, F32, F16, BF16 = 0, 1, 2, 3
PC_IDENTITY, PC_JACOBI, PC_AINV = 0, 1, 3
OK, ERR_ARG, NOT_CONVERGED, BREAKDOWN, NONFINITE = 0, 1, 4, 5, 6


class Params(C.Structure):
    _fields_ = [
        ("nlevels", C.c_int), ("m", C.c_int * 4), ("a_prec", C.c_int * 4), ("v_prec", C.c_int * 4),
        ("rich_m", C.c_int), ("rich_a_prec", C.c_int), ("rich_v_prec", C.c_int), ("m_prec", C.c_int),
        ("precond", C.c_int), ("c", C.c_int), ("omega_fixed", C.c_double), ("diag_scale", C.c_int),
        ("row_scale", C.c_int), ("scale_cast", C.c_int), ("cgs_passes", C.c_int), ("tol", C.c_double),
        ("max_outer", C.c_int), ("inner_rtol", C.c_double),
    ]


class RichState(C.Structure):
    _fields_ = [("omega", C.c_double * 8), ("c_ntr", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("outer_iters", C.c_int), ("restarts", C.c_int), ("rel_res_true", C.c_double),
        ("m_applies", C.c_int64), ("r_calls", C.c_int64), ("r_update_calls", C.c_int64),
        ("omega", C.c_double * 8), ("hist", C.POINTER(C.c_double)), ("hist_cap", C.c_int),
        ("hist_len", C.c_int), ("true_hist", C.POINTER(C.c_double)), ("true_cap", C.c_int),
        ("true_len", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        L.orc_round.argtypes = [C.c_int, dp, dp, C.c_int64]
        L.orc_problem_create.argtypes = [C.c_int32, ip, ip, dp, C.c_int, C.c_int, C.c_int]
        L.orc_problem_create.restype = C.c_void_p
        L.orc_problem_destroy.argtypes = [C.c_void_p]
        L.orc_problem_set_ainv.argtypes = [C.c_void_p, C.c_double]
        L.orc_problem_get.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_problem_get.restype = C.c_int64
        L.orc_default_params.argtypes = [C.POINTER(Params)]
        L.orc_spmv.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, dp]
        L.orc_spmv_orig.argtypes = [C.c_void_p, dp, dp]
        L.orc_apply.argtypes = [C.c_void_p, C.POINTER(Params), C.POINTER(RichState), C.c_int, dp, dp]
        L.orc_solve.argtypes = [C.c_void_p, C.POINTER(Params), dp, dp, C.POINTER(Stats)]
        L.orc_solve.restype = C.c_int
        L.orc_outer_arnoldi.argtypes = [C.c_void_p, C.POINTER(Params), dp, C.c_int, dp, dp, dp]
        L.orc_outer_arnoldi.restype = C.c_int
        L.orc_inner_arnoldi.argtypes = [C.c_void_p, C.POINTER(Params), C.POINTER(RichState), C.c_int, dp, dp,
                                         dp, dp, dp, dp]
        L.orc_inner_arnoldi.restype = C.c_int
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def round_to(prec: int, x) -> np.ndarray:
    """Round float64 values to `prec` (F32/F16/BF16) with ties-to-even."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib().orc_round(prec, _dp(x), _dp(y), x.size)
    return y


def params(**kw) -> Params:
    """Default F3R parameters (100, 8, 4, 2), c = 64, CGS2, tol 1e-9, with overrides.

    List-valued fields (m, a_prec, v_prec) may be given as Python lists.
    """
    p = Params()
    lib().orc_default_params(C.byref(p))
    for k, v in kw.items():
        if k in ("m", "a_prec", "v_prec"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def preset(name: str, **kw) -> Params:
    """Named solver configurations of Sec. 5 and Sec. 6.

    fp16-F3R / fp32-F3R / fp64-F3R (Sec. 5), bf16-F3R (16-bit brain float in
    place of fp16 with per-row scaling), fgmres64 (restarted fp64 FGMRES(64)
    with M), and the depth variants of Table 4: F2 and fp16-F2 (an inner
    FGMRES(64), fp32 or fp16), F3, fp16-F3 (the inner F8 with fp16 vectors)
    and F4 (its F2 with fp16 vectors).
    """
    if name == "fp16-F3R":
        p = params()
    elif name == "bf16-F3R":
        p = params(a_prec=[F64, F32, BF16, BF16], rich_a_prec=BF16, rich_v_prec=BF16, m_prec=BF16,
                   row_scale=1)
    elif name == "fp32-F3R":
        p = params(a_prec=[F64, F32, F32, F32], rich_a_prec=F32, rich_v_prec=F32, m_prec=F32)
    elif name == "fp64-F3R":
        p = params(a_prec=[F64, F64, F64, F64], v_prec=[F64, F64, F64, F64], rich_a_prec=F64,
                   rich_v_prec=F64, m_prec=F64)
    elif name == "fgmres64":
        p = params(nlevels=1, m=[64, 0, 0, 0], rich_m=0, m_prec=F64, max_outer=19200)
    elif name == "F2":
        p = params(nlevels=2, m=[100, 64, 0, 0], a_prec=[F64, F32, F32, F32], rich_m=0, m_prec=F16)
    elif name == "fp16-F2":
        p = params(nlevels=2, m=[100, 64, 0, 0], a_prec=[F64, F16, F32, F32], v_prec=[F64, F16, F32, F32], rich_m=0,
                   m_prec=F16)
    elif name == "F3":
        p = params(nlevels=3, m=[100, 8, 8, 0], rich_m=0, m_prec=F16)
    elif name == "fp16-F3":
        p = params(nlevels=3, m=[100, 8, 8, 0], v_prec=[F64, F32, F16, F32], rich_m=0, m_prec=F16)
    elif name == "F4":
        p = params(nlevels=4, m=[100, 8, 4, 2], a_prec=[F64, F32, F16, F16], v_prec=[F64, F32, F32, F16],
                   rich_m=0, m_prec=F16)
    else:
        raise KeyError(name)
    for k, v in kw.items():
        if k in ("m", "a_prec", "v_prec"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def num_threads() -> int:
    return lib().orc_num_threads()


class Result:
    def __init__(self, x, st: Stats, hist, true_hist):
        self.x = x
        self.status = st.status
        self.outer_iters = st.outer_iters
        self.restarts = st.restarts
        self.rel_res_true = st.rel_res_true
        self.m_applies = st.m_applies
        self.r_calls = st.r_calls
        self.r_update_calls = st.r_update_calls
        self.omega = list(st.omega)
        self.hist = hist
        self.true_hist = true_hist


class Problem:
    """The oracle's copy of one matrix with its scaled and rounded variants."""

    WHICH = {"d": 0, "ahat": 1, "a32": 2, "a16": 3, "abf16": 4, "rs16": 5, "rsbf16": 6,
             "m64": 7, "m32": 8, "m16": 9, "mbf16": 10, "ainv_l": 11, "ainv_u": 12, "ainv_dinv": 13}

    def __init__(self, prob, diag_scale=1, row_scale=0, precond=PC_JACOBI, ainv_alpha=1.0):
        self.n = prob.n
        self._rp = np.ascontiguousarray(prob.rowptr, dtype=np.int32)
        self._ci = np.ascontiguousarray(prob.colidx, dtype=np.int32)
        self._v = np.ascontiguousarray(prob.val, dtype=np.float64)
        self.h = lib().orc_problem_create(self.n, _ip(self._rp), _ip(self._ci), _dp(self._v),
                                          diag_scale, row_scale, precond)
        if precond == PC_AINV:
            # the boost is a single-precision parameter of the solver (f3r_params.ainv_alpha)
            lib().orc_problem_set_ainv(self.h, float(np.float32(ainv_alpha)))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_problem_destroy(self.h)
            self.h = None

    def get(self, what: str) -> np.ndarray:
        w = self.WHICH[what]
        size = lib().orc_problem_get(self.h, w, None)
        out = np.empty(size)
        lib().orc_problem_get(self.h, w, _dp(out))
        return out

    def spmv(self, a_prec: int, v_prec: int, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n)
        lib().orc_spmv(self.h, a_prec, v_prec, _dp(x), _dp(y))
        return y

    def spmv_orig(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n)
        lib().orc_spmv_orig(self.h, _dp(x), _dp(y))
        return y

    def apply(self, prm: Params, state: RichState, level: int, v) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.float64)
        z = np.empty(self.n)
        lib().orc_apply(self.h, C.byref(prm), C.byref(state), level, _dp(v), _dp(z))
        return z

    def solve(self, prm: Params, b, x0=None, hist_cap: int = 20000) -> Result:
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        hist = np.zeros(hist_cap)
        th = np.zeros(1024)
        st = Stats()
        st.hist = _dp(hist)
        st.hist_cap = hist_cap
        st.true_hist = _dp(th)
        st.true_cap = 1024
        lib().orc_solve(self.h, C.byref(prm), _dp(b), _dp(x), C.byref(st))
        return Result(x, st, hist[:min(st.hist_len, hist_cap)].copy(), th[:min(st.true_len, 1024)].copy())

    def outer_arnoldi(self, prm: Params, b, steps: int):
        b = np.ascontiguousarray(b, dtype=np.float64)
        V = np.zeros((steps + 1, self.n))
        Z = np.zeros((steps, self.n))
        H = np.zeros((steps, steps + 1))  # column-major (steps+1) x steps
        lib().orc_outer_arnoldi(self.h, C.byref(prm), _dp(b), steps, _dp(V), _dp(Z), _dp(H))
        return V, Z, H.T.copy()

    def inner_arnoldi(self, prm: Params, state: RichState, level: int, v):
        """One call of inner FGMRES level `level` with its basis recorded.

        Returns (z, V, Z, H, g, k): the level's output z, the basis V ((m+1) x n),
        the preconditioned vectors Z (m x n), the Hessenberg matrix H ((m+1) x m,
        before rotation), the rotated right-hand side g (m+1) and the number of
        columns k the level kept.
        """
        m = prm.m[level]
        v = np.ascontiguousarray(v, dtype=np.float64)
        z = np.empty(self.n)
        V = np.zeros((m + 1, self.n))
        Z = np.zeros((m, self.n))
        H = np.zeros((m, m + 1))  # column-major (m+1) x m
        g = np.zeros(m + 1)
        k = lib().orc_inner_arnoldi(self.h, C.byref(prm), C.byref(state), level, _dp(v), _dp(z), _dp(V),
                                    _dp(Z), _dp(H), _dp(g))
        return z, V, Z, H.T.copy(), g, k


def rich_state(c_ntr: int = 1, omega=None) -> RichState:
    s = RichState()
    s.c_ntr = c_ntr
    for k in range(8):
        s.omega[k] = 1.0 if omega is None else (omega[k] if k < len(omega) else 1.0)
    return s
