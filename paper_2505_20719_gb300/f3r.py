"""ctypes binding of libf3r.so (include/f3r.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
pointers are passed through unchanged and the library tells host from device
memory.  There is no CPU fallback: if the library is not built or no GPU is
usable, calls raise F3RError.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libf3r.so")

F64, F32, F16, BF16 = 0, 1, 2, 3
PC_IDENTITY, PC_JACOBI, PC_LEARNED, PC_AINV = 0, 1, 2, 3
KRYLOV_CG, KRYLOV_BICGSTAB = 1, 2
LEARNED_NPARAMS = 6337
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of memory", 4: "not converged",
          5: "breakdown", 6: "non-finite value", 7: "device wait timed out", 8: "unsupported"}
OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, NOT_CONVERGED, ERR_BREAKDOWN, ERR_NONFINITE = 0, 1, 2, 3, 4, 5, 6
ERR_TIMEOUT, ERR_UNSUPPORTED = 7, 8


class F3RError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")


class Params(C.Structure):
    _fields_ = [
        ("nlevels", C.c_int), ("m", C.c_int * 4), ("a_prec", C.c_int * 4), ("v_prec", C.c_int * 4),
        ("rich_m", C.c_int), ("rich_a_prec", C.c_int), ("rich_v_prec", C.c_int), ("m_prec", C.c_int),
        ("precond", C.c_int), ("c", C.c_int), ("omega_fixed", C.c_double), ("diag_scale", C.c_int),
        ("row_scale", C.c_int), ("scale_cast", C.c_int), ("cgs_passes", C.c_int), ("tol", C.c_double),
        ("max_outer", C.c_int), ("use_graphs", C.c_int), ("keep_omega", C.c_int), ("fuse_cgs", C.c_int),
        ("inner_rtol", C.c_float), ("ainv_alpha", C.c_float),
        ("fuse_step", C.c_int), ("batch_split", C.c_int), ("batch_wide", C.c_int), ("reserved", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("outer_iters", C.c_int), ("restarts", C.c_int), ("rel_res_true", C.c_double),
        ("m_applies", C.c_int64), ("r_calls", C.c_int64), ("r_update_calls", C.c_int64),
        ("omega", C.c_double * 8), ("hist", C.POINTER(C.c_double)), ("hist_cap", C.c_int),
        ("hist_len", C.c_int), ("true_hist", C.POINTER(C.c_double)), ("true_cap", C.c_int),
        ("true_len", C.c_int), ("t_solve_ms", C.c_double), ("kernel_launches", C.c_int64),
        ("graph_launches", C.c_int64),
    ]


class SystemDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("val", C.c_void_p), ("nrhs", C.c_int32)]


class BatchResult(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_int), ("restarts", C.c_int),
                ("rel_res_true", C.c_double), ("m_applies", C.c_int64), ("r_calls", C.c_int64),
                ("t_solve_ms", C.c_double), ("system", C.c_int), ("rhs", C.c_int), ("path", C.c_int)]


_lib = None


def lib():
    """Load libf3r.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise F3RError(ERR_CUDA, f"libf3r.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.f3r_default_params.argtypes = [C.POINTER(Params)]
        L.f3r_setup.argtypes = [C.POINTER(vp), C.c_int32, C.c_int64, vp, vp, vp, C.POINTER(Params), vp]
        L.f3r_solve.argtypes = [vp, vp, vp, C.POINTER(Stats), vp]
        L.f3r_spmv.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp]
        L.f3r_apply.argtypes = [vp, C.c_int, vp, vp, vp]
        L.f3r_get_rich_state.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.f3r_set_rich_state.argtypes = [vp, C.POINTER(C.c_double), C.c_int64]
        L.f3r_export.argtypes = [vp, C.c_int, vp]
        L.f3r_matrix_info.argtypes = [vp, C.POINTER(C.c_int64)]
        L.f3r_matrix_info.restype = C.c_int
        L.f3r_get_basis.argtypes = [vp, C.c_int, C.c_int, vp, vp]
        L.f3r_device_bytes.argtypes = [vp]
        L.f3r_device_bytes.restype = C.c_int64
        L.f3r_destroy.argtypes = [vp]
        L.f3r_trim_memory.argtypes = []
        L.f3r_status_str.restype = C.c_char_p
        L.f3r_profile_enable.argtypes = [vp, C.c_int]
        L.f3r_profile_enable.restype = C.c_int
        L.f3r_profile_get.argtypes = [vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
        L.f3r_profile_get.restype = C.c_int
        L.f3r_profile_slots.restype = C.c_int
        L.f3r_profile_slot_name.argtypes = [C.c_int]
        L.f3r_profile_slot_name.restype = C.c_char_p
        L.f3r_setup_batched.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(SystemDesc), C.POINTER(Params), vp]
        L.f3r_setup_batched.restype = C.c_int
        L.f3r_solve_batched.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(BatchResult), vp]
        L.f3r_solve_batched.restype = C.c_int
        L.f3r_batched_set_cluster.argtypes = [vp, C.c_int]
        L.f3r_batched_set_cluster.restype = C.c_int
        L.f3r_batched_autotune.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int), vp]
        L.f3r_batched_autotune.restype = C.c_int
        L.f3r_batched_instances.argtypes = [vp]
        L.f3r_batched_instances.restype = C.c_int
        L.f3r_batched_set_shape.argtypes = [vp, C.c_int, C.c_int]
        L.f3r_batched_info.argtypes = [vp, C.POINTER(C.c_int64)]
        L.f3r_batched_wide_info.argtypes = [vp, C.POINTER(C.c_int64)]
        L.f3r_batched_device_bytes.argtypes = [vp]
        L.f3r_batched_device_bytes.restype = C.c_int64
        L.f3r_destroy_batched.argtypes = [vp]
        L.f3r_learned_load.argtypes = [vp, vp, C.c_int]
        L.f3r_learned_get.argtypes = [vp, vp]
        L.f3r_learned_apply.argtypes = [vp, vp, vp, vp]
        L.f3r_learned_loss_grad.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp]
        L.f3r_learned_train.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_float, vp, vp]
        L.f3r_learned_set_loss.argtypes = [vp, C.c_int]
        L.f3r_solve_krylov.argtypes = [vp, C.c_int, vp, vp, C.c_int, C.POINTER(Stats), vp]
        L.f3r_solve_krylov.restype = C.c_int
        for name in ("f3r_learned_load", "f3r_learned_get", "f3r_learned_apply", "f3r_learned_loss_grad",
                     "f3r_learned_train", "f3r_learned_set_loss"):
            getattr(L, name).restype = C.c_int
        L.f3r_round16.argtypes = [C.c_int, vp, vp, C.c_int64, vp]
        L.f3r_round16.restype = C.c_int
        L.f3r_residual_noalloc.argtypes = [C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.f3r_residual_noalloc.restype = C.c_int
        for name in ("f3r_default_params", "f3r_setup", "f3r_solve", "f3r_spmv", "f3r_apply",
                     "f3r_get_rich_state", "f3r_set_rich_state", "f3r_export"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return C.c_void_p(a.ctypes.data)
    raise TypeError(type(a))


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _check(code, where):
    if code != OK:
        raise F3RError(code, where)


def _set(p, kw):
    for k, v in kw.items():
        if k in ("m", "a_prec", "v_prec"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def trim_memory():
    """Return the device memory the library's pools keep for later contexts."""
    _check(lib().f3r_trim_memory(), "f3r_trim_memory")


def default_params(**kw) -> Params:
    p = Params()
    _check(lib().f3r_default_params(C.byref(p)), "f3r_default_params")
    return _set(p, kw)


def preset(name: str, **kw) -> Params:
    """Named configurations: fp16-F3R (Table 1), bf16-F3R (bf16 inner storage
    with per-row scaling), fp32-F3R and fp64-F3R (Sec. 5), fgmres64 (fp64
    restarted FGMRES(64) with M, Sec. 5), and the depth variants F2, fp16-F2,
    F3, fp16-F3 and F4 of Table 4.  Their fp16-vector levels compute in fp32 and round
    every stored V and Z value to fp16 (held in fp32 arrays)."""
    if name == "fp16-F3R":
        p = default_params()
    elif name == "bf16-F3R":
        p = default_params(a_prec=[F64, F32, BF16, BF16], rich_a_prec=BF16, rich_v_prec=BF16, m_prec=BF16,
                           row_scale=1)
    elif name == "fp32-F3R":
        p = default_params(a_prec=[F64, F32, F32, F32], rich_a_prec=F32, rich_v_prec=F32, m_prec=F32)
    elif name == "fp64-F3R":
        p = default_params(a_prec=[F64, F64, F64, F64], v_prec=[F64, F64, F64, F64], rich_a_prec=F64,
                           rich_v_prec=F64, m_prec=F64)
    elif name == "fgmres64":
        p = default_params(nlevels=1, m=[64, 0, 0, 0], rich_m=0, m_prec=F64, max_outer=19200)
    elif name == "F2":
        # Table 4: (F100, F64, M), the inner FGMRES(64) in fp32
        p = default_params(nlevels=2, m=[100, 64, 0, 0], a_prec=[F64, F32, F32, F32], rich_m=0, m_prec=F16)
    elif name == "fp16-F2":
        # Table 4: the inner FGMRES(64) with fp16 A and fp16 vectors
        p = default_params(nlevels=2, m=[100, 64, 0, 0], a_prec=[F64, F16, F32, F32], v_prec=[F64, F16, F32, F32],
                           rich_m=0, m_prec=F16)
    elif name == "F3":
        # Table 4: (F100, F8, F8, M), the inner F8 with fp16 A and fp32 vectors
        p = default_params(nlevels=3, m=[100, 8, 8, 0], rich_m=0, m_prec=F16)
    elif name == "fp16-F3":
        # Table 4: F3 with fp16 vectors in the inner F8
        p = default_params(nlevels=3, m=[100, 8, 8, 0], v_prec=[F64, F32, F16, F32], rich_m=0, m_prec=F16)
    elif name == "F4":
        # Table 4: (F100, F8, F4, F2, M), the F2 with fp16 A and fp16 vectors
        p = default_params(nlevels=4, m=[100, 8, 4, 2], a_prec=[F64, F32, F16, F16], v_prec=[F64, F32, F32, F16],
                           rich_m=0, m_prec=F16)
    else:
        raise KeyError(name)
    return _set(p, kw)


class Result:
    def __init__(self, st: Stats, hist, true_hist):
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
        self.t_solve_ms = st.t_solve_ms
        self.kernel_launches = st.kernel_launches
        self.graph_launches = st.graph_launches


class Solver:
    """One f3r_ctx: the matrix set up on the current CUDA device."""

    def __init__(self, rowptr, colidx, val, params: Params = None, stream=None):
        self.h = C.c_void_p()
        n = len(rowptr) - 1
        nnz = int(rowptr[-1])
        self.n = n
        self.params = params if params is not None else default_params()
        _check(lib().f3r_setup(C.byref(self.h), n, nnz, _ptr(rowptr), _ptr(colidx), _ptr(val),
                               C.byref(self.params), _stream(stream)), "f3r_setup")

    @classmethod
    def from_problem(cls, prob, params: Params = None, stream=None):
        return cls(np.ascontiguousarray(prob.rowptr, dtype=np.int32),
                   np.ascontiguousarray(prob.colidx, dtype=np.int32),
                   np.ascontiguousarray(prob.val, dtype=np.float64), params, stream)

    def close(self):
        if self.h and _lib is not None:
            _lib.f3r_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b, x, stream=None, hist_cap: int = 4096, check: bool = False) -> Result:
        """x holds x0 on entry and the solution on exit (host or device arrays)."""
        hist = np.zeros(hist_cap)
        th = np.zeros(256)
        st = Stats()
        st.hist = hist.ctypes.data_as(C.POINTER(C.c_double))
        st.hist_cap = hist_cap
        st.true_hist = th.ctypes.data_as(C.POINTER(C.c_double))
        st.true_cap = 256
        code = lib().f3r_solve(self.h, _ptr(b), _ptr(x), C.byref(st), _stream(stream))
        if code not in (OK, NOT_CONVERGED, ERR_NONFINITE) or (check and code != OK):
            raise F3RError(code, "f3r_solve")
        return Result(st, hist[:min(st.hist_len, hist_cap)].copy(), th[:min(st.true_len, 256)].copy())

    def solve_krylov(self, method: str, b, x, max_iters: int = 100000, stream=None,
                     hist_cap: int = 1 << 17) -> Result:
        """The paper's comparators on this context's matrix: method 'cg' or
        'bicgstab' (fp64, preconditioner D^-1/2 M D^-1/2)."""
        m = {"cg": KRYLOV_CG, "bicgstab": KRYLOV_BICGSTAB}[method]
        hist = np.zeros(hist_cap)
        th = np.zeros(4)
        st = Stats()
        st.hist = hist.ctypes.data_as(C.POINTER(C.c_double))
        st.hist_cap = hist_cap
        st.true_hist = th.ctypes.data_as(C.POINTER(C.c_double))
        st.true_cap = 4
        code = lib().f3r_solve_krylov(self.h, m, _ptr(b), _ptr(x), int(max_iters), C.byref(st), _stream(stream))
        if code not in (OK, NOT_CONVERGED, ERR_NONFINITE, ERR_BREAKDOWN):
            raise F3RError(code, "f3r_solve_krylov")
        return Result(st, hist[:min(st.hist_len, hist_cap)].copy(), th[:min(st.true_len, 4)].copy())

    def spmv(self, p: int, vp: int, x, y, stream=None):
        _check(lib().f3r_spmv(self.h, p, vp, _ptr(x), _ptr(y), _stream(stream)), "f3r_spmv")

    def apply(self, level: int, x, z, stream=None):
        _check(lib().f3r_apply(self.h, level, _ptr(x), _ptr(z), _stream(stream)), "f3r_apply")

    def get_basis(self, level: int, k: int, out, stream=None):
        """V[k] of FGMRES level `level` after the last call (f3r_get_basis) into `out`."""
        _check(lib().f3r_get_basis(self.h, level, k, _ptr(out), _stream(stream)), "f3r_get_basis")
        return out

    def rich_state(self):
        om = (C.c_double * 8)()
        cn = C.c_int64()
        _check(lib().f3r_get_rich_state(self.h, om, C.byref(cn)), "f3r_get_rich_state")
        return list(om), cn.value

    def set_rich_state(self, omega, c_ntr: int):
        om = (C.c_double * 8)(*([float(w) for w in omega] + [1.0] * (8 - len(omega))))
        _check(lib().f3r_set_rich_state(self.h, om, c_ntr), "f3r_set_rich_state")

    def export(self, which: int, nnz: int = None) -> np.ndarray:
        """Set-up arrays in CSR order: 0 d, 1 A^ f64, 2 A^ f32, 3 A^/s f16 bits,
        4 A^/s bf16 bits, 5 row scales, 6 M (m_prec); approximate inverse:
        7 L Dt^-1, 8 Dt^-1 U (f16 bits, nnz), 9 Dt^-1 (f16 bits, n); 10 the
        column each windowed entry stands for (int32, nnz)."""
        n = self.n
        if which == 0:
            out = np.empty(n, np.float64)
        elif which == 1:
            out = np.empty(nnz, np.float64)
        elif which == 2:
            out = np.empty(nnz, np.float32)
        elif which in (3, 4, 7, 8):
            out = np.empty(nnz, np.uint16)
        elif which == 9:
            out = np.empty(n, np.uint16)
        elif which == 10:
            out = np.empty(nnz, np.int32)
        elif which == 5:
            out = np.empty(n, np.float32)
        else:
            mp = self.params.m_prec
            out = np.empty(n, {F64: np.float64, F32: np.float32}.get(mp, np.uint16))
        _check(lib().f3r_export(self.h, which, _ptr(out)), "f3r_export")
        return out

    # ------------------------------------------------------------ learned M
    def learned_load(self, params, train: bool = False):
        """Load the flat fp32 parameter vector (LEARNED_NPARAMS values)."""
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == LEARNED_NPARAMS
        _check(lib().f3r_learned_load(self.h, p.ctypes.data, 1 if train else 0), "f3r_learned_load")

    def learned_get(self) -> np.ndarray:
        out = np.empty(LEARNED_NPARAMS, np.float32)
        _check(lib().f3r_learned_get(self.h, out.ctypes.data), "f3r_learned_get")
        return out

    def learned_apply(self, r, z, stream=None):
        _check(lib().f3r_learned_apply(self.h, _ptr(r), _ptr(z), _stream(stream)), "f3r_learned_apply")

    def learned_set_loss(self, kind: int):
        """0: error loss ||M(r) - e||^2/||e||^2; 1: residual loss ||A16 M(r) - r||^2/||r||^2."""
        _check(lib().f3r_learned_set_loss(self.h, int(kind)), "f3r_learned_set_loss")

    def learned_loss_grad(self, R, E, stream=None):
        """R, E: device fp32 (P, n).  Returns (loss, grad)."""
        loss = np.zeros(1, np.float32)
        grad = np.zeros(LEARNED_NPARAMS, np.float32)
        _check(lib().f3r_learned_loss_grad(self.h, _ptr(R), _ptr(E), R.shape[0], loss.ctypes.data, grad.ctypes.data,
                                           _stream(stream)), "f3r_learned_loss_grad")
        return float(loss[0]), grad

    def learned_train(self, R, E, steps: int, batch: int, lr: float, stream=None) -> np.ndarray:
        hist = np.zeros(max(steps, 1), np.float32)
        _check(lib().f3r_learned_train(self.h, _ptr(R), _ptr(E), R.shape[0], steps, batch, lr, hist.ctypes.data,
                                       _stream(stream)), "f3r_learned_train")
        return hist[:steps]

    def profile(self, enable: bool):
        """Turn the per-kernel event profiler on (resetting it) or off."""
        _check(lib().f3r_profile_enable(self.h, 1 if enable else 0), "f3r_profile_enable")

    def profile_report(self) -> dict:
        """{'<kind>_L<level>': {'launches': n, 'ms': total device ms}} of the profiled launches."""
        out = {}
        for slot in range(lib().f3r_profile_slots()):
            cnt, tms = C.c_int64(), C.c_double()
            _check(lib().f3r_profile_get(self.h, slot, C.byref(cnt), C.byref(tms)), "f3r_profile_get")
            if cnt.value:
                name = lib().f3r_profile_slot_name(slot).decode() + f"_L{slot % 4}"
                out[name] = {"launches": cnt.value, "ms": tms.value}
        return out

    @property
    def device_bytes(self) -> int:
        return lib().f3r_device_bytes(self.h)

    def matrix_info(self) -> dict:
        """Storage of the set-up matrix (f3r_matrix_info)."""
        out = (C.c_int64 * 8)()
        _check(lib().f3r_matrix_info(self.h, out), "f3r_matrix_info")
        keys = ("windowed", "win_max", "nsell", "wmax", "nslices", "index_bytes", "win_chunk", "m_unit")
        return {k: int(v) for k, v in zip(keys, out)}


def round16(prec: int, x, out, stream=None):
    """f3r_round16: the library's fp32 -> 16-bit store conversion of device
    array x (float32) into out (16-bit patterns, int16 or uint16 storage)."""
    _check(lib().f3r_round16(prec, _ptr(x), _ptr(out), int(x.numel()), _stream(stream)), "f3r_round16")
    return out


class BatchedSolver:
    """Many systems (each with nrhs right-hand sides): f3r_setup_batched /
    f3r_solve_batched.  Every instance is solved in one persistent launch:
    systems below params.batch_split rows on one thread-block cluster each,
    larger systems on wide teams of params.batch_wide clusters (or, with
    batch_wide < 0, one after another by the single-system path)."""

    def __init__(self, systems, params: Params = None, stream=None):
        """systems: list of (rowptr, colidx, val, nrhs) with host (numpy) or
        device (torch) arrays."""
        self.h = C.c_void_p()
        self._keep = systems
        arr = (SystemDesc * len(systems))()
        self.ns = []
        for k, (rp, ci, va, nrhs) in enumerate(systems):
            n = len(rp) - 1
            self.ns.append(n)
            arr[k] = SystemDesc(n, int(rp[-1]), _ptr(rp), _ptr(ci), _ptr(va), nrhs)
        self.params = params if params is not None else default_params()
        _check(lib().f3r_setup_batched(C.byref(self.h), len(systems), arr, C.byref(self.params),
                                       _stream(stream)), "f3r_setup_batched")
        self.ninst = lib().f3r_batched_instances(self.h)

    def set_cluster(self, k: int):
        _check(lib().f3r_batched_set_cluster(self.h, k), "f3r_batched_set_cluster")

    def set_shape(self, cluster: int, threads: int):
        _check(lib().f3r_batched_set_shape(self.h, cluster, threads), "f3r_batched_set_shape")

    def info(self) -> dict:
        """How the batch runs (f3r_batched_info)."""
        out = (C.c_int64 * 8)()
        _check(lib().f3r_batched_info(self.h, out), "f3r_batched_info")
        keys = ("cluster", "threads", "instances_launch", "instances_single", "rows_launch", "rows_single",
                "grid", "graph_launches")
        return {k: int(v) for k, v in zip(keys, out)}

    def wide_info(self) -> dict:
        """The wide teams of the last launch (f3r_batched_wide_info)."""
        out = (C.c_int64 * 4)()
        _check(lib().f3r_batched_wide_info(self.h, out), "f3r_batched_wide_info")
        return {k: int(v) for k, v in zip(("clusters_per_team", "teams", "instances", "rows"), out)}

    def autotune(self, B, X, stream=None) -> int:
        """Pick the team shape (cluster size, threads per block) by timing one
        outer iteration of the batch; returns the cluster size; X is zeroed."""
        bp = (C.c_void_p * self.ninst)(*[b.data_ptr() for b in B])
        xp = (C.c_void_p * self.ninst)(*[x.data_ptr() for x in X])
        ch = C.c_int()
        _check(lib().f3r_batched_autotune(self.h, bp, xp, C.byref(ch), _stream(stream)), "f3r_batched_autotune")
        return ch.value

    def solve(self, B, X, stream=None):
        """B, X: lists (one per instance) of device fp64 tensors; X holds x0."""
        assert len(B) == self.ninst and len(X) == self.ninst
        bp = (C.c_void_p * self.ninst)(*[b.data_ptr() for b in B])
        xp = (C.c_void_p * self.ninst)(*[x.data_ptr() for x in X])
        res = (BatchResult * self.ninst)()
        code = lib().f3r_solve_batched(self.h, bp, xp, res, _stream(stream))
        if code not in (OK, NOT_CONVERGED, ERR_NONFINITE):
            raise F3RError(code, "f3r_solve_batched")
        return code, list(res)

    @property
    def device_bytes(self) -> int:
        return lib().f3r_batched_device_bytes(self.h)

    def close(self):
        if self.h and _lib is not None:
            _lib.f3r_destroy_batched(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def arnoldi_training_pairs(rowptr, colidx, val, b, npairs: int, tol: float = 1e-10, stream=None):
    """Training pairs (r, e) for the learned preconditioner from the fp64
    solver's own vectors: the Arnoldi vectors v_0..v_{npairs-1} of one cycle
    of the outer fp64 FGMRES on A x = b (all levels fp64), mapped into the
    scaled system the Richardson level works in, r = D^-1/2 v, with e =
    A^^-1 r = D^1/2 A^-1 v from fp64 solves to `tol`.  Inputs are CUDA tensors
    (the CSR arrays and b); returns two (npairs, n) float32 CUDA tensors."""
    import torch

    n = len(rowptr) - 1
    dev = b.device
    rec = Solver(rowptr, colidx, val, preset("fp64-F3R", tol=1e-300, max_outer=npairs,
                                             m=[max(npairs, 1), 8, 4, 0]), stream=stream)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    rec.solve(b, x, stream=stream)  # npairs outer iterations, one cycle: V[0..npairs] kept
    d = torch.from_numpy(rec.export(0)).to(dev)  # D^-1/2
    V = torch.empty(npairs, n, dtype=torch.float64, device=dev)
    for k in range(npairs):
        rec.get_basis(0, k, V[k], stream=stream)
    rec.close()
    sol = Solver(rowptr, colidx, val, preset("fp64-F3R", tol=tol), stream=stream)
    R = torch.empty(npairs, n, dtype=torch.float32, device=dev)
    E = torch.empty(npairs, n, dtype=torch.float32, device=dev)
    for k in range(npairs):
        x.zero_()
        sol.solve(V[k], x, stream=stream)  # A x = v_k
        R[k] = (d * V[k]).float()
        E[k] = (x / d).float()
    sol.close()
    return R, E
