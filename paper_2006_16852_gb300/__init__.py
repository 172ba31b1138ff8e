"""Python binding of the GB300 sparse linear-operator library (``libgk.so``).

The functions mirror the C ABI of ``include/gk.h`` one to one and only
marshal arguments: every step of the computation runs in the library's CUDA
kernels.  Vectors may be torch CUDA tensors (the usual case; their data
pointers are passed through) or host arrays (numpy or CPU tensors), which the
library stages itself.  Work goes to the current torch CUDA stream unless a
stream is given.

There is no fallback: ``load()`` raises if ``libgk.so`` has not been built
(``python -m paper_2006_16852_gb300.build`` or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgk.so")

OK = 0
ERR_NAMES = {1: "GK_ERR_ARG", 2: "GK_ERR_DIM", 3: "GK_ERR_DTYPE", 4: "GK_ERR_NOT_DEVICE",
             5: "GK_ERR_CSR", 6: "GK_ERR_FORMAT", 7: "GK_ERR_SINGULAR", 8: "GK_ERR_UNSUPPORTED",
             9: "GK_ERR_CUDA", 10: "GK_ERR_ALLOC", 11: "GK_ERR_TIMEOUT"}
F64, F32 = 0, 1
FORMATS = {"csr": 0, "csr_merge": 1, "ell": 2, "hyb": 3, "auto": 4}
FORMAT_NAMES = {v: k for k, v in FORMATS.items()}
SOLVERS = {"cg": 0, "bicgstab": 1, "ir_cg": 2, "fcg": 3, "cgs": 4, "gmres": 5}
STOP_NONE, STOP_CONVERGED, STOP_MAX_ITERS, STOP_BREAKDOWN, STOP_NAN, STOP_TIME = range(6)

# every symbol include/gk.h declares
EXPORTS = ("gk_last_error", "gk_version", "gk_matrix_create_csr", "gk_matrix_get_info",
           "gk_matrix_destroy", "gk_apply", "gk_apply_adv", "gk_apply_dot", "gk_precond_generate", "gk_precond_apply",
           "gk_precond_get_blocks", "gk_precond_destroy", "gk_solver_generate", "gk_solve",
           "gk_solver_destroy", "gk_solver_get_info", "gk_batch_create", "gk_batch_solve",
           "gk_batch_autotune", "gk_batch_set_threads", "gk_batch_get_info", "gk_batch_destroy",
           "gk_wsnet_create", "gk_wsnet_num_params", "gk_wsnet_set_params", "gk_wsnet_get_params",
           "gk_wsnet_set_loss",
           "gk_wsnet_forward", "gk_wsnet_gradients", "gk_wsnet_train_step", "gk_wsnet_infer_bf16",
           "gk_wsnet_check",
           "gk_wsnet_features", "gk_wsnet_warm_start", "gk_wsnet_destroy", "gk_dot", "gk_dot_noalloc", "gk_gather_dot", "gk_fp64_rate",
           "gk_wait_selftest")
BATCH_CLASSES = 8
BATCH_BLOCK_SIZES = (32, 64, 128, 256)


class GkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Criteria(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int64), ("reduction_factor", ctypes.c_double),
                ("rel_to_b", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("time_limit_s", ctypes.c_double), ("inner_reduction", ctypes.c_double),
                ("inner_max_iters", ctypes.c_int32), ("krylov_dim", ctypes.c_int32)]


class Status(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("spmvs", ctypes.c_int64), ("rel_res", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("ref_norm", ctypes.c_double),
                ("stop_reason", ctypes.c_int32), ("device_error", ctypes.c_int32),
                ("outer_iters", ctypes.c_int64), ("form", ctypes.c_int32), ("idle_iters", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SolverInfo(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("inner_format", ctypes.c_int32), ("n", ctypes.c_int64),
                ("inner_fp16_blocks", ctypes.c_int64), ("inner_fp32_blocks", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64)]


class BatchStatus(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("stop_reason", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("outer_iters", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class MatrixInfo(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("format", ctypes.c_int32), ("dtype", ctypes.c_int32), ("ell_width", ctypes.c_int64),
                ("tail_rows", ctypes.c_int64), ("tail_nnz", ctypes.c_int64),
                ("short_items", ctypes.c_int64), ("long_rows", ctypes.c_int64), ("tiles", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("spmv_bytes", ctypes.c_int64), ("split_rows", ctypes.c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["format_name"] = FORMAT_NAMES.get(self.format, str(self.format))
        return d


_lib = None


def load(path: str | None = None):
    """Load ``libgk.so`` and declare the C signatures.  Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                          "(the library has no CPU fallback)")
    L = ctypes.CDLL(path)
    vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    L.gk_last_error.restype = ctypes.c_char_p
    L.gk_last_error.argtypes = []
    L.gk_version.restype = i32
    L.gk_version.argtypes = []
    sig = {
        "gk_matrix_create_csr": [i64, i64, i64, vp, vp, vp, i32, i32, vp, ctypes.POINTER(vp)],
        "gk_matrix_get_info": [vp, ctypes.POINTER(MatrixInfo)],
        "gk_matrix_destroy": [vp],
        "gk_apply": [vp, vp, vp, vp],
        "gk_apply_adv": [f64, vp, vp, f64, vp, vp],
        "gk_apply_dot": [vp, vp, vp, vp, vp, vp],
        "gk_precond_generate": [vp, i32, vp, ctypes.POINTER(vp)],
        "gk_precond_apply": [vp, vp, vp, vp],
        "gk_precond_get_blocks": [vp, vp, i64, vp],
        "gk_precond_destroy": [vp],
        "gk_solver_generate": [vp, vp, i32, ctypes.POINTER(Criteria), ctypes.POINTER(vp)],
        "gk_solve": [vp, vp, vp, ctypes.POINTER(Status), vp],
        "gk_solver_destroy": [vp],
        "gk_solver_get_info": [vp, ctypes.POINTER(SolverInfo)],
        "gk_batch_create": [i64, vp, i64, vp, vp, vp, i32, vp, ctypes.POINTER(vp)],
        "gk_batch_solve": [vp, i32, i32, ctypes.POINTER(Criteria), vp, vp, vp, vp],
        "gk_batch_autotune": [vp, i32, i32, ctypes.POINTER(Criteria), vp, vp, vp, vp],
        "gk_batch_set_threads": [vp, i32, i32, vp],
        "gk_batch_get_info": [vp, i32, i32, vp, vp, vp],
        "gk_batch_destroy": [vp],
        "gk_wsnet_create": [i32, i32, i32, vp, ctypes.POINTER(vp)],
        "gk_wsnet_num_params": [vp, ctypes.POINTER(i64)],
        "gk_wsnet_set_params": [vp, vp, vp],
        "gk_wsnet_get_params": [vp, vp, vp],
        "gk_wsnet_set_loss": [vp, i32],
        "gk_wsnet_forward": [vp, i32, vp, vp, vp],
        "gk_wsnet_gradients": [vp, i32, vp, vp, vp, vp, vp],
        "gk_wsnet_train_step": [vp, i32, vp, vp, ctypes.c_float, vp, vp],
        "gk_wsnet_infer_bf16": [vp, i32, vp, vp, vp],
        "gk_wsnet_check": [vp, vp],
        "gk_wsnet_features": [vp, vp, vp, vp, f64, vp, vp, vp],
        "gk_wsnet_warm_start": [vp, vp, vp, vp, f64, vp, vp],
        "gk_wsnet_destroy": [vp],
        "gk_dot": [i64, vp, vp, vp, vp],
        "gk_dot_noalloc": [i64, vp, vp, vp, vp],
        "gk_gather_dot": [i64, vp, vp, vp, i64, vp, vp],
        "gk_fp64_rate": [i64, vp, vp],
        "gk_wait_selftest": [vp, vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib = L
    return L


def lib():
    return load()


def _check(rc: int):
    if rc != OK:
        raise GkError(rc, lib().gk_last_error().decode(errors="replace"))


def _ptr(a) -> int:
    """Data pointer of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream, *arrays) -> int:
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    for a in arrays:
        if getattr(a, "is_cuda", False):
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return 0


def _check_vec(a, n: int, name: str, dtype_bits: int = 64):
    if a is None:
        raise ValueError(f"{name} is None")
    size = a.numel() if hasattr(a, "numel") else a.size
    if size != n:
        raise GkError(2, f"{name} has {size} entries, expected {n}")
    dt = str(a.dtype)
    if "float64" not in dt:
        raise GkError(3, f"{name} must be float64, got {dt}")


class Matrix:
    """A CSR operator (library-owned copy) in one of the storage formats."""

    def __init__(self, rowptr, col, val, n_cols: int | None = None, fmt: str = "csr", stream=None):
        n_rows = (rowptr.numel() if hasattr(rowptr, "numel") else rowptr.size) - 1
        nnz = col.numel() if hasattr(col, "numel") else col.size
        n_cols = n_rows if n_cols is None else int(n_cols)
        for a, want in ((rowptr, "int32"), (col, "int32"), (val, "float64")):
            if want not in str(a.dtype):
                raise GkError(3, f"CSR arrays must be int32/int32/float64, got {a.dtype}")
        h = ctypes.c_void_p()
        _check(lib().gk_matrix_create_csr(n_rows, n_cols, nnz, _ptr(rowptr), _ptr(col), _ptr(val), F64,
                                          FORMATS[fmt], _stream(stream, rowptr, col, val),
                                          ctypes.byref(h)))
        self.handle = h
        self.n_rows, self.n_cols, self.nnz = n_rows, n_cols, nnz

    def info(self) -> dict:
        inf = MatrixInfo()
        _check(lib().gk_matrix_get_info(self.handle, ctypes.byref(inf)))
        return inf.as_dict()

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.gk_matrix_destroy(h)
            self.handle = None


def apply(A: Matrix, b, x, stream=None):
    """x = A b (Section 4.2)."""
    _check_vec(b, A.n_cols, "b")
    _check_vec(x, A.n_rows, "x")
    _check(lib().gk_apply(A.handle, _ptr(b), _ptr(x), _stream(stream, b, x)))
    return x


def apply_dot(A: Matrix, b, x, u, result, stream=None):
    """x = A b and result[0] = u . x in one fused pass (device tensors)."""
    _check_vec(b, A.n_cols, "b")
    _check_vec(x, A.n_rows, "x")
    _check_vec(u, A.n_rows, "u")
    _check(lib().gk_apply_dot(A.handle, _ptr(b), _ptr(x), _ptr(u), _ptr(result), _stream(stream, b, x, u)))
    return result


def apply_adv(alpha: float, A: Matrix, b, beta: float, x, stream=None):
    """x = alpha A b + beta x (Section 4.2)."""
    _check_vec(b, A.n_cols, "b")
    _check_vec(x, A.n_rows, "x")
    _check(lib().gk_apply_adv(float(alpha), A.handle, _ptr(b), float(beta), _ptr(x), _stream(stream, b, x)))
    return x


class Precond:
    """Jacobi (block_size 1) or block-Jacobi (2..32) preconditioner of A."""

    def __init__(self, A: Matrix, block_size: int = 1, stream=None):
        h = ctypes.c_void_p()
        _check(lib().gk_precond_generate(A.handle, int(block_size), _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.n = A.n_rows
        self.block_size = int(block_size)

    def blocks(self, stream=None):
        import numpy as np
        bs, n = self.block_size, self.n
        total = n if bs == 1 else (n // bs) * bs * bs + (n % bs) ** 2
        out = np.zeros(max(total, 1))
        _check(lib().gk_precond_get_blocks(self.handle, out.ctypes.data, out.size, _stream(stream)))
        return out[:total]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.gk_precond_destroy(h)
            self.handle = None


def precond_generate(A: Matrix, block_size: int = 1, stream=None) -> Precond:
    return Precond(A, block_size, stream)


def precond_apply(P: Precond, r, z, stream=None):
    """z = M^{-1} r."""
    _check_vec(r, P.n, "r")
    _check_vec(z, P.n, "z")
    _check(lib().gk_precond_apply(P.handle, _ptr(r), _ptr(z), _stream(stream, r, z)))
    return z


@dataclass
class SolveStatus:
    iters: int
    spmvs: int
    rel_res: float
    rel_res_true: float
    ref_norm: float
    stop_reason: int
    device_error: int
    outer_iters: int
    form: int = 0
    idle_iters: int = 0


FORM_GRAPH, FORM_HOST, FORM_CLUSTER, FORM_GRID = 0, 1, 2, 3


class Solver:
    """Krylov solver operator S_A bound to A (Section 3.1): kind cg, bicgstab,
    fcg, cgs, gmres, or ir_cg (mixed-precision refinement)."""

    def __init__(self, A: Matrix, P: Precond | None = None, kind: str = "cg", max_iters: int = 1000,
                 reduction_factor: float = 1e-10, rel_to_b: bool = True, check_every: int = 0,
                 time_limit_s: float = 0.0, inner_reduction: float = 0.0, inner_max_iters: int = 0,
                 krylov_dim: int = 0):
        crit = Criteria(int(max_iters), float(reduction_factor), 1 if rel_to_b else 0, int(check_every),
                        float(time_limit_s), float(inner_reduction), int(inner_max_iters), int(krylov_dim))
        h = ctypes.c_void_p()
        _check(lib().gk_solver_generate(A.handle, P.handle if P is not None else None, SOLVERS[kind],
                                        ctypes.byref(crit), ctypes.byref(h)))
        self.handle = h
        self.n = A.n_rows
        self._keep = (A, P)

    def info(self) -> dict:
        inf = SolverInfo()
        _check(lib().gk_solver_get_info(self.handle, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in SolverInfo._fields_}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.gk_solver_destroy(h)
            self.handle = None


def solver_generate(A: Matrix, P: Precond | None = None, kind: str = "cg", **criteria) -> Solver:
    return Solver(A, P, kind, **criteria)


def solve(S: Solver, b, x, stream=None) -> SolveStatus:
    """x = S_A(b); x holds the initial guess on entry (Section 2.1)."""
    _check_vec(b, S.n, "b")
    _check_vec(x, S.n, "x")
    st = Status()
    _check(lib().gk_solve(S.handle, _ptr(b), _ptr(x), ctypes.byref(st), _stream(stream, b, x)))
    return SolveStatus(**{f: getattr(st, f) for f, _ in Status._fields_})


def dot(x, y, result, stream=None):
    """result[0] = x . y with a reproducible reduction order (device tensors)."""
    n = x.numel()
    _check_vec(y, n, "y")
    _check(lib().gk_dot(n, _ptr(x), _ptr(y), _ptr(result), _stream(stream, x, y, result)))
    return result


def dot_noalloc(x, y, result, stream=None):
    """As dot(), through the entry point that allocates no device memory."""
    n = x.numel()
    _check_vec(y, n, "y")
    _check(lib().gk_dot_noalloc(n, _ptr(x), _ptr(y), _ptr(result), _stream(stream, x, y, result)))
    return result


def gather_dot(c, v, x, result, stream=None):
    """result[0] = sum_k v[k] x[c[k]] (device tensors; c int32): the SpMV's
    per-entry work without its rows, the gather ceiling of the SpMV kernels."""
    n = c.numel()
    _check_vec(v, n, "v")
    _check(lib().gk_gather_dot(n, _ptr(c), _ptr(v), _ptr(x), x.numel(), _ptr(result),
                               _stream(stream, c, v, x, result)))
    return result


def fp64_rate(iters: int = 20000, stream=None) -> float:
    """The device's measured FP64 fused multiply-add rate in TFLOP/s."""
    r = ctypes.c_double(0.0)
    _check(lib().gk_fp64_rate(iters, ctypes.byref(r), _stream(stream)))
    return r.value


def wait_selftest(stream=None) -> int:
    """Runs one bounded device-side wait that nothing satisfies; returns the
    device error word it leaves (1: the wait gave up, as designed)."""
    err = ctypes.c_int32(-1)
    _check(lib().gk_wait_selftest(ctypes.byref(err), _stream(stream)))
    return err.value


class Batch:
    """Independent small systems in one block-diagonal CSR matrix (``sys_ptr``:
    numpy int64 offsets of the systems' first rows, n_sys + 1 entries)."""

    def __init__(self, sys_ptr, rowptr, col, val, dtype: str = "f64", stream=None):
        import numpy as np
        sp = np.ascontiguousarray(np.asarray(sys_ptr, dtype=np.int64))
        for a, want in ((rowptr, "int32"), (col, "int32"), (val, "float64")):
            if want not in str(a.dtype):
                raise GkError(3, f"CSR arrays must be int32/int32/float64, got {a.dtype}")
        nnz = col.numel() if hasattr(col, "numel") else col.size
        h = ctypes.c_void_p()
        _check(lib().gk_batch_create(sp.size - 1, sp.ctypes.data, nnz, _ptr(rowptr), _ptr(col), _ptr(val),
                                     F32 if dtype == "f32" else F64, _stream(stream, rowptr, col, val),
                                     ctypes.byref(h)))
        self.handle = h
        self.sys_ptr = sp
        self.n_sys = sp.size - 1
        self.n_rows = int(sp[-1])
        self.nnz = nnz

    @staticmethod
    def _crit(max_iters, reduction_factor, rel_to_b, inner_reduction=0.0, inner_max_iters=0):
        return Criteria(int(max_iters), float(reduction_factor), 1 if rel_to_b else 0, 0, 0.0,
                        float(inner_reduction), int(inner_max_iters), 0)

    def solve(self, b, x, kind: str = "cg", jacobi: bool = True, max_iters: int = 1000,
              reduction_factor: float = 1e-10, rel_to_b: bool = True, status: bool = True,
              inner_reduction: float = 0.0, inner_max_iters: int = 0, stream=None):
        """Solve every system (x: initial guesses in, solutions out); kind cg,
        bicgstab or ir_cg.  Returns a dict of numpy arrays (iters,
        stop_reason, rel_res, outer_iters) when status."""
        import numpy as np
        _check_vec(b, self.n_rows, "b")
        _check_vec(x, self.n_rows, "x")
        crit = self._crit(max_iters, reduction_factor, rel_to_b, inner_reduction, inner_max_iters)
        st = (BatchStatus * self.n_sys)() if status else None
        _check(lib().gk_batch_solve(self.handle, SOLVERS[kind], 1 if jacobi else 0, ctypes.byref(crit),
                                    _ptr(b), _ptr(x), ctypes.addressof(st) if status else None,
                                    _stream(stream, b, x)))
        if not status:
            return None
        raw = np.frombuffer(st, dtype=np.dtype([("iters", np.int32), ("stop_reason", np.int32),
                                                ("rel_res", np.float64), ("outer_iters", np.int32),
                                                ("reserved_", np.int32)]))
        return {k: raw[k].copy() for k in ("iters", "stop_reason", "rel_res", "outer_iters")}

    def autotune(self, b, kind: str = "cg", jacobi: bool = True, max_iters: int = 1000,
                 reduction_factor: float = 1e-10, rel_to_b: bool = True, inner_reduction: float = 0.0,
                 inner_max_iters: int = 0, stream=None):
        """Time block sizes 32/64/128/256 per size class and keep the fastest.
        Returns (chosen sizes per class, {class: {size: ms}}) over non-empty classes."""
        _check_vec(b, self.n_rows, "b")
        crit = self._crit(max_iters, reduction_factor, rel_to_b, inner_reduction, inner_max_iters)
        t = (ctypes.c_int32 * BATCH_CLASSES)()
        ms = (ctypes.c_double * (4 * BATCH_CLASSES))()
        _check(lib().gk_batch_autotune(self.handle, SOLVERS[kind], 1 if jacobi else 0, ctypes.byref(crit),
                                       _ptr(b), ctypes.addressof(t), ctypes.addressof(ms), _stream(stream, b)))
        chosen = list(t)
        times = {c: dict(zip(BATCH_BLOCK_SIZES, list(ms)[4 * c:4 * c + 4]))
                 for c in range(BATCH_CLASSES) if chosen[c]}
        return chosen, times

    def set_threads(self, threads, kind: str = "cg", jacobi: bool = True):
        """Block size per size class (0 = built-in default)."""
        t = (ctypes.c_int32 * BATCH_CLASSES)(*[int(v) for v in threads])
        _check(lib().gk_batch_set_threads(self.handle, SOLVERS[kind], 1 if jacobi else 0, ctypes.addressof(t)))

    def info(self, kind: str = "cg", jacobi: bool = True) -> dict:
        cnt, nmax, thr = ((ctypes.c_int32 * BATCH_CLASSES)() for _ in range(3))
        _check(lib().gk_batch_get_info(self.handle, SOLVERS[kind], 1 if jacobi else 0, ctypes.addressof(cnt),
                                       ctypes.addressof(nmax), ctypes.addressof(thr)))
        return {"counts": list(cnt), "nmax": list(nmax), "threads": list(thr)}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.gk_batch_destroy(h)
            self.handle = None


WSNET_DILATIONS = (1, 2, 4, 8, 16, 32)


class WsNet:
    """The warm-start network (see gk_wsnet_* in include/gk.h).  Tensors are
    torch CUDA float32 (inputs (B, 2, H, W), outputs (B, 1, H, W)); parameter
    vectors are numpy float32 on the host."""

    def __init__(self, H: int, W: int, batch_max: int = 16, dilations=WSNET_DILATIONS):
        d = (ctypes.c_int32 * 6)(*[int(v) for v in dilations])
        h = ctypes.c_void_p()
        _check(lib().gk_wsnet_create(int(H), int(W), int(batch_max), ctypes.addressof(d), ctypes.byref(h)))
        self.handle = h
        self.H, self.W, self.batch_max = int(H), int(W), int(batch_max)
        self.dilations = tuple(int(v) for v in dilations)
        n = ctypes.c_int64()
        _check(lib().gk_wsnet_num_params(h, ctypes.byref(n)))
        self.nparams = n.value

    def set_params(self, params, stream=None):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.nparams:
            raise GkError(2, f"expected {self.nparams} parameters, got {p.size}")
        _check(lib().gk_wsnet_set_params(self.handle, p.ctypes.data, _stream(stream)))

    def set_loss(self, kind: str):
        """'mse' or 'energy' (the A-norm of the error)."""
        _check(lib().gk_wsnet_set_loss(self.handle, {"mse": 0, "energy": 1}[kind]))

    def get_params(self, stream=None):
        import numpy as np
        p = np.empty(self.nparams, dtype=np.float32)
        _check(lib().gk_wsnet_get_params(self.handle, p.ctypes.data, _stream(stream)))
        return p

    def _bx(self, x):
        if x.dim() != 4 or tuple(x.shape[1:]) != (2, self.H, self.W) or x.dtype.__str__() != "torch.float32":
            raise GkError(2, f"input must be float32 (B, 2, {self.H}, {self.W}), got {tuple(x.shape)} {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("input must be contiguous")
        return x.shape[0]

    def forward(self, x, y, stream=None):
        B = self._bx(x)
        _check(lib().gk_wsnet_forward(self.handle, B, _ptr(x), _ptr(y), _stream(stream, x, y)))
        return y

    def gradients(self, x, target, stream=None):
        """(loss, flat gradient as numpy float32)."""
        import numpy as np
        B = self._bx(x)
        loss = ctypes.c_float()
        g = np.empty(self.nparams, dtype=np.float32)
        _check(lib().gk_wsnet_gradients(self.handle, B, _ptr(x), _ptr(target), ctypes.addressof(loss), g.ctypes.data,
                                        _stream(stream, x, target)))
        return loss.value, g

    def train_step(self, x, target, lr: float, loss_out=None, stream=None):
        """One Adam step; loss_out: optional device float32 tensor of one element."""
        B = self._bx(x)
        _check(lib().gk_wsnet_train_step(self.handle, B, _ptr(x), _ptr(target), float(lr),
                                         _ptr(loss_out) if loss_out is not None else None,
                                         _stream(stream, x, target)))

    def infer_bf16(self, x, y, stream=None):
        B = self._bx(x)
        _check(lib().gk_wsnet_infer_bf16(self.handle, B, _ptr(x), _ptr(y), _stream(stream, x, y)))
        return y

    def check(self, stream=None):
        """Waits for the stream; raises GkError (GK_ERR_TIMEOUT) if a
        tensor-core completion wait of an inference gave up."""
        _check(lib().gk_wsnet_check(self.handle, _stream(stream)))

    def features(self, g, b, feat, x=None, target=None, out_scale: float = 1.0, stream=None):
        _check(lib().gk_wsnet_features(self.handle, _ptr(g), _ptr(b), _ptr(x), float(out_scale), _ptr(feat),
                                       _ptr(target), _stream(stream, g, b)))

    def warm_start(self, g, b, x0, out_scale: float, A: Matrix | None = None, stream=None):
        """x0 = the network's prediction (scaled by the A-norm-optimal factor when A is given)."""
        _check(lib().gk_wsnet_warm_start(self.handle, A.handle if A is not None else None, _ptr(g), _ptr(b),
                                         float(out_scale), _ptr(x0), _stream(stream, g, b, x0)))
        return x0

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.gk_wsnet_destroy(h)
            self.handle = None
