"""CPU oracle for the sparse linear-operator hot path (sequential but for the
SpMV row loops, which OpenMP may split over threads without changing any
result).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never imports,
links or calls it, and it shares no code with the CUDA path.

The arithmetic lives in ``gk_oracle.c`` (plain C, built with
``-ffp-contract=off`` so every fused multiply-add is an explicit ``fma``);
this module only builds it and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gk_oracle.c")
_HDR = os.path.join(_HERE, "gk_oracle.h")
_LIB = os.path.join(_HERE, "libgk_oracle.so")

STOP_NONE, STOP_CONVERGED, STOP_MAX_ITERS, STOP_BREAKDOWN, STOP_NAN = 0, 1, 2, 3, 4
PREC_NONE, PREC_SCALAR_JACOBI, PREC_BLOCK_JACOBI = 0, 1, 2
OK, ERR_ARG, ERR_SINGULAR = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libgk_oracle.so`` with gcc."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-fopenmp", "-o", tmp, _SRC, "-lm"]
    if subprocess.run(cmd).returncode != 0:
        # no OpenMP runtime: the same source, sequential
        subprocess.run([c for c in cmd if c != "-fopenmp"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Criteria(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int64), ("reduction_factor", ctypes.c_double),
                ("rel_to_b", ctypes.c_int32)]


class _Status(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("spmvs", ctypes.c_int64), ("rel_res", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("ref_norm", ctypes.c_double),
                ("stop_reason", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class _Precond(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("dinv", ctypes.c_void_p), ("blocks", ctypes.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        i64, f64, vp = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        L.or_csr_spmv.argtypes = [i64, vp, vp, vp, vp, f64, f64, vp]
        L.or_csr_spmv.restype = None
        L.or_csr_spmv_dot2.argtypes = [i64, vp, vp, vp, vp, vp, vp]
        L.or_csr_spmv_dot2.restype = None
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_set_threads.restype = ctypes.c_int
        L.or_dot.argtypes = [i64, vp, vp]
        L.or_dot.restype = f64
        L.or_norm2.argtypes = [i64, vp]
        L.or_norm2.restype = f64
        L.or_jacobi_scalar.argtypes = [i64, vp, vp, vp, vp]
        L.or_jacobi_scalar.restype = ctypes.c_int
        L.or_block_jacobi_size.argtypes = [i64, ctypes.c_int32]
        L.or_block_jacobi_size.restype = i64
        L.or_block_jacobi_generate.argtypes = [i64, vp, vp, vp, ctypes.c_int32, vp, vp]
        L.or_block_jacobi_generate.restype = ctypes.c_int
        L.or_precond_apply.argtypes = [i64, ctypes.POINTER(_Precond), vp, vp]
        L.or_precond_apply.restype = None
        L.or_hyb_width.argtypes = [i64, vp, i64, i64]
        L.or_hyb_width.restype = i64
        L.or_block_jacobi_precision.argtypes = [i64, vp, vp, vp, ctypes.c_int32, vp, vp, vp]
        L.or_block_jacobi_precision.restype = None
        L.or_ir_cg.argtypes = [i64, vp, vp, vp, ctypes.POINTER(_Precond), vp, vp, ctypes.POINTER(_Criteria),
                               f64, i64, ctypes.POINTER(_Status), ctypes.POINTER(i64)]
        L.or_ir_cg.restype = ctypes.c_int
        for name in ("or_cg_f32", "or_bicgstab_f32"):
            f = getattr(L, name)
            f.argtypes = [i64, vp, vp, vp, ctypes.c_int32, vp, vp, ctypes.POINTER(_Criteria),
                          ctypes.POINTER(_Status)]
            f.restype = ctypes.c_int
        L.or_gmres.argtypes = [i64, vp, vp, vp, ctypes.POINTER(_Precond), vp, vp, ctypes.POINTER(_Criteria),
                               ctypes.c_int32, ctypes.POINTER(_Status), vp]
        L.or_gmres.restype = ctypes.c_int
        for name in ("or_cg", "or_bicgstab", "or_cgs", "or_fcg"):
            f = getattr(L, name)
            f.argtypes = [i64, vp, vp, vp, ctypes.POINTER(_Precond), vp, vp,
                          ctypes.POINTER(_Criteria), ctypes.POINTER(_Status), vp]
            f.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


def _csr(A):
    rowptr, col, val = A
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    return rowptr, col, val


def spmv(A, x, alpha=1.0, beta=0.0, y=None):
    """``alpha*A@x + beta*y`` with the ordered row sum (Section 4.2)."""
    rowptr, col, val = _csr(A)
    n = rowptr.shape[0] - 1
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(n) if y is None else np.array(y, dtype=np.float64, copy=True)
    lib().or_csr_spmv(n, _p(rowptr), _p(col), _p(val), _p(x), float(alpha), float(beta), _p(out))
    return out


def spmv_accurate(A, x):
    """Dot2-accurate row sums and the bound ``(|A||x|)_i``."""
    rowptr, col, val = _csr(A)
    n = rowptr.shape[0] - 1
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(n)
    b = np.zeros(n)
    lib().or_csr_spmv_dot2(n, _p(rowptr), _p(col), _p(val), _p(x), _p(y), _p(b))
    return y, b


def set_threads(n: int = 0) -> int:
    """Threads of the SpMV row loops (0: all cores); returns the count in effect."""
    return int(lib().or_set_threads(int(n)))


def dot(x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib().or_dot(x.shape[0], _p(x), _p(y))


def norm2(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().or_norm2(x.shape[0], _p(x))


def jacobi_scalar(A):
    rowptr, col, val = _csr(A)
    n = rowptr.shape[0] - 1
    d = np.zeros(n)
    rc = lib().or_jacobi_scalar(n, _p(rowptr), _p(col), _p(val), _p(d))
    if rc != OK:
        raise ZeroDivisionError("zero or missing diagonal")
    return d


def block_jacobi(A, bs):
    """Inverse diagonal blocks (row-major, concatenated)."""
    rowptr, col, val = _csr(A)
    n = rowptr.shape[0] - 1
    blocks = np.zeros(max(1, lib().or_block_jacobi_size(n, bs)))
    bad = ctypes.c_int64(-1)
    rc = lib().or_block_jacobi_generate(n, _p(rowptr), _p(col), _p(val), bs, _p(blocks),
                                        ctypes.addressof(bad))
    if rc == ERR_SINGULAR:
        raise ZeroDivisionError(f"singular diagonal block {bad.value}")
    if rc != OK:
        raise ValueError("bad block size")
    return blocks[: lib().or_block_jacobi_size(n, bs)]


@dataclass
class Precond:
    kind: int = PREC_NONE
    block_size: int = 1
    dinv: np.ndarray | None = None
    blocks: np.ndarray | None = None

    def _c(self):
        return _Precond(self.kind, self.block_size, _p(self.dinv), _p(self.blocks))


def precond(A, kind: str = "none", block_size: int = 1) -> Precond:
    if kind == "none":
        return Precond()
    if kind == "jacobi":
        return Precond(PREC_SCALAR_JACOBI, 1, jacobi_scalar(A))
    if kind == "block_jacobi":
        return Precond(PREC_BLOCK_JACOBI, block_size, None, block_jacobi(A, block_size))
    raise ValueError(kind)


def precond_apply(P: Precond, r):
    r = np.ascontiguousarray(r, dtype=np.float64)
    z = np.zeros_like(r)
    c = P._c()
    lib().or_precond_apply(r.shape[0], ctypes.byref(c), _p(r), _p(z))
    return z


def hyb_width(A, vt=8, it=4):
    rowptr, _, _ = _csr(A)
    return int(lib().or_hyb_width(rowptr.shape[0] - 1, _p(rowptr), vt, it))


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    spmvs: int
    rel_res: float
    rel_res_true: float
    ref_norm: float
    stop_reason: int
    history: np.ndarray | None


def _solve(name, A, b, x0=None, P: Precond | None = None, max_iters=1000, tol=1e-10,
           rel_to_b=True, history=False):
    rowptr, col, val = _csr(A)
    n = rowptr.shape[0] - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    crit = _Criteria(int(max_iters), float(tol), 1 if rel_to_b else 0)
    st = _Status()
    P = P or Precond()
    pc = P._c()
    hist = np.full(int(max_iters) + 2, np.nan) if history else None
    rc = getattr(lib(), name)(n, _p(rowptr), _p(col), _p(val), ctypes.byref(pc), _p(b), _p(x),
                              ctypes.byref(crit), ctypes.byref(st), _p(hist))
    if rc != OK:
        raise RuntimeError(f"{name} failed: {rc}")
    if hist is not None:
        hist = hist[: st.iters + 1]
    return SolveResult(x, st.iters, st.spmvs, st.rel_res, st.rel_res_true, st.ref_norm,
                       st.stop_reason, hist)


def cg(A, b, **kw) -> SolveResult:
    return _solve("or_cg", A, b, **kw)


def bicgstab(A, b, **kw) -> SolveResult:
    return _solve("or_bicgstab", A, b, **kw)


def cgs(A, b, **kw) -> SolveResult:
    return _solve("or_cgs", A, b, **kw)


def fcg(A, b, **kw) -> SolveResult:
    return _solve("or_fcg", A, b, **kw)


def gmres(A, b, x0=None, P: Precond | None = None, max_iters=1000, tol=1e-10, rel_to_b=True, krylov_dim=30,
          history=False) -> SolveResult:
    """Restarted GMRES(krylov_dim) with right preconditioning."""
    rowptr, col, val = _csr(A)
    n = rowptr.shape[0] - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    crit = _Criteria(int(max_iters), float(tol), 1 if rel_to_b else 0)
    st = _Status()
    P = P or Precond()
    pc = P._c()
    hist = np.full(int(max_iters) + 2, np.nan) if history else None
    rc = lib().or_gmres(n, _p(rowptr), _p(col), _p(val), ctypes.byref(pc), _p(b), _p(x), ctypes.byref(crit),
                        int(krylov_dim), ctypes.byref(st), _p(hist))
    if rc != OK:
        raise RuntimeError(f"or_gmres failed: {rc}")
    if hist is not None:
        hist = hist[: st.iters + 1]
    return SolveResult(x, st.iters, st.spmvs, st.rel_res, st.rel_res_true, st.ref_norm, st.stop_reason, hist)


def block_jacobi_precision(A, bs, blocks):
    """Per-block storage precision (0 FP16, 1 FP32) and kappa_1 of the inverse blocks."""
    rowptr, col, val = _csr(A)
    n = rowptr.shape[0] - 1
    nb = (n + bs - 1) // bs
    prec = np.zeros(max(nb, 1), dtype=np.uint8)
    kappa = np.zeros(max(nb, 1))
    blocks = np.ascontiguousarray(blocks, dtype=np.float64)
    lib().or_block_jacobi_precision(n, _p(rowptr), _p(col), _p(val), bs, _p(blocks), _p(prec), _p(kappa))
    return prec[:nb], kappa[:nb]


def ir_cg(A, b, x0=None, P: Precond | None = None, max_iters=100000, tol=1e-10, rel_to_b=True,
          inner_reduction=1e-5, inner_max=None):
    """Mixed-precision iterative refinement; returns (SolveResult, outer steps)."""
    rowptr, col, val = _csr(A)
    n = rowptr.shape[0] - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    crit = _Criteria(int(max_iters), float(tol), 1 if rel_to_b else 0)
    st = _Status()
    P = P or Precond()
    pc = P._c()
    outer = ctypes.c_int64(0)
    rc = lib().or_ir_cg(n, _p(rowptr), _p(col), _p(val), ctypes.byref(pc), _p(b), _p(x), ctypes.byref(crit),
                        float(inner_reduction), int(inner_max or max_iters), ctypes.byref(st), ctypes.byref(outer))
    if rc != OK:
        raise RuntimeError(f"or_ir_cg failed: {rc}")
    return SolveResult(x, st.iters, st.spmvs, st.rel_res, st.rel_res_true, st.ref_norm, st.stop_reason,
                       None), outer.value


def _solve_f32(name, A, b, x0=None, jacobi=True, max_iters=1000, tol=1e-6, rel_to_b=True):
    rowptr, col, val = _csr(A)
    n = rowptr.shape[0] - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    crit = _Criteria(int(max_iters), float(tol), 1 if rel_to_b else 0)
    st = _Status()
    rc = getattr(lib(), name)(n, _p(rowptr), _p(col), _p(val), 1 if jacobi else 0, _p(b), _p(x),
                              ctypes.byref(crit), ctypes.byref(st))
    if rc != OK:
        raise RuntimeError(f"{name} failed: {rc}")
    return SolveResult(x, st.iters, st.spmvs, st.rel_res, st.rel_res_true, st.ref_norm, st.stop_reason, None)


def cg_f32(A, b, **kw) -> SolveResult:
    """CG in single precision (float values, vectors and sums)."""
    return _solve_f32("or_cg_f32", A, b, **kw)


def bicgstab_f32(A, b, **kw) -> SolveResult:
    """BiCGSTAB in single precision (float values, vectors and sums)."""
    return _solve_f32("or_bicgstab_f32", A, b, **kw)


def batch_system(sys_ptr, A, s):
    """Rows and columns [sys_ptr[s], sys_ptr[s+1]) of a block-diagonal CSR
    matrix as a CSR triple of its own (columns shifted to start at 0)."""
    rowptr, col, val = _csr(A)
    r0, r1 = int(sys_ptr[s]), int(sys_ptr[s + 1])
    k0, k1 = int(rowptr[r0]), int(rowptr[r1])
    return ((rowptr[r0:r1 + 1] - k0).astype(np.int32), (col[k0:k1] - r0).astype(np.int32),
            val[k0:k1].copy())


def batch_solve(sys_ptr, A, b, kind="cg", jacobi=True, dtype="f64", systems=None, x0=None, **kw):
    """Solve the independent systems one after another (each by cg /
    bicgstab, their FP32 forms, or ir_cg -- whose results carry the number
    of refinement steps as `.outer`).  Returns (x, list of SolveResult) over
    `systems` (default: all); entries of x outside those systems are left at
    x0."""
    n = int(sys_ptr[-1])
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    systems = range(len(sys_ptr) - 1) if systems is None else systems
    out = []
    for s in systems:
        r0, r1 = int(sys_ptr[s]), int(sys_ptr[s + 1])
        sub = batch_system(sys_ptr, A, s)
        if kind == "ir_cg":
            P = precond(sub, "jacobi") if jacobi else None
            res, outer = ir_cg(sub, b[r0:r1], x0=x[r0:r1], P=P, **kw)
            res.outer = outer
        elif dtype == "f32":
            f = cg_f32 if kind == "cg" else bicgstab_f32
            res = f(sub, b[r0:r1], x0=x[r0:r1], jacobi=jacobi, **kw)
        else:
            P = precond(sub, "jacobi") if jacobi else None
            f = cg if kind == "cg" else bicgstab
            res = f(sub, b[r0:r1], x0=x[r0:r1], P=P, **kw)
        x[r0:r1] = res.x
        out.append(res)
    return x, out
