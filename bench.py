#!/usr/bin/env python
"""Benchmark of the sparse linear-operator hot path on one GB300 (or N replicas).

One step is one pass of the whole path over the "SpMV and FP64 CG sweep"
workload:

  (a) 27-point stencil on a 128^3 grid (n = 2,097,152, nnz = 55,742,968)
  (b) power-law matrix, n = 1,000,000, row lengths Zipf(1.8) capped at 10^4,
      symmetrised and made diagonally dominant (nnz ~ 29M)

  * SpMV x -> A x three times back to back in every format: (a) CSR-binned,
    CSR-merge, ELL, HYB; (b) CSR-merge, HYB, CSR-binned (ELL refuses (b):
    padding > 8x nnz)
  * preconditioner generation: scalar Jacobi and block Jacobi (bs 8) of (a),
    block Jacobi (bs 4) of (b)
  * (a) CG to ||r|| <= 1e-10 ||b|| from x0 = 0, b = A x*: plain FP64 CG
    (CSR), Jacobi-CG and block-Jacobi-CG (ELL), and the mixed-precision forms
    (FP64 refinement around FP32 CG with Jacobi or adaptive FP16/FP32 block
    Jacobi); "chosen form" = the fastest of the preconditioned/mixed forms
  * (b) Jacobi-CG and block-Jacobi BiCGSTAB to 1e-10 (HYB)

value = algorithmic bytes of the step / device time of the step (GB/s).

Beside the step (not part of its value) the line carries "mixed": the
mixed-precision workload (7-point variable-coefficient diffusion on 256^3,
log-normal sigma 1) solved to 1e-12 by plain FP64 CG and by FP64 refinement
around FP32 CG with Jacobi or adaptive FP16/FP32 block Jacobi; and
"learned": CG to 1e-10 on held-out 256x256 random-coefficient diffusion
problems from the trained network's x0 and from zero; and "batched": 10,000
small variable-coefficient systems solved per system in one graph launch
(FP64 CG / BiCGSTAB / refinement to 1e-10, FP32 CG / BiCGSTAB to 1e-6), with
solves/s and the time against plain FP64 CG on the block-diagonal matrix;
"krylov": BiCGSTAB, CGS and GMRES on a convection-diffusion matrix, CG, FCG
and GMRES on (a), to 1e-10; "latency": CG on Poisson-2D 64^2 (and 256^2) in
every form -- the one-launch cluster (or cooperative-grid) form, the graph,
host-checked loops -- per iteration; "stream": the library's reduction
kernel against a device copy and the STREAM triad; "paper_bandwidth": the
paper's solver-bandwidth experiment (Section 7.3) on this GPU -- the five
Krylov solvers unpreconditioned for a fixed iteration count on (a), bytes
from the paper's Table 2 model and from this library's own, against the
triad; "paper_context": the paper's own numbers with their GPUs (Tables 1-3),
context only.
Inputs are larger than the 129 MB L2 (711 MB and ~371 MB per SpMV).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV GB/s (% HBM peak); time to 1e-10 residual, chosen form vs plain FP64 CG"
UNIT = "GB/s"
WORKLOAD = ("SpMV + Krylov sweep, FP64 values / int32 indices: (a) 27-point stencil 128^3 "
            "(n=2,097,152, nnz=55,742,968), (b) power-law Zipf(1.8) cap 1e4, n=1,000,000, symmetrised, "
            "diagonally dominant")

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel per launch on workload (a); valid only while the ELL
# kernel's source (spmv_source_hash) is the one it was measured on.
NCU_TRAFFIC = {"f9e3c748108c7546": {"dot": 714036992}}

# nominal GB300 rates (context beside the measured peaks)
NOMINAL_HBM_GBS = 7900.0
NOMINAL_FP64_TFLOPS = 1.25

# back-to-back applies per format and matrix in one step (the per-launch time
# of the roofline is their average)
SPMV_REPS = 3


# ---------------------------------------------------------------------------
# algorithmic byte model (value 8 B, index 4 B; a gathered vector is counted
# once, as if it stayed in L2 after its first use; padding is not counted).
# The stored operator's bytes depend on the format:
#   CSR (binned and merge-path): nnz (VT + IT) + (n + 1) IT
#   ELL:                          nnz (VT + IT)
#   HYB:                          nnz_ell (VT + IT) + nnz_coo (VT + 2 IT)
# ---------------------------------------------------------------------------

def infer_bytes_per_pixel(width=32, layers=6):
    """Compulsory bytes per pixel of one warm-start inference as the library
    runs it: the two FP32 input features read once, each hidden BF16
    activation but the last (width channels, layers - 2 of them) written
    once and read once, the nine FP32 tap planes into which the last hidden
    layer folds the one-channel output layer written once and read once,
    and the FP32 output written once (weights are a few KB and stay in
    cache)."""
    return 2 * 4 + (layers - 2) * width * 2 * 2 + 9 * 4 * 2 + 4


def matrix_bytes(nnz, n_rows, fmt="csr", tail_nnz=0, vt=8, it=4):
    if fmt in ("csr", "csr_merge"):
        return nnz * (vt + it) + (n_rows + 1) * it
    if fmt == "ell":
        return nnz * (vt + it)
    if fmt == "hyb":
        return (nnz - tail_nnz) * (vt + it) + tail_nnz * (vt + 2 * it)
    raise ValueError(fmt)


def spmv_bytes(nnz, n_rows, n_cols, beta=False, fmt="csr", tail_nnz=0):
    return matrix_bytes(nnz, n_rows, fmt, tail_nnz) + n_cols * 8 + n_rows * 8 + (n_rows * 8 if beta else 0)


def resid_bytes(nnz, n, fmt="csr", tail_nnz=0):  # r = b - A x with ||r||, ||b||
    return spmv_bytes(nnz, n, n, fmt=fmt, tail_nnz=tail_nnz) + 8 * n


def prec_extra(prec, bs):
    """Bytes per row one preconditioner apply reads beyond its input vector."""
    if prec == "none":
        return 0
    if prec == "jacobi":
        return 8
    return 8 * bs


def cg_bytes(iters, nnz, n, prec="none", bs=1, fmt="csr", tail_nnz=0):
    pe = prec_extra(prec, bs)
    rb = resid_bytes(nnz, n, fmt, tail_nnz)
    setup = rb + (16 + pe) * n
    z_store = 8 if prec == "block" else 0
    # K1: SpMV q = A p (p.q in the epilogue); K2: x, p, q, r (+M) in, x, r (+z) out;
    # K3: p, r or z (+dinv) in, p out
    k2 = (32 + pe + 16 + z_store) * n
    k3 = (24 + (8 if prec == "jacobi" else 0)) * n
    per_it = spmv_bytes(nnz, n, n, fmt=fmt, tail_nnz=tail_nnz) + k2 + k3
    return setup + iters * per_it + rb


def bicgstab_bytes(iters, spmvs, nnz, n, prec="none", bs=1, fmt="csr", tail_nnz=0):
    pe = prec_extra(prec, bs)
    hat = 0 if prec == "none" else 8
    full = (spmvs - 2 - iters)  # SpMVs of full iterations beyond one per iteration
    half = iters - full         # iterations that ended at the half step
    rb = resid_bytes(nnz, n, fmt, tail_nnz)
    sb = spmv_bytes(nnz, n, n, fmt=fmt, tail_nnz=tail_nnz)
    setup = rb + 32 * n
    k1 = (24 + pe + 8 + hat) * n
    k3 = (16 + pe + 8 + hat) * n
    k5 = 64 * n
    full_it = 2 * sb + 16 * n + k1 + k3 + k5
    half_it = sb + 8 * n + k1 + k3 + 40 * n
    return setup + full * full_it + half * half_it + rb


def ir_bytes(inner, outer, nnz, n, prec="none", bs=1, fp16_frac=0.0, fmt="csr", tail_nnz=0):
    """FP64 refinement around an FP32 CG inner solve (GK_IR_CG).

    Outer step: r = b - A x in FP64 (SpMV + b), the start of the inner solve
    (r64 in; r32, d32, p32 out; M), and x += ||r|| d (x in/out, d in).  Inner
    iteration: FP32 SpMV (FP32 values, the same indices, x and y in FP32),
    update (d, p, q, r, M in; d, r out), direction (p, r or z, M in; p out);
    with block Jacobi d's update is in the direction step instead (update: q,
    r, M in; r, z out; direction: p, d, z in; p, d out).  Block-Jacobi
    blocks cost 2 (FP16) or 4 (FP32) bytes per entry."""
    if prec == "none":
        pe = 0.0
    elif prec == "jacobi":
        pe = 4.0
    else:
        pe = bs * (2.0 * fp16_frac + 4.0 * (1.0 - fp16_frac))
    spmv32 = matrix_bytes(nnz, n, fmt, tail_nnz, vt=4) + n * 4 + n * 4
    if prec == "block":
        per_inner = spmv32 + (8 + pe + 8) * n + (12 + 8) * n
    else:
        per_inner = spmv32 + (16 + pe + 8) * n + (12 + (4 if prec == "jacobi" else 0)) * n
    rb = resid_bytes(nnz, n, fmt, tail_nnz)
    per_outer = rb + (8 + 12 + pe) * n + 20 * n
    return int(outer * per_outer + inner * per_inner + rb)


def bj_out_elems(n, bs):
    """Doubles of the generated preconditioner: n (scalar) or the inverse blocks."""
    if bs == 1:
        return n
    full, last = divmod(n, bs)
    return full * bs * bs + last * last


def in_block_entries(A, bs):
    """Stored entries of A inside its diagonal blocks of bs rows (the diagonal for bs = 1)."""
    rowptr, col, _ = A
    rows = np.repeat(np.arange(rowptr.size - 1, dtype=np.int64), np.diff(rowptr))
    return int(np.count_nonzero(rows // bs == col.astype(np.int64) // bs))


def precond_bytes(n, bs, in_block):
    """Preconditioner generation: the row pointers, one 32-byte sector of
    column indices per row for the binary search that locates the row's
    entries inside its block (they are a contiguous run of the sorted
    columns), those entries (value + index), and the inverse written."""
    return (n + 1) * 4 + 32 * n + in_block * 12 + 8 * bj_out_elems(n, bs)


def precond_fp64_ops(n, bs):
    """FP64 operation slots of the generation: bs^3 - bs multiply-adds and bs
    divisions per block (counted as 8 slots each), or one division per row."""
    if bs == 1:
        return 8 * n
    full, last = divmod(n, bs)
    per = lambda m: m ** 3 - m + 8 * m
    return full * per(bs) + (per(last) if last else 0)


def table2_bytes(kind, iters, nnz, n, vt=8, it=4, k=100):
    """Memory access volume (reads, writes) of a full unpreconditioned run as
    the paper models it for a COO SpMV (Table 2): vt value bytes, it index
    bytes.  iters counts what the table counts -- CG and FCG iterations;
    BiCGSTAB and CGS steps with one SpMV each (a full iteration is two, hence
    the table's ceil(iters/2) and floor(iters/2) terms); GMRES Arnoldi steps
    with restart k (r = iters mod k, iter_r the orthogonalisation steps)."""
    spmv = 2 * nnz * vt + 2 * nnz * it  # one COO apply: values, gathered x, row and column indices
    c, f = (iters + 1) // 2, iters // 2
    if kind == "cg":
        reads = (4 * n + 2 * nnz) * vt + 2 * nnz * it + iters * ((15 * n) * vt + spmv)
        writes = (5 * n + 2) * vt + iters * (5 * n + 2) * vt
    elif kind == "fcg":
        reads = (4 * n + 2 * nnz) * vt + 2 * nnz * it + iters * ((17 * n) * vt + spmv)
        writes = (6 * n + 3) * vt + iters * (6 * n + 3) * vt
    elif kind == "bicgstab":
        reads = ((5 * n + 2 * nnz) * vt + 2 * nnz * it + c * ((16 * n) * vt + spmv)
                 + f * ((13 * n) * vt + spmv))
        writes = (10 * n + 6) * vt + c * (4 * n + 2) * vt + f * (4 * n + 3) * vt
    elif kind == "cgs":
        reads = ((5 * n + 2 * nnz) * vt + 2 * nnz * it + c * ((14 * n) * vt + spmv)
                 + f * ((6 * n) * vt + spmv))
        writes = (10 * n + 2) * vt + c * (6 * n + 3) * vt + f * (4 * n) * vt
    elif kind == "gmres":
        q, r = divmod(iters, k)
        iter_r = q * (k - 1) * k // 2 + (r - 1) * r // 2
        reads = ((11 * n + 2 * nnz + 2.5 * r + n * r + r * r / 2 + 1) * vt + 2 * nnz * it
                 + q * ((1 + 2.5 * k + 10 * n + 2 * nnz + k * k / 2 + k * n) * vt + 2 * nnz * it)
                 + iters * ((7 * n + 5 + 2 * nnz) * vt + 2 * nnz * it + 8) + iter_r * (4 * n + 4) * vt)
        writes = ((6 * n + r + 2 * k + 3) * vt + 8 + q * ((k + 6 * n + 2) * vt + 8)
                  + iters * ((4 * n + 8) * vt + 8) + iter_r * (n + 2) * vt)
    else:
        raise ValueError(kind)
    return reads, writes


def table2_cg_bytes(iters, nnz, n, vt=8, it=4):
    """Total memory access volume of a full CG run as the paper models it (Table 2)."""
    return sum(table2_bytes("cg", iters, nnz, n, vt, it))


def spmv_launches(info):
    f = info["format_name"]
    if f == "csr_merge":
        return 2
    if f == "hyb":
        return 3 if info["tail_rows"] > 0 else 1
    if f == "csr":
        return 2 if info.get("split_rows", 0) > 0 else 1
    return 1


def solve_launches(kind, iters, spmvs, spmv_l, idle=0):
    """Kernels one solve launches; idle = the status's idle_iters, the
    iterations launched after the stop (a graph's loop body runs whole
    passes), whose kernels do nothing but are launched all the same."""
    if kind == "cg":
        # init, setup SpMV, start, iterations x (SpMV + 2), final SpMV
        return 2 + spmv_l + (iters + idle) * (spmv_l + 2) + spmv_l
    full = spmvs - 2 - iters
    half = iters - full
    return 2 + spmv_l + full * (2 * spmv_l + 3) + half * (spmv_l + 3) + spmv_l


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

REASON_FIELDS = ["clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                 "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"gk_clocks_{os.getpid()}.csv")

    def start(self):
        q = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," + ",".join(REASON_FIELDS)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                               parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_inputs(small=False):
    import workloads as W
    if small:
        A = W.stencil27(32)
        B = W.powerlaw(20000, seed=3)
    else:
        A = W.stencil27(128)
        B = W.powerlaw(1_000_000, seed=3)
    na, nb = A[0].size - 1, B[0].size - 1
    return {"a": A, "b": B, "xa": W.uniform_vector(na, 2), "xb": W.uniform_vector(nb, 3),
            "xs_a": W.uniform_vector(na, 4), "xs_b": W.uniform_vector(nb, 5)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def spmv_source_hash():
    """sha256 prefix of the ELL kernel's source: the epilogue section and the
    GK_ELL section of spmv.cu (the counters stay valid while these are
    unchanged, whatever else the file holds)."""
    src = open(os.path.join(ROOT, "paper_2006_16852_gb300", "csrc", "spmv.cu")).read()
    a = src.index("// epilogue")
    b = src.index("// Grid-wide reduction of (a0, a1)")
    c = src.index("// GK_ELL (and the ELL part of GK_HYB)")
    d = src.index("// GK_CSR_MERGE")
    return hashlib.sha256((src[a:b] + src[c:d]).encode()).hexdigest()[:16]


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class GpuStep:
    """All handles and device buffers of one step, created once."""

    def __init__(self, inp, dev, tol=1e-10, check_every=0):
        import torch
        import paper_2006_16852_gb300 as gk
        self.gk, self.torch, self.dev = gk, torch, dev
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        A, B = inp["a"], inp["b"]
        self.na, self.nb = A[0].size - 1, B[0].size - 1
        self.nnza, self.nnzb = A[1].size, B[1].size
        dA = [t(v) for v in A]
        dB = [t(v) for v in B]
        self.mats = {}
        for f in ("csr", "csr_merge", "ell", "hyb"):
            self.mats[("a", f)] = gk.Matrix(*dA, fmt=f)
        for f in ("csr_merge", "hyb", "csr"):
            self.mats[("b", f)] = gk.Matrix(*dB, fmt=f)
        self.dA, self.dB = dA, dB
        self.x = {"a": t(inp["xa"]), "b": t(inp["xb"])}
        self.y = {"a": torch.zeros(self.na, dtype=torch.float64, device=dev),
                  "b": torch.zeros(self.nb, dtype=torch.float64, device=dev)}
        self.dot_out = torch.zeros(1, dtype=torch.float64, device=dev)
        # right-hand sides b = A x* (computed by the library on the device)
        self.rhs = {}
        for k, xs in (("a", inp["xs_a"]), ("b", inp["xs_b"])):
            r = torch.zeros(self.na if k == "a" else self.nb, dtype=torch.float64, device=dev)
            gk.apply(self.mats[(k, "csr" if k == "a" else "csr_merge")], t(xs), r)
            self.rhs[k] = r
        crit = dict(max_iters=5000, reduction_factor=tol, check_every=check_every)
        M = self.mats
        # name: (solver, matrix key, preconditioner kind, block size, method, format)
        self.solvers = {
            "a_cg_plain_csr": (gk.Solver(M[("a", "csr")], None, "cg", **crit), "a", "none", 1, "cg", "csr"),
            "a_cg_jacobi_ell": (gk.Solver(M[("a", "ell")], gk.Precond(M[("a", "ell")], 1), "cg", **crit), "a",
                                "jacobi", 1, "cg", "ell"),
            "a_cg_bj8_ell": (gk.Solver(M[("a", "ell")], gk.Precond(M[("a", "ell")], 8), "cg", **crit), "a",
                             "block", 8, "cg", "ell"),
            "b_cg_jacobi_hyb": (gk.Solver(M[("b", "hyb")], gk.Precond(M[("b", "hyb")], 1), "cg", **crit), "b",
                                "jacobi", 1, "cg", "hyb"),
            "b_bicgstab_bj4_hyb": (gk.Solver(M[("b", "hyb")], gk.Precond(M[("b", "hyb")], 4), "bicgstab", **crit),
                                   "b", "block", 4, "bicgstab", "hyb"),
            # mixed precision: FP64 refinement around FP32 CG (adaptive FP16/FP32 blocks)
            "a_ircg_jacobi_ell": (gk.Solver(M[("a", "ell")], gk.Precond(M[("a", "ell")], 1), "ir_cg", **crit),
                                  "a", "jacobi", 1, "ir_cg", "ell"),
            "a_ircg_bj8_ell": (gk.Solver(M[("a", "ell")], gk.Precond(M[("a", "ell")], 8), "ir_cg", **crit),
                               "a", "block", 8, "ir_cg", "ell"),
        }
        self.fp16_frac = {}
        for name, v in self.solvers.items():
            if v[4] == "ir_cg" and v[2] == "block":
                inf = v[0].info()
                tot = inf["inner_fp16_blocks"] + inf["inner_fp32_blocks"]
                self.fp16_frac[name] = inf["inner_fp16_blocks"] / max(tot, 1)
        self.xsol = {k: torch.zeros(self.na if v[1] == "a" else self.nb, dtype=torch.float64, device=dev)
                     for k, v in self.solvers.items()}
        self.gens = [("a", "csr", 1), ("a", "csr", 8), ("b", "csr_merge", 4)]
        self.in_block = {(k, bs): in_block_entries(inp[k], bs) for k, _, bs in self.gens}
        self.stream = torch.cuda.current_stream(dev)

    def n_of(self, k):
        return self.na if k == "a" else self.nb

    def nnz_of(self, k):
        return self.nnza if k == "a" else self.nnzb

    def run(self, record=None, host=None):
        """One step.  record: dict receiving per-part event pairs.  host: if
        given, a dict of pinned host buffers; vectors then go through the C
        ABI as host pointers (end-to-end mode)."""
        gk, torch = self.gk, self.torch
        ev = lambda: torch.cuda.Event(enable_timing=True)
        parts = []
        for (k, f), M in self.mats.items():
            e0, e1 = ev(), ev()
            e0.record(self.stream)
            for _ in range(SPMV_REPS):
                if host is None:
                    gk.apply(M, self.x[k], self.y[k])
                else:
                    gk.apply(M, host["x" + k], host["y" + k])
            e1.record(self.stream)
            parts.append((f"spmv_{k}_{f}", e0, e1, ("spmv", k, M)))
        # the SpMV with the fused dot of the CG steps (the step's dominant
        # kernel), on (a) in ELL; device vectors in both modes
        e0, e1 = ev(), ev()
        e0.record(self.stream)
        for _ in range(SPMV_REPS):
            gk.apply_dot(self.mats[("a", "ell")], self.x["a"], self.y["a"], self.rhs["a"], self.dot_out)
        e1.record(self.stream)
        parts.append(("spmvdot_a_ell", e0, e1, ("spmvdot", "a", self.mats[("a", "ell")])))
        for k, f, bs in self.gens:
            e0, e1 = ev(), ev()
            e0.record(self.stream)
            P = gk.Precond(self.mats[(k, f)], bs)
            e1.record(self.stream)
            parts.append((f"precond_{k}_bs{bs}", e0, e1, ("precond", k, bs)))
            del P
        statuses = {}
        for name, (S, k, prec, bs, kind, fmt) in self.solvers.items():
            e0, e1 = ev(), ev()
            e0.record(self.stream)
            if host is None:
                self.xsol[name].zero_()
                st = gk.solve(S, self.rhs[k], self.xsol[name])
            else:
                host["x0" + k][:] = 0.0
                st = gk.solve(S, host["rhs" + k], host["x0" + k])
            e1.record(self.stream)
            statuses[name] = st
            parts.append((f"solve_{name}", e0, e1, ("solve", name, st)))
        if record is not None:
            record.append(parts)
        return statuses

    def fmt_of(self, M):
        """(format, HYB tail entries) of a matrix handle, for the byte model."""
        inf = M.info()
        return inf["format_name"], inf["tail_nnz"] if inf["format_name"] == "hyb" else 0

    def part_bytes(self, tag):
        kind = tag[0]
        if kind in ("spmv", "spmvdot"):
            k = tag[1]
            fmt, tail = self.fmt_of(tag[2])
            one = spmv_bytes(self.nnz_of(k), self.n_of(k), self.n_of(k), fmt=fmt, tail_nnz=tail)
            return SPMV_REPS * (one + (8 * self.n_of(k) if kind == "spmvdot" else 0))
        if kind == "precond":
            k, bs = tag[1], tag[2]
            return precond_bytes(self.n_of(k), bs, self.in_block[(k, bs)])
        name, st = tag[1], tag[2]
        S, k, prec, bs, sk, fmt = self.solvers[name]
        f, tail = self.fmt_of(self.mats[(k, fmt)])
        if sk == "ir_cg":
            return ir_bytes(st.iters, st.outer_iters, self.nnz_of(k), self.n_of(k), prec, bs,
                            self.fp16_frac.get(name, 0.0), fmt=f, tail_nnz=tail)
        if sk == "cg":
            return cg_bytes(st.iters, self.nnz_of(k), self.n_of(k), prec, bs, fmt=f, tail_nnz=tail)
        return bicgstab_bytes(st.iters, st.spmvs, self.nnz_of(k), self.n_of(k), prec, bs, fmt=f, tail_nnz=tail)

    def part_launches(self, tag):
        kind = tag[0]
        if kind in ("spmv", "spmvdot"):
            return SPMV_REPS * spmv_launches(tag[2].info())
        if kind == "precond":
            # scalar Jacobi: one kernel; block Jacobi up to bs 8: extraction + inversion
            return 2 if 1 < tag[2] <= 8 else 1
        name, st = tag[1], tag[2]
        S, k, prec, bs, sk, fmt = self.solvers[name]
        info = self.mats[(k, fmt)].info()
        if sk == "ir_cg":
            # init; per outer step: FP64 residual SpMV, start, apply; per inner
            # iteration: FP32 SpMV (+ overflow kernel for HYB), update, direction
            inner_spmv = 2 if (info["format_name"] == "hyb" and info["tail_rows"] > 0) else 1
            return (1 + (st.outer_iters + 1) * spmv_launches(info) + 2 * st.outer_iters
                    + (st.iters + st.idle_iters) * (inner_spmv + 2))
        return solve_launches(sk, st.iters, st.spmvs, spmv_launches(info), idle=st.idle_iters)


# ---------------------------------------------------------------------------
# batched small systems (reported beside the step, not part of its value)
# ---------------------------------------------------------------------------

BATCH_WORKLOAD = ("10,000 independent SPD systems, 2D 5-point variable-coefficient diffusion (cell coefficients "
                  "log-normal sigma=0.5, harmonic-mean faces, Dirichlet), grid side U{6..32} (n 36..1024), seed 5; "
                  "b uniform[-1,1], x0 = 0")
# nominal FP64 rate of a GB300 (the batched FP64 solves are bound by the FP64 pipe)
FP64_PEAK_TFLOPS = 1.25


def batch_fp64_flops(kind, jac, iters, nnz_s, n_s):
    """FP64 flops (2 per fused multiply-add) of the batched FP64 solves: per
    CG iteration a row costs its nonzeros + 7 FMA-class operations with Jacobi
    (sigma, x, r, z, r.z, r.r, p) or + 6 without; BiCGSTAB: 2 SpMVs + 14 (+2
    with Jacobi); plus the initial residual."""
    per_row = {"cg": 7 if jac else 6, "bicgstab": 16 if jac else 14}[kind]
    spmvs = 2 if kind == "bicgstab" else 1
    return 2.0 * float(np.sum(iters * (spmvs * nnz_s + per_row * n_s) + nnz_s + 2 * n_s))


BATCH_FORMS = ("fp64_cg_jacobi", "fp64_bicgstab_jacobi", "fp64_ir_cg_jacobi", "fp32_cg_jacobi",
               "fp32_bicgstab_jacobi")


def run_batched(dev, reps=3, n_sys=10000, only=None, tune=True, plain=True):
    import torch
    import paper_2006_16852_gb300 as gk
    import workloads as W
    sys_ptr, A = W.batch_varcoef2d(n_sys, seed=5)
    n = int(sys_ptr[-1])
    rowptr = A[0]
    nnz_s = (rowptr[sys_ptr[1:]] - rowptr[sys_ptr[:-1]]).astype(np.float64)
    n_s = np.diff(sys_ptr).astype(np.float64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dA = [t(a) for a in A]
    b = t(W.uniform_vector(n, 28))
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            x.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    forms = {}
    launches = {}
    Bs = {"f64": gk.Batch(sys_ptr, *dA, dtype="f64"), "f32": gk.Batch(sys_ptr, *dA, dtype="f32")}
    cfgs = [("fp64_cg_jacobi", "f64", "cg", 1e-10), ("fp64_bicgstab_jacobi", "f64", "bicgstab", 1e-10),
            ("fp64_ir_cg_jacobi", "f64", "ir_cg", 1e-10), ("fp32_cg_jacobi", "f32", "cg", 1e-6),
            ("fp32_bicgstab_jacobi", "f32", "bicgstab", 1e-6)]
    for name, dt, kind, tol in cfgs:
        if only and name not in only:
            continue
        B = Bs[dt]
        if tune:
            chosen, _ = B.autotune(b, kind=kind, jacobi=True, reduction_factor=tol, max_iters=20000)
        else:
            chosen = B.info(kind=kind)["threads"]
        x.zero_()
        st = B.solve(b, x, kind=kind, jacobi=True, reduction_factor=tol, max_iters=20000)
        ms = timed(lambda: B.solve(b, x, kind=kind, jacobi=True, reduction_factor=tol, max_iters=20000,
                                   status=False))
        f = {"ms": round(ms, 3), "solves_per_s": round(n_sys / (ms * 1e-3)), "tol": tol,
             "converged": int((st["stop_reason"] == gk.STOP_CONVERGED).sum()),
             "iters_mean": round(float(st["iters"].mean()), 2), "iters_max": int(st["iters"].max()),
             "block_sizes_per_class": chosen}
        if kind == "ir_cg":
            f["outer_mean"] = round(float(st["outer_iters"].mean()), 3)
        if dt == "f64" and kind != "ir_cg":
            fl = batch_fp64_flops(kind, True, st["iters"].astype(np.float64), nnz_s, n_s)
            f["fp64_tflops"] = round(fl / (ms * 1e-3) / 1e12, 4)
        forms[name] = f
        launches[name] = sum(1 for c in chosen if c)
    out = {"workload": BATCH_WORKLOAD, "n_sys": n_sys, "rows": n, "nnz": int(A[1].size),
           "timing": "CUDA events around each gk_batch_solve graph launch, median of %d, inputs resident" % reps,
           "forms": forms, "gpu_launches_per_solve": launches}
    if not plain or "fp64_cg_jacobi" not in forms:
        return out
    # plain FP64 CG through the unbatched path on the block-diagonal matrix
    # (ELL, one global criterion ||r|| <= 1e-10 ||b||)
    M = gk.Matrix(*dA, fmt="ell")
    S = gk.Solver(M, None, "cg", max_iters=20000, reduction_factor=1e-10)
    x.zero_()
    st = gk.solve(S, b, x)
    plain_ms = timed(lambda: gk.solve(S, b, x))
    r = torch.zeros_like(b)
    gk.apply(M, x, r)
    r = (b - r).cpu().numpy()
    bh = b.cpu().numpy()
    seg = lambda v: np.sqrt(np.add.reduceat(v * v, sys_ptr[:-1]))
    per_sys = seg(r) / seg(bh)
    chosen_form = min((k for k in ("fp64_cg_jacobi", "fp64_bicgstab_jacobi", "fp64_ir_cg_jacobi") if k in forms),
                      key=lambda k: forms[k]["ms"])
    cg64 = forms["fp64_cg_jacobi"]
    ach = cg64["fp64_tflops"]
    rate = gk.fp64_rate()
    out.update({
        "time_to_tol_ms": {"plain_fp64_cg_unbatched": round(plain_ms, 3), "plain_iters": st.iters,
                           "plain_per_system_rel_res_max": float(per_sys.max()),
                           "chosen_form": chosen_form, "chosen_ms": forms[chosen_form]["ms"],
                           "speedup_vs_plain": round(plain_ms / forms[chosen_form]["ms"], 2)},
        "roofline": {"kernel": "batch_kernel<double, CG, Jacobi> (one block per system, FP64)", "bound": "alu",
                     "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "peak_source": "nominal GB300 FP64 rate", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                     "measured_fp64_tflops": round(rate, 4), "frac_of_measured": round(ach / rate, 4),
                     "traffic": None},
    })
    return out


# ---------------------------------------------------------------------------
# mixed precision at its own workload (reported beside the step)
# ---------------------------------------------------------------------------

MIXED_WORKLOAD = ("7-point variable-coefficient diffusion on a {s}^3 grid (n={n:,}, nnz={nnz:,}), cell "
                  "coefficients log-normal sigma=1 i.i.d. (seed 4), harmonic-mean faces, Dirichlet; b uniform[-1,1] "
                  "(seed 7), x0 = 0, ||r|| <= 1e-12 ||b||")


def run_mixed(dev, side=256, tol=1e-12):
    """Plain FP64 CG against FP64 refinement around FP32 CG (Jacobi or
    adaptive FP16/FP32 block Jacobi of 8, 16, 32) on the mixed-precision
    workload; one warm-up solve and one timed solve per form."""
    import torch
    import paper_2006_16852_gb300 as gk
    import workloads as W
    A = W.varcoef3d(side, sigma=1.0, seed=4)
    n, nnz = A[0].size - 1, A[1].size
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dA = [t(a) for a in A]
    del A
    b = t(W.uniform_vector(n, 7))
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    M = gk.Matrix(*dA, fmt="ell")
    del dA
    crit = dict(max_iters=200000, reduction_factor=tol)
    forms = {"plain_fp64_cg": (None, "cg"), "fp64_cg_bj16": (16, "cg"), "ir_cg_jacobi": (1, "ir_cg"),
             "ir_cg_bj8": (8, "ir_cg"), "ir_cg_bj16": (16, "ir_cg"), "ir_cg_bj32": (32, "ir_cg")}
    out = {}
    for name, (bs, kind) in forms.items():
        P = gk.Precond(M, bs) if bs else None
        S = gk.Solver(M, P, kind, **crit)
        ms = []
        for _ in range(2):
            x.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = gk.solve(S, b, x)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        if st.stop_reason != gk.STOP_CONVERGED:
            raise RuntimeError(f"mixed {name} did not converge: {st}")
        prec = "none" if not bs else ("jacobi" if bs == 1 else "block")
        f = {"ms": round(ms[-1], 2), "iters": st.iters, "rel_res_true": st.rel_res_true}
        if kind == "ir_cg":
            inf = S.info()
            tot = inf["inner_fp16_blocks"] + inf["inner_fp32_blocks"]
            frac = inf["inner_fp16_blocks"] / tot if tot else 0.0
            f["outer_iters"] = st.outer_iters
            if tot:
                f["fp16_block_fraction"] = round(frac, 4)
            by = ir_bytes(st.iters, st.outer_iters, nnz, n, prec, bs or 1, frac, fmt="ell")
        else:
            by = cg_bytes(st.iters, nnz, n, prec, bs or 1, fmt="ell")
        f["GB/s"] = round(by / (ms[-1] * 1e-3) / 1e9, 1)
        out[name] = f
        del S, P
    plain = out["plain_fp64_cg"]["ms"]
    chosen = min((k for k in out if k != "plain_fp64_cg"), key=lambda k: out[k]["ms"])
    return {"workload": MIXED_WORKLOAD.format(s=side, n=n, nnz=nnz),
            "timing": "CUDA events around gk_solve (device-side graph loop), second of two solves, inputs resident",
            "forms": out,
            "time_to_tol_ms": {"plain_fp64_cg": plain, "chosen_form": chosen, "chosen_ms": out[chosen]["ms"],
                               "speedup_vs_plain": round(plain / out[chosen]["ms"], 3)}}


# ---------------------------------------------------------------------------
# learned warm start (reported beside the step)
# ---------------------------------------------------------------------------

LEARNED_WORKLOAD = ("2D diffusion on a 256x256 grid (n=65,536), cell coefficients exp(GRF), GRF a sum of 16 random "
                    "Fourier modes (correlation length 0.1, sigma 1), source 4 Gaussian bumps (seeds (6, i, .)); "
                    "held-out problems i >= 1,000,000; Jacobi-CG to ||r|| <= 1e-10 ||b||")
# FP32 FMA issue rate of a GB300: 152 SMs x 128 lanes x 2 flops at 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def run_learned(dev, problems=8):
    import torch
    import paper_2006_16852_gb300 as gk
    from paper_2006_16852_gb300 import learned as LN
    path = os.path.join(LN.DATA_DIR, "wsnet_256.npz")
    if not os.path.exists(path):
        return {"unavailable": "no trained weights at paper_2006_16852_gb300/data/wsnet_256.npz"}
    net, scale, meta = LN.load(path)
    idx = range(1_000_000, 1_000_000 + problems)
    res = LN.evaluate(net, idx, scale)
    summ = LN.summarize(res)
    # the same problems to looser targets, where the start matters more
    loose = {}
    for tol in (1e-4, 1e-6):
        ls = LN.summarize(LN.evaluate(net, idx, scale, tol=tol))
        loose[f"{tol:g}"] = {k: ls[k] for k in ("iters_zero", "iters_warm", "iters_ratio", "ms_zero", "ms_warm",
                                               "time_ratio")}
    # plain FP64 CG (no preconditioner, zero start) on the same problems
    import workloads as W
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    plain_ms, plain_it = 0.0, 0
    stream = torch.cuda.current_stream(dev)
    for i in idx:
        g, A, b = W.grf_problem(net.H, i)
        M = gk.Matrix(*[t(a) for a in A], fmt="ell")
        S = gk.Solver(M, None, "cg", max_iters=50000, reduction_factor=1e-10)
        bd = t(b)
        for _ in range(2):
            x = torch.zeros_like(bd)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = gk.solve(S, bd, x)
            e1.record(stream)
            e1.synchronize()
        plain_ms += e0.elapsed_time(e1)
        plain_it += st.iters
    # BF16 inference alone: one problem (the warm start's case) and a batch
    # of 64 (enough tiles for every SM)
    macs = net.H * net.W * sum(a * b * 9 for a, b in zip((2, 32, 32, 32, 32, 32), (32, 32, 32, 32, 32, 1)))
    inf = {}
    bnet, _, _ = LN.load(path, batch_max=64)
    for B, nt in ((1, net), (64, bnet)):
        feat = torch.zeros((B, 2, net.H, net.W), dtype=torch.float32, device=dev)
        feat[:, 0].normal_()
        feat[:, 1].normal_()
        y = torch.zeros((B, 1, net.H, net.W), dtype=torch.float32, device=dev)
        for _ in range(3):
            nt.infer_bf16(feat, y)
        nt.check()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        e0.record(stream)
        for _ in range(reps):
            nt.infer_bf16(feat, y)
        e1.record(stream)
        e1.synchronize()
        nt.check()
        ms = e0.elapsed_time(e1) / reps
        inf[B] = (ms, 2.0 * B * macs / (ms * 1e-3) / 1e12)
    bf16_peak = peaks().get("bf16_tflops")
    hbm = peaks().get("hbm_gbs")
    inf_ms, tfl = inf[1]
    # compulsory activation bytes per pixel of one inference (the byte
    # model of infer_bytes_per_pixel)
    bpp = infer_bytes_per_pixel()
    by64 = 64 * net.H * net.W * bpp
    ai = 2.0 * macs / (net.H * net.W * bpp)
    gbs64 = by64 / (inf[64][0] * 1e-3) / 1e9
    best = "warm" if summ["ms_warm"] < summ["ms_zero"] else "zero"
    return {
        "workload": LEARNED_WORKLOAD, "network": {"layers": 6, "width": 32, "dilations": list(net.dilations),
                                                  "weights": "BF16 (trained in FP32)", "params": net.nparams},
        "training": {k: meta[k] for k in ("samples", "epochs", "batch", "lr", "loss", "data_seconds",
                                          "train_seconds", "loss_history") if k in meta},
        "eval": summ,
        "eval_looser_targets": loose,
        "time_to_tol_ms": {"plain_fp64_cg": round(plain_ms, 3), "plain_iters": plain_it,
                           "jacobi_cg_zero_start": summ["ms_zero"], "jacobi_cg_learned_start": summ["ms_warm"],
                           "chosen_form": "jacobi_cg_" + ("learned" if best == "warm" else "zero") + "_start",
                           "speedup_vs_plain": round(plain_ms / min(summ["ms_warm"], summ["ms_zero"]), 3),
                           "learned_vs_zero_start": round(summ["ms_zero"] / summ["ms_warm"], 4)},
        "inference": {"kernel": "conv_first_tc_kernel and conv_tc_kernel (tcgen05.mma BF16 x BF16 -> FP32 in "
                                "tensor memory) for the first five layers (the first with K = 18 padded to 32), "
                                "the last (32 -> 1) folded into the fifth's epilogue as nine tap planes that "
                                "conv_last_sum_kernel adds",
                      "batch1": {"ms": round(inf_ms, 4), "tflops": round(tfl, 2),
                                 "frac_of_bf16_peak": round(tfl / bf16_peak, 5) if bf16_peak else None,
                                 "note": "42.7 MB of activations: L2-resident, latency-bound"},
                      "batch64": {"ms": round(inf[64][0], 4), "tflops": round(inf[64][1], 2),
                                  "frac_of_bf16_peak": round(inf[64][1] / bf16_peak, 5) if bf16_peak else None},
                      "roofline": {"workload": "batch 64", "bound": "hbm",
                                   "arithmetic_intensity_flop_per_byte": round(ai, 1),
                                   "ridge_flop_per_byte": round(bf16_peak * 1e3 / hbm, 1) if bf16_peak and hbm
                                   else None,
                                   "bytes_per_pixel": bpp, "bytes": by64,
                                   "achieved": round(gbs64, 1), "peak": hbm, "unit": "GB/s",
                                   "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                                   "frac": round(gbs64 / hbm, 4) if hbm else None},
                      "bf16_peak_tflops": bf16_peak,
                      "cuda_core_fp32_issue_peak_tflops": round(FP32_PEAK_TFLOPS, 1)},
    }


# ---------------------------------------------------------------------------
# the rest of the Krylov family (reported beside the step)
# ---------------------------------------------------------------------------

KRYLOV_WORKLOAD = ("nonsymmetric 2D convection-diffusion (first-order upwind, wind 0.5) on a 1024x1024 grid "
                   "(n=1,048,576, nnz=5,238,784) and the 27-point stencil on 128^3 for the symmetric methods; "
                   "x* uniform[-1,1], b = A x*, x0 = 0, ||r|| <= 1e-10 ||b||, scalar Jacobi, ELL")


def run_krylov(dev):
    """Time to 1e-10 of every Krylov method on a matrix it applies to."""
    import torch
    import paper_2006_16852_gb300 as gk
    import workloads as W
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.current_stream(dev)
    out = {}
    mats = {"convdiff1024": W.convdiff2d(1024, 0.5), "stencil27_128": W.stencil27(128)}
    runs = [("convdiff1024", "bicgstab", {}), ("convdiff1024", "cgs", {}), ("convdiff1024", "gmres", {"krylov_dim": 30}),
            ("stencil27_128", "cg", {}), ("stencil27_128", "fcg", {}), ("stencil27_128", "gmres", {"krylov_dim": 30})]
    built = {}
    for name, A in mats.items():
        n = A[0].size - 1
        M = gk.Matrix(*[t(a) for a in A], fmt="ell")
        b = torch.zeros(n, dtype=torch.float64, device=dev)
        gk.apply(M, t(W.uniform_vector(n, 11)), b)
        built[name] = (M, gk.Precond(M, 1), b, A[1].size, n)
    for name, kind, extra in runs:
        M, P, b, nnz, n = built[name]
        S = gk.Solver(M, P, kind, max_iters=20000, reduction_factor=1e-10, **extra)
        for rep_ in range(2):
            x = torch.zeros_like(b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = gk.solve(S, b, x)
            e1.record(stream)
            e1.synchronize()
        ms = e0.elapsed_time(e1)
        rec = {"ms": round(ms, 3), "iters": st.iters, "spmvs": st.spmvs, "rel_res_true": st.rel_res_true,
               "converged": st.stop_reason == gk.STOP_CONVERGED,
               "ms_per_spmv": round(ms / max(st.spmvs, 1), 4)}
        if kind in ("cg", "fcg"):
            rec["GB/s_cg_model"] = round(cg_bytes(st.iters, nnz, n, "jacobi", 1, fmt="ell") / (ms * 1e-3) / 1e9, 1)
        out[f"{name}_{kind}"] = rec
    return {"workload": KRYLOV_WORKLOAD, "timing": "CUDA events around gk_solve, the second of two solves",
            "solves": out}


# ---------------------------------------------------------------------------
# latency of one iteration on the small configuration (reported beside the step)
# ---------------------------------------------------------------------------

LATENCY_WORKLOAD = ("Poisson-2D 64x64 (n=4,096, nnz=20,224; L2-resident), x* uniform[-1,1] (seed 1), b = A x*, "
                    "x0 = 0, ||r|| <= 1e-10 ||b||")


def run_latency(dev):
    """Per-iteration time of CG on the small Poisson problem, where every
    kernel is latency-bound: the default form (one launch of a 16-CTA
    thread-block cluster), the whole solve as one graph whose loop the GPU
    controls (check_every -1), and host-driven loops that read the status
    after every iteration (check_every 1, the paper's host-side check) or
    after every 10."""
    import torch
    import paper_2006_16852_gb300 as gk
    import workloads as W
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.current_stream(dev)
    A = W.poisson2d(64)
    n = 4096
    out = {}
    names = {0: "default", -1: "graph", 1: "host1", 10: "host10"}
    forms = {gk.FORM_GRAPH: "graph", gk.FORM_HOST: "host", gk.FORM_CLUSTER: "cluster", gk.FORM_GRID: "grid"}
    for fmt in ("csr", "ell"):
        M = gk.Matrix(*[t(a) for a in A], fmt=fmt)
        b = torch.zeros(n, dtype=torch.float64, device=dev)
        gk.apply(M, t(W.uniform_vector(n, 1)), b)
        for prec in (0, 1):
            P = gk.Precond(M, 1) if prec else None
            for every in (0, -1, 1, 10):
                S = gk.Solver(M, P, "cg", max_iters=5000, reduction_factor=1e-10, check_every=every)
                best = None
                for _ in range(5):
                    x = torch.zeros_like(b)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    st = gk.solve(S, b, x)
                    e1.record(stream)
                    e1.synchronize()
                    ms = e0.elapsed_time(e1)
                    best = ms if best is None else min(best, ms)
                key = f"{fmt}_{'jacobi' if prec else 'plain'}_{names[every]}"
                out[key] = {"form": forms.get(st.form, st.form), "ms": round(best, 4), "iters": st.iters,
                            "us_per_iter": round(1e3 * best / max(st.iters, 1), 3), "rel_res_true": st.rel_res_true}
    # BiCGSTAB on a small nonsymmetric system: the cluster form and the graph
    A3 = W.convdiff2d(64, 0.5)
    M3 = gk.Matrix(*[t(a) for a in A3], fmt="csr")
    b3 = torch.zeros(4096, dtype=torch.float64, device=dev)
    gk.apply(M3, t(W.uniform_vector(4096, 1)), b3)
    P3 = gk.Precond(M3, 1)
    for every in (0, -1):
        S = gk.Solver(M3, P3, "bicgstab", max_iters=5000, reduction_factor=1e-10, check_every=every)
        best = None
        for _ in range(5):
            x = torch.zeros_like(b3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = gk.solve(S, b3, x)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[f"convdiff64_bicgstab_jacobi_{names[every]}"] = {
            "form": forms.get(st.form, st.form), "ms": round(best, 4), "iters": st.iters,
            "us_per_iter": round(1e3 * best / max(st.iters, 1), 3), "rel_res_true": st.rel_res_true}
    # a mid-size system: the default form is the cooperative grid
    A2 = W.poisson2d(256)
    M2 = gk.Matrix(*[t(a) for a in A2], fmt="csr")
    b2 = torch.zeros(65536, dtype=torch.float64, device=dev)
    gk.apply(M2, t(W.uniform_vector(65536, 1)), b2)
    P2 = gk.Precond(M2, 1)
    for every in (0, -1):
        S = gk.Solver(M2, P2, "cg", max_iters=5000, reduction_factor=1e-10, check_every=every)
        best = None
        for _ in range(3):
            x = torch.zeros_like(b2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = gk.solve(S, b2, x)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[f"poisson256_jacobi_{names[every]}"] = {"form": forms.get(st.form, st.form), "ms": round(best, 4),
                                                    "iters": st.iters,
                                                    "us_per_iter": round(1e3 * best / max(st.iters, 1), 3),
                                                    "rel_res_true": st.rel_res_true}
    return {"workload": LATENCY_WORKLOAD + "; BiCGSTAB with Jacobi on upwind convection-diffusion 64x64; and "
                                           "Poisson-2D 256x256 (n=65,536) with Jacobi for the mid-size form",
            "timing": "CUDA events around gk_solve, best of 5 (3 for 256x256)",
            "paper_host_overhead_us_per_iter": [1.0, 1.5], "solves": out}


# ---------------------------------------------------------------------------
# the paper's own numbers (context: other GPUs, 2020) and its solver-bandwidth
# experiment repeated here
# ---------------------------------------------------------------------------

PAPER_CONTEXT = {
    "source": "arXiv 2006.16852, Section 7 (Tables 1-3); one GPU per run",
    "krylov_solver_bandwidth": {
        "setup": "BiCGSTAB, CG, CGS, FCG, GMRES(100); COO SpMV, no preconditioner, 10,000 iterations, "
                 "10 SuiteSparse matrices; bytes from the Table 2 model",
        "V100": {"GB/s": [600, 800], "frac_of_stream_triad": "> 0.80", "stream_triad_GB/s": 812.6,
                 "hbm_nominal_GB/s": 900},
        "RadeonVII": {"GB/s": [500, 700], "frac_of_stream_triad": "> 0.70 (GMRES slightly less)",
                      "stream_triad_GB/s": 809.8, "hbm_nominal_GB/s": 1024},
    },
    "stream_GB/s_table3": {
        "V100": {"copy": 790.475, "mul": 787.301, "add": 811.312, "triad": 812.617, "dot": 844.321},
        "RadeonVII": {"copy": 841.669, "mul": 841.934, "add": 806.632, "triad": 809.754, "dot": 635.677},
    },
    "solver_overhead_us_per_iteration_table1": {"bicgstab": 1.26, "cg": 1.28, "cgs": 1.00, "fcg": 1.45,
                                                "gmres": 1.51},
}

PAPER_BW_WORKLOAD = ("27-point stencil on 128^3 (n=2,097,152, nnz=55,742,968), GK_CSR, no preconditioner, "
                     "x* uniform[-1,1], b = A x*, x0 = 0, a fixed iteration count (reduction factor 1e-300): "
                     "200 SpMVs in every solver's loop; GMRES restart 100")


def run_paper_bandwidth(dev, triad_gbs=None):
    """The paper's solver-bandwidth experiment (Section 7.3) on this GPU: each
    of the five Krylov solvers unpreconditioned for a fixed number of
    iterations, its memory volume from the paper's Table 2 model divided by
    the device time, against the STREAM triad measured in the same run.  The
    Table 2 model is written for a COO SpMV: it counts a row and a column
    index and one read of x per stored entry, where the CSR kernel here
    stores no row indices and finds x in L1/L2 after its first read, so that
    figure exceeds what crosses HBM; the CG and BiCGSTAB runs also carry this
    library's own byte model (each vector once), the bytes that do."""
    import torch
    import paper_2006_16852_gb300 as gk
    import workloads as W
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.current_stream(dev)
    A = W.stencil27(128)
    n, nnz = A[0].size - 1, A[1].size
    M = gk.Matrix(*[t(a) for a in A], fmt="csr")
    b = torch.zeros(n, dtype=torch.float64, device=dev)
    gk.apply(M, t(W.uniform_vector(n, 11)), b)
    runs = [("cg", 200, {}), ("fcg", 200, {}), ("bicgstab", 100, {}), ("cgs", 100, {}),
            ("gmres", 200, {"krylov_dim": 100})]
    out = {}
    for kind, iters, extra in runs:
        S = gk.Solver(M, None, kind, max_iters=iters, reduction_factor=1e-300, **extra)
        for _ in range(2):
            x = torch.zeros_like(b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = gk.solve(S, b, x)
            e1.record(stream)
            e1.synchronize()
        ms = e0.elapsed_time(e1)
        steps = st.spmvs - 2 if kind in ("bicgstab", "cgs") else st.iters
        rd, wr = table2_bytes(kind, steps, nnz, n, k=extra.get("krylov_dim", 100))
        gbs = (rd + wr) / (ms * 1e-3) / 1e9
        rec = {"iters": st.iters, "spmvs": st.spmvs, "table2_iter": steps, "stop_reason": st.stop_reason,
               "ms": round(ms, 3), "table2_model_bytes": int(rd + wr),
               "table2_model_bytes_per_s_GB": round(gbs, 1)}
        if triad_gbs:
            # model bytes over the triad rate: a ratio above 1 counts bytes that never cross HBM
            # (Table 2 charges x and a row index per stored entry), so it is not a bandwidth fraction
            rec["table2_model_over_triad"] = round(gbs / triad_gbs, 3)
        own = None
        if kind == "cg":
            own = cg_bytes(st.iters, nnz, n, "none")
        elif kind == "bicgstab":
            own = bicgstab_bytes(st.iters, st.spmvs, nnz, n, "none")
        if own is not None:
            rec["model_GB/s"] = round(own / (ms * 1e-3) / 1e9, 1)
            if triad_gbs:
                rec["model_frac_of_triad"] = round(own / (ms * 1e-3) / 1e9 / triad_gbs, 3)
        out[kind] = rec
    del M, b
    torch.cuda.empty_cache()
    return {"workload": PAPER_BW_WORKLOAD, "stream_triad_GB/s": triad_gbs,
            "timing": "CUDA events around gk_solve, the second of two solves",
            "note": "table2_model_* divide the paper's Table 2 model volume (COO: x and a row index per stored "
                    "entry) by the time; they are model bytes, not traffic, and exceed the triad on this matrix. "
                    "model_GB/s (CG, BiCGSTAB) uses this library's byte model, the bytes that cross HBM.",
            "solvers": out}


# ---------------------------------------------------------------------------
# stream probes (reported beside the step): the library's own reduction
# kernel against a plain device copy on the same device
# ---------------------------------------------------------------------------

def run_gather_ceiling(step, reps=20):
    """The random-gather ceiling of the power-law SpMV: gk_gather_dot over
    (b)'s own column/value stream (29 M entries, columns uniform over 10^6
    rows) -- the SpMV's per-entry work without its rows -- timed back to
    back with GK_CSR's apply of (b) and with the same stream's columns
    replaced by a uniformly random draw; CUDA events around reps
    back-to-back calls, median of 5 such runs after 3 warm-ups."""
    import torch
    gk = step.gk
    dev = step.dev
    stream = step.stream
    rowptr, col, val = step.dB
    n, nnz = step.nb, step.nnzb
    x = step.x["b"]
    res = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.Generator(device="cpu").manual_seed(7)
    col_rand = torch.randint(0, n, (nnz,), generator=g, dtype=torch.int32).to(dev)
    M = step.mats[("b", "csr")]

    def timed(fn):
        for _ in range(3):
            fn()
        ms = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1) / reps)
        return statistics.median(ms)

    t_gather = timed(lambda: gk.gather_dot(col, val, x, res))
    t_rand = timed(lambda: gk.gather_dot(col_rand, val, x, res))
    t_csr = timed(lambda: gk.apply(M, x, step.y["b"]))
    by = nnz * 12 + n * 8
    del col_rand
    return {"workload": "(b) power-law, its CSR column/value stream: %d entries, x of %d doubles (8 MB, "
                        "L2-resident)" % (nnz, n),
            "gather_dot_ms": round(t_gather, 4), "gather_dot_GB/s": round(by / (t_gather * 1e-3) / 1e9, 1),
            "gather_dot_uniform_cols_ms": round(t_rand, 4), "gk_csr_apply_ms": round(t_csr, 4),
            "gk_csr_over_ceiling": round(t_csr / t_gather, 3),
            "timing": "CUDA events around %d back-to-back calls, median of 5 such runs after 3 warm-ups, the "
                      "three kernels in one process" % reps}


def run_stream(dev, n=1 << 27):
    """gk_dot over two vectors of n doubles (1 GiB each: larger than L2),
    against torch's device copy of one of them (read + write bytes) and the
    STREAM triad a = b + 0.4 c (the paper's bandwidth reference, Section 7.3);
    the best of 10 after 3 warm-up runs, CUDA events."""
    import torch
    import paper_2006_16852_gb300 as gk
    x = torch.rand(n, dtype=torch.float64, device=dev)
    y = torch.rand(n, dtype=torch.float64, device=dev)
    z = torch.empty_like(x)
    r = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def best(fn):
        for _ in range(3):
            fn()
        t = None
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            t = ms if t is None else min(t, ms)
        return t

    dot_ms = best(lambda: gk.dot(x, y, r))
    copy_ms = best(lambda: z.copy_(x))
    triad_ms = best(lambda: torch.add(y, x, alpha=0.4, out=z))
    hbm = peaks().get("hbm_gbs")
    out = {"vector_doubles": n,
           "gk_dot": {"ms": round(dot_ms, 4), "GB/s": round(16.0 * n / (dot_ms * 1e-3) / 1e9, 1)},
           "torch_copy": {"ms": round(copy_ms, 4), "GB/s": round(16.0 * n / (copy_ms * 1e-3) / 1e9, 1)},
           "torch_triad": {"ms": round(triad_ms, 4), "GB/s": round(24.0 * n / (triad_ms * 1e-3) / 1e9, 1)}}
    if hbm:
        out["gk_dot"]["frac_of_measured_hbm"] = round(out["gk_dot"]["GB/s"] / hbm, 4)
    del x, y, z
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# replicas (N > 1): one process per GPU, no data-path collective; the timed
# region is bracketed by barriers and the slowest rank's time counts
# ---------------------------------------------------------------------------

def rank_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, bytes_per_rank, seconds):
    """Whole-job GB/s of `world` replicas that each moved bytes_per_rank in
    at most `seconds` (the slowest rank's time)."""
    return world * bytes_per_rank / seconds / 1e9


def run_gpu(args):
    import torch
    import paper_2006_16852_gb300 as gk
    gk.load()
    rank, world, local = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    inp = make_inputs(args.small)
    step = GpuStep(inp, dev, check_every=args.host_loop)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step.run()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    rec = []
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t0.record(step.stream)
    for _ in range(args.steps):
        step.run(record=rec)
    t1.record(step.stream)
    barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(t0.elapsed_time(t1), dist, dev)

    # per-part figures from the recorded events
    part_ms, part_bytes, launches = {}, {}, 0
    iters, outers = {}, {}
    for parts in rec:
        for name, e0, e1, tag in parts:
            part_ms.setdefault(name, []).append(e0.elapsed_time(e1))
            part_bytes.setdefault(name, []).append(step.part_bytes(tag))
            launches += step.part_launches(tag)
            if tag[0] == "solve":
                iters[tag[1]] = tag[2].iters
                if tag[2].outer_iters:
                    outers[tag[1]] = tag[2].outer_iters
                if tag[2].stop_reason != gk.STOP_CONVERGED:
                    raise RuntimeError(f"{tag[1]} did not converge: {tag[2]}")
    step_bytes = sum(sum(v) for v in part_bytes.values()) / args.steps
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, step_bytes, ms_per_step * 1e-3)

    pk = peaks()
    hbm = pk.get("hbm_gbs")
    dom = "spmvdot_a_ell"
    dom_ms = statistics.mean(part_ms[dom]) / SPMV_REPS
    dom_bytes = part_bytes[dom][0] // SPMV_REPS
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    tr = NCU_TRAFFIC.get(spmv_source_hash(), {}).get("dot")
    roofline = {"kernel": "spmv_ell_kernel<EPI_DOT> (ELL SpMV of (a) with the fused dot product: the kernel "
                          "that dominates the step inside the ELL CG solves, timed through gk_apply_dot)",
                "bound": "hbm",
                "achieved": round(achieved, 1), "peak": hbm if hbm else 6800.0, "unit": "GB/s",
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback",
                "frac": round(achieved / (hbm if hbm else 6800.0), 4),
                "traffic": tr, "algorithmic_bytes": dom_bytes, "avg_launch_ms": round(dom_ms, 4)}
    # the same against the nominal HBM rate, and the FP64 co-bound: one FMA
    # per stored entry and one per row (the fused dot), at the nominal FP64
    # rate of a GB300 and at the rate this GPU is measured to retire FP64
    # FMAs (gk_fp64_rate, outside the timed region)
    roofline["frac_of_nominal_hbm"] = round(achieved / NOMINAL_HBM_GBS, 4)
    hbm_floor = dom_bytes / ((hbm or 6800.0) * 1e9) * 1e3
    fmas = step.nnza + step.na
    fp64_floor = 2.0 * fmas / (NOMINAL_FP64_TFLOPS * 1e12) * 1e3
    fp64_rate = step.gk.fp64_rate()
    fp64_floor_meas = 2.0 * fmas / (fp64_rate * 1e12) * 1e3
    effective = max(hbm_floor, fp64_floor_meas)
    roofline["fp64_measured_tflops"] = round(fp64_rate, 4)
    roofline["floors_ms"] = {"hbm": round(hbm_floor, 4), "fp64_fma_nominal": round(fp64_floor, 4),
                             "fp64_fma_measured": round(fp64_floor_meas, 4), "effective": round(effective, 4)}
    roofline["frac_of_effective_floor"] = round(effective / dom_ms, 4)

    def summary(name):
        reps = SPMV_REPS if name.startswith("spmv") else 1
        ms = statistics.median(part_ms[name]) / reps
        by = part_bytes[name][0] / reps
        return {"ms": round(ms, 4), "GB/s": round(by / (ms * 1e-3) / 1e9, 1),
                "frac_hbm": round(by / (ms * 1e-3) / 1e9 / (hbm or 6800.0), 3)}

    spmv = {n[5:]: summary(n) for n in part_ms if n.startswith("spmv_")}
    spmv["a_ell_fused_dot"] = summary("spmvdot_a_ell")
    solves = {}
    for n in part_ms:
        if n.startswith("solve_"):
            s = summary(n)
            s["iters"] = iters[n[6:]]
            if n[6:] in outers:
                s["outer_iters"] = outers[n[6:]]
            solves[n[6:]] = s
    precs = {n[8:]: summary(n) for n in part_ms if n.startswith("precond_")}
    for k, _, bs in step.gens:
        p = precs[f"{k}_bs{bs}"]
        fl = precond_fp64_ops(step.n_of(k), bs)
        p["fp64_floor_ms"] = round(fl / (NOMINAL_FP64_TFLOPS * 0.5e12) * 1e3, 4)
        p["frac_fp64"] = round(p["fp64_floor_ms"] / p["ms"], 3)
        # the same floor at the FP64 rate this GPU is measured to retire
        p["fp64_floor_measured_ms"] = round(fl / (fp64_rate * 0.5e12) * 1e3, 4)
        p["frac_fp64_measured"] = round(p["fp64_floor_measured_ms"] / p["ms"], 3)
    plain = solves["a_cg_plain_csr"]["ms"]
    chosen = min(("a_cg_jacobi_ell", "a_cg_bj8_ell", "a_ircg_jacobi_ell", "a_ircg_bj8_ell"),
                 key=lambda k: solves[k]["ms"])

    # end to end: the same step through the C ABI with pinned host vectors
    host = {}
    for k in ("a", "b"):
        n = step.n_of(k)
        for nm in ("x", "y", "rhs", "x0"):
            host[nm + k] = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        host["x" + k][:] = inp["x" + k]
        host["rhs" + k][:] = step.rhs[k].cpu().numpy()
    h2d = d2h = 0
    for (k, f) in step.mats:
        h2d += SPMV_REPS * 8 * step.n_of(k)
        d2h += SPMV_REPS * 8 * step.n_of(k)
    for name, (S, k, prec, bs, kind, fmt) in step.solvers.items():
        h2d += 16 * step.n_of(k)
        d2h += 8 * step.n_of(k)
    for _ in range(max(1, args.warmup // 2)):
        step.run(host=host)
    barrier()
    e2e_steps = max(1, min(args.steps, 5))
    w0 = time.perf_counter()
    e2e_bytes = 0
    for _ in range(e2e_steps):
        rr = []
        step.run(record=rr, host=host)
        e2e_bytes += sum(step.part_bytes(tag) for _, _, _, tag in rr[0])
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - w0, dist, dev)
    e2e_value = whole_job_rate(world, e2e_bytes / e2e_steps, e2e_s / e2e_steps)

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.small else "small test variant (27-pt 32^3, power-law 2e4)",
                   "formats": {"a": ["csr", "csr_merge", "ell", "hyb"], "b": ["csr_merge", "hyb", "csr"]},
                   "solvers": {k: f"{v[4]} + {v[2]}{'' if v[2] != 'block' else ' bs%d' % v[3]} on ({v[1]}) "
                                  f"in {v[5]}" for k, v in step.solvers.items()},
                   "tolerance": "||r|| <= 1e-10 ||b||, x0 = 0, b = A x*",
                   "l2": "inputs larger than L2 (129 MB): no flush needed",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "frac_hbm": round(value / (hbm or 6800.0), 4),
        "time_to_tol_ms": {"plain_fp64_cg": plain, "chosen_form": chosen, "chosen_ms": solves[chosen]["ms"],
                           "speedup_vs_plain": round(plain / solves[chosen]["ms"], 3)},
        "spmv": spmv, "solves": solves, "precond_generate": precs,
        "paper_table2_cg_bytes_plain": table2_cg_bytes(solves["a_cg_plain_csr"]["iters"], step.nnza, step.na),
        "roofline": roofline,
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
    }
    if not args.no_batched:
        out["batched"] = run_batched(dev)
    if not args.no_mixed:
        out["mixed"] = run_mixed(dev, side=args.mixed_side)
    if not args.no_learned:
        out["learned"] = run_learned(dev)
    if not args.no_krylov:
        out["krylov"] = run_krylov(dev)
    if not args.no_latency:
        out["latency"] = run_latency(dev)
    out["gather_ceiling"] = run_gather_ceiling(step)
    if not args.no_stream:
        out["stream"] = run_stream(dev)
        out["paper_bandwidth"] = run_paper_bandwidth(dev, out["stream"]["torch_triad"]["GB/s"])
    out["paper_context"] = PAPER_CONTEXT
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(inp, args.cpu_budget)
    if dist is not None:
        dist.destroy_process_group()
    return out if rank == 0 else None


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(inp, cg_iters):
    """A bounded slice of the step on the oracle: one SpMV of (a) and of (b)
    and cg_iters Jacobi-CG iterations on (a).  Returns (bytes, seconds)."""
    import oracle
    A, B = inp["a"], inp["b"]
    na, nb = A[0].size - 1, B[0].size - 1
    t0 = time.perf_counter()
    oracle.spmv(A, inp["xa"])
    oracle.spmv(B, inp["xb"])
    b = oracle.spmv(A, inp["xs_a"])
    t1 = time.perf_counter()
    P = oracle.precond(A, "jacobi")
    t2 = time.perf_counter()
    r = oracle.cg(A, b, P=P, tol=1e-10, max_iters=cg_iters)
    t3 = time.perf_counter()
    by = (spmv_bytes(A[1].size, na, na) * 2 + spmv_bytes(B[1].size, nb, nb)
          + cg_bytes(r.iters, A[1].size, na, "jacobi"))
    return by, (t1 - t0) + (t3 - t2), r.iters


def cpu_baseline(inp, budget_s):
    """The oracle on the host's cores: its SpMV row loops on every core
    (OpenMP, static chunks; results unchanged), its dot products and vector
    steps sequential; and the same sample on one thread beside it."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    # size the CG part to about budget_s seconds from two short probes
    _, s2, _ = oracle_sample(inp, 2)
    _, s6, _ = oracle_sample(inp, 6)
    per_it = max((s6 - s2) / 4.0, 1e-4)
    it = max(2, int((budget_s - s2) / per_it))
    by, s, iters = oracle_sample(inp, it)
    oracle.set_threads(1)
    by1, s1, _ = oracle_sample(inp, max(2, it // 4))
    oracle.set_threads(0)
    return {"value": round(by / s / 1e9, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle (plain C; SpMV row loops on {cores} threads, dot products and vector updates "
                      f"sequential): SpMV of (a) x2 and (b) x1, Jacobi-CG on (a) for {iters} iterations; {s:.1f} s",
            "one_thread": {"value": round(by1 / s1 / 1e9, 3), "cores": 1,
                           "sample": f"the same with {max(2, it // 4)} CG iterations on one thread; {s1:.1f} s"}}


def run_reference(args):
    """The oracle timed as the reference arm, on the same metric and config
    (under a multi-process launch rank 0 alone runs it; the others return
    without work).  Its SpMV row loops use every host core."""
    rank = rank_env()[0]
    if rank != 0:
        return None
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    inp = make_inputs(args.small)
    cg_iters = 2
    for _ in range(args.warmup):
        oracle_sample(inp, cg_iters)
    tot_b = tot_s = 0.0
    for _ in range(args.steps):
        b, s, _ = oracle_sample(inp, cg_iters)
        tot_b += b
        tot_s += s
    value = tot_b / tot_s / 1e9
    sample = (f"oracle (plain C; SpMV row loops on {cores} threads, dot products and vector updates sequential), "
              f"per step: SpMV of (a) x2 and (b) x1, Jacobi-CG on (a) for {cg_iters} iterations")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot_s / args.steps * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.small else "small test variant"},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_spmv_only(args):
    """Repeated applies of one matrix/format (for profiler captures)."""
    import torch
    import paper_2006_16852_gb300 as gk
    import workloads as W
    gk.load()
    parts = args.spmv_only.split(":")
    mat, fmt = parts[0], parts[1]
    dot = len(parts) > 2 and parts[2] == "dot"
    if mat == "a":
        A = W.stencil27(128 if not args.small else 32)
    else:
        A = W.powerlaw(1_000_000 if not args.small else 20000, seed=3)
    n = A[0].size - 1
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    M = gk.Matrix(t(A[0]), t(A[1]), t(A[2]), fmt=fmt)
    x, y = t(W.uniform_vector(n, 2)), torch.zeros(n, dtype=torch.float64, device="cuda")
    u, res = t(W.uniform_vector(n, 3)), torch.zeros(1, dtype=torch.float64, device="cuda")
    op = (lambda: gk.apply_dot(M, x, y, u, res)) if dot else (lambda: gk.apply(M, x, y))
    for _ in range(args.warmup):
        op()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        op()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    inf = M.info()
    by = spmv_bytes(A[1].size, n, n, fmt=inf["format_name"],
                    tail_nnz=inf["tail_nnz"] if inf["format_name"] == "hyb" else 0) + (8 * n if dot else 0)
    return {"spmv_only": args.spmv_only, "ms": round(ms, 4), "GB/s": round(by / ms / 1e6, 1),
            "info": M.info()}


def run_infer_only(args):
    """Repeated BF16 inferences of the committed network on a batch (for
    profiler captures of the tensor-core convolution)."""
    import torch
    import paper_2006_16852_gb300 as gk
    from paper_2006_16852_gb300 import learned as LN
    gk.load()
    B = args.infer_only
    net, _, _ = LN.load(os.path.join(LN.DATA_DIR, "wsnet_256.npz"), batch_max=B)
    x = torch.randn((B, 2, net.H, net.W), dtype=torch.float32, device="cuda")
    y = torch.zeros((B, 1, net.H, net.W), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        net.infer_bf16(x, y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        net.infer_bf16(x, y)
    e1.record()
    torch.cuda.synchronize()
    net.check()
    ms = e0.elapsed_time(e1) / args.steps
    macs = net.H * net.W * sum(a * b * 9 for a, b in zip((2, 32, 32, 32, 32, 32), (32, 32, 32, 32, 32, 1)))
    return {"infer_only": B, "ms": round(ms, 4), "TFLOP/s": round(2.0 * B * macs / (ms * 1e-3) / 1e12, 2)}


def run_precond_only(args):
    """Repeated preconditioner generations of matrix a|b (CSR) with one
    block size (profiling aid)."""
    import torch
    import paper_2006_16852_gb300 as gk
    import workloads as W
    gk.load()
    mat, bs = args.precond_only.split(":")
    bs = int(bs)
    if mat == "a":
        A = W.stencil27(128 if not args.small else 32)
    else:
        A = W.powerlaw(1_000_000 if not args.small else 20000, seed=3)
    n = A[0].size - 1
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    M = gk.Matrix(t(A[0]), t(A[1]), t(A[2]), fmt="csr")
    for _ in range(args.warmup):
        gk.Precond(M, bs)
    torch.cuda.synchronize()
    ms = []
    for _ in range(max(args.steps, 1)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P = gk.Precond(M, bs)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        del P
    by = precond_bytes(n, bs, in_block_entries(A, bs))
    med = statistics.median(ms)
    fl = precond_fp64_ops(n, bs)
    return {"precond_only": args.precond_only, "ms": round(med, 4), "GB/s": round(by / (med * 1e-3) / 1e9, 1),
            "fp64_floor_ms": round(fl / (NOMINAL_FP64_TFLOPS * 0.5e12) * 1e3, 4)}


def run_solve_only(args):
    """Repeated solves of one configuration MAT:FMT:PREC:KIND, e.g. a:ell:1:cg
    (MAT a = 27-point 128^3, b = power-law 10^6, c = convection-diffusion
    1024^2; PREC = 0 none, 1 scalar Jacobi, 2..32 block Jacobi), for
    profiling."""
    import torch
    import paper_2006_16852_gb300 as gk
    import workloads as W
    gk.load()
    mat, fmt, prec, kind = args.solve_only.split(":")
    prec = int(prec)
    if mat == "a":
        A = W.stencil27(128 if not args.small else 32)
    elif mat == "c":
        A = W.convdiff2d(1024 if not args.small else 128, 0.5)
    else:
        A = W.powerlaw(1_000_000 if not args.small else 20000, seed=3)
    n = A[0].size - 1
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    M = gk.Matrix(t(A[0]), t(A[1]), t(A[2]), fmt=fmt)
    P = gk.Precond(M, prec) if prec else None
    S = gk.Solver(M, P, kind, max_iters=5000, reduction_factor=1e-10, check_every=args.host_loop)
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    gk.apply(M, t(W.uniform_vector(n, 4)), b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        x.zero_()
        gk.solve(S, b, x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        x.zero_()
        st = gk.solve(S, b, x)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    return {"solve_only": args.solve_only, "ms": round(ms, 3), "iters": st.iters,
            "us_per_iter": round(1e3 * ms / max(st.iters, 1), 2), "stop": st.stop_reason,
            "rel_res_true": st.rel_res_true}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gk", "reference"], default="gk")
    ap.add_argument("--small", action="store_true", help="small matrices (quick checks)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched small-system solves")
    ap.add_argument("--batched-only", action="store_true", help="only the batched small-system solves")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision workload")
    ap.add_argument("--mixed-only", action="store_true", help="only the mixed-precision workload")
    ap.add_argument("--mixed-side", type=int, default=256, help="grid side of the mixed-precision workload")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm start")
    ap.add_argument("--no-krylov", action="store_true", help="skip the FCG / CGS / GMRES section")
    ap.add_argument("--krylov-only", action="store_true", help="only the FCG / CGS / GMRES section")
    ap.add_argument("--no-latency", action="store_true", help="skip the per-iteration latency section")
    ap.add_argument("--no-stream", action="store_true",
                    help="skip the stream probes and the paper's solver-bandwidth experiment")
    ap.add_argument("--paper-only", action="store_true",
                    help="only the stream probes and the paper's solver-bandwidth experiment")
    ap.add_argument("--infer-only", type=int, default=0, metavar="B",
                    help="only BF16 inferences of the committed network on a batch of B (profiling)")
    ap.add_argument("--latency-only", action="store_true", help="only the per-iteration latency section")
    ap.add_argument("--learned-only", action="store_true", help="only the learned warm start")
    ap.add_argument("--batch-systems", type=int, default=10000, help="--batched-only: number of systems")
    ap.add_argument("--batch-forms", default=None, help="--batched-only: comma list of " + ", ".join(BATCH_FORMS))
    ap.add_argument("--batch-no-tune", action="store_true",
                    help="--batched-only: default block sizes instead of the autotuner")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle CG in cpu_baseline")
    ap.add_argument("--spmv-only", metavar="MAT:FMT[:dot]", default=None,
                    help="only time repeated applies of matrix a|b in one format, with ':dot' the apply "
                         "with the fused dot product of the Krylov steps (profiling aid)")
    ap.add_argument("--precond-only", metavar="MAT:BS", default=None,
                    help="only time repeated preconditioner generations of matrix a|b (profiling aid)")
    ap.add_argument("--solve-only", metavar="MAT:FMT:PREC:KIND", default=None,
                    help="only time repeated solves of one configuration (profiling aid)")
    ap.add_argument("--host-loop", type=int, default=0, metavar="K",
                    help="launch solver iterations from the host, reading the stop flag every K "
                         "iterations, instead of the device-side graph loop (profilers cannot see "
                         "kernels inside conditional graph nodes)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gk" and not args.small:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.krylov_only or args.latency_only:
        import torch
        import paper_2006_16852_gb300 as gk
        gk.load()
        run = run_krylov if args.krylov_only else run_latency
        out = run(torch.device("cuda:0"))
    elif args.paper_only:
        import torch
        import paper_2006_16852_gb300 as gk
        gk.load()
        dev = torch.device("cuda:0")
        st = run_stream(dev)
        out = {"stream": st, "paper_bandwidth": run_paper_bandwidth(dev, st["torch_triad"]["GB/s"]),
               "paper_context": PAPER_CONTEXT}
    elif args.learned_only:
        import torch
        import paper_2006_16852_gb300 as gk
        gk.load()
        out = run_learned(torch.device("cuda:0"))
    elif args.mixed_only:
        import torch
        import paper_2006_16852_gb300 as gk
        gk.load()
        out = run_mixed(torch.device("cuda:0"), side=args.mixed_side)
    elif args.batched_only:
        import torch
        import paper_2006_16852_gb300 as gk
        gk.load()
        out = run_batched(torch.device("cuda:0"), n_sys=args.batch_systems,
                          only=args.batch_forms.split(",") if args.batch_forms else None,
                          tune=not args.batch_no_tune, plain=not args.batch_forms)
    elif args.spmv_only:
        out = run_spmv_only(args)
    elif args.infer_only:
        out = run_infer_only(args)
    elif args.solve_only:
        out = run_solve_only(args)
    elif args.precond_only:
        out = run_precond_only(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
