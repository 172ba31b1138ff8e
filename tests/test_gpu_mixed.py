"""GPU parity of the mixed-precision refinement solver (GK_IR_CG) against the
oracle's FP64-outer / FP32-inner refinement, and of its adaptive FP16/FP32
block storage decisions (bit-exact: the inverse blocks are bit-identical and
kappa_1 is summed in the same order)."""
import numpy as np
import pytest

import workloads as W
from helpers import to_dev, to_np

pytestmark = pytest.mark.gpu


def _gk_ir(gk, A, b, fmt, prec, **crit):
    n = A[0].size - 1
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt=fmt)
    P = gk.Precond(M, prec) if prec else None
    S = gk.Solver(M, P, "ir_cg", **crit)
    x = to_dev(np.zeros(n))
    st = gk.solve(S, to_dev(b), x)
    return st, to_np(x), S.info()


CASES = {
    "poisson64": (W.poisson2d(64), 1711.7),
    "stencil27_20": (W.stencil27(20), 400.0),
    "powerlaw_20000": (W.powerlaw(20000, seed=5), 50.0),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("fmt", ["ell", "hyb", "csr", "csr_merge"])
@pytest.mark.parametrize("prec", [0, 1, 8])
def test_ir_cg_matches_oracle(gk, orc, name, fmt, prec):
    A, kappa = CASES[name]
    if fmt == "ell" and name == "powerlaw_20000":
        pytest.skip("ELL refuses the power-law matrix")
    n = A[0].size - 1
    xs = W.uniform_vector(n, 3)
    b = orc.spmv(A, xs)
    st, x, info = _gk_ir(gk, A, b, fmt, prec, max_iters=20000, reduction_factor=1e-10)
    P = orc.precond(A, {0: "none", 1: "jacobi", 8: "block_jacobi"}[prec], 8)
    ref, outer = orc.ir_cg(A, b, P=P, tol=1e-10)
    assert st.stop_reason == gk.STOP_CONVERGED == ref.stop_reason
    assert st.rel_res_true <= 1e-10
    assert abs(st.outer_iters - outer) <= 1, (st.outer_iters, outer)
    assert abs(st.iters - ref.iters) <= max(5, ref.iters // 8), (st.iters, ref.iters)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 2e-10
    assert info["inner_format"] == (2 if fmt in ("ell", "hyb") else 0)


@pytest.mark.parametrize("name,bs", [("poisson64", 4), ("poisson64", 8), ("stencil27_20", 16),
                                     ("powerlaw_20000", 4), ("tridiag", 4), ("tridiag", 8)])
def test_adaptive_block_precision_matches_oracle(gk, orc, name, bs):
    A = W.poisson1d(1000) if name == "tridiag" else CASES[name][0]
    n = A[0].size - 1
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt="csr")
    S = gk.Solver(M, gk.Precond(M, bs), "ir_cg")
    info = S.info()
    blocks = orc.block_jacobi(A, bs)
    prec, _ = orc.block_jacobi_precision(A, bs, blocks)
    assert info["inner_fp16_blocks"] == int((prec == 0).sum())
    assert info["inner_fp32_blocks"] == int((prec == 1).sum())
    assert info["inner_fp16_blocks"] + info["inner_fp32_blocks"] == (n + bs - 1) // bs


def test_ir_edge_cases(gk, orc):
    A = W.poisson2d(16)
    xs = W.uniform_vector(256, 1)
    b = orc.spmv(A, xs)
    # exact initial guess: the first FP64 residual is zero
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]))
    S = gk.Solver(M, None, "ir_cg")
    x = to_dev(xs)
    st = gk.solve(S, to_dev(b), x)
    assert st.stop_reason == gk.STOP_CONVERGED and st.iters == 0 and st.outer_iters == 0
    # NaN right-hand side
    st, _, _ = _gk_ir(gk, A, np.full(256, np.nan), "csr", 1)
    assert st.stop_reason == gk.STOP_NAN
    # iteration limit on the inner total
    st, _, _ = _gk_ir(gk, A, b, "csr", 1, max_iters=5, reduction_factor=1e-14)
    assert st.stop_reason == gk.STOP_MAX_ITERS
    # loose inner solves need more outer steps
    s1, _, _ = _gk_ir(gk, A, b, "csr", 1, inner_reduction=1e-2)
    s2, _, _ = _gk_ir(gk, A, b, "csr", 1, inner_reduction=1e-6)
    assert s1.stop_reason == s2.stop_reason == gk.STOP_CONVERGED and s1.outer_iters > s2.outer_iters


@pytest.mark.parametrize("bs", [8, 16, 32])
def test_ir_varcoef3d_adaptive_blocks_to_1e12(gk, orc, bs):
    """The mixed-precision workload's operator (7-point, log-normal sigma = 1
    coefficients) at 24^3: refinement with adaptive FP16/FP32 block Jacobi to
    1e-12 -- the oracle's FP16/FP32 split exactly, its number of refinement
    steps within 1, and the FP64 criterion met on the true residual."""
    A = W.varcoef3d(24, sigma=1.0, seed=4)
    n = A[0].size - 1
    xs = W.uniform_vector(n, 3)
    b = orc.spmv(A, xs)
    st, x, info = _gk_ir(gk, A, b, "ell", bs, max_iters=100000, reduction_factor=1e-12)
    P = orc.precond(A, "block_jacobi", bs)
    prec, _ = orc.block_jacobi_precision(A, bs, P.blocks)
    ref, outer = orc.ir_cg(A, b, P=P, tol=1e-12, max_iters=100000)
    assert info["inner_fp16_blocks"] == int((prec == 0).sum()) > 0
    assert info["inner_fp32_blocks"] == int((prec == 1).sum())
    assert st.stop_reason == gk.STOP_CONVERGED == ref.stop_reason
    assert abs(st.outer_iters - outer) <= 1, (st.outer_iters, outer)
    assert abs(st.iters - ref.iters) <= max(5, ref.iters // 8), (st.iters, ref.iters)
    r = b - orc.spmv(A, x)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)
    assert np.linalg.norm(x - ref.x) <= 1e-6 * np.linalg.norm(ref.x)


def test_ir_varcoef3d_full_size(gk, orc):
    """The mixed-precision workload at its full size (256^3, n = 16,777,216,
    nnz = 117,047,296), refinement with adaptive block Jacobi (bs 16) to
    1e-12: the FP16/FP32 decisions of all 1,048,576 blocks equal the
    oracle's, and the oracle's FP64 SpMV confirms the residual."""
    A = W.varcoef3d(256, sigma=1.0, seed=4)
    n = A[0].size - 1
    assert n == 16_777_216 and A[1].size == 117_047_296
    b = W.uniform_vector(n, 7)
    st, x, info = _gk_ir(gk, A, b, "ell", 16, max_iters=200000, reduction_factor=1e-12)
    P = orc.precond(A, "block_jacobi", 16)
    prec, _ = orc.block_jacobi_precision(A, 16, P.blocks)
    assert info["inner_fp16_blocks"] == int((prec == 0).sum())
    assert info["inner_fp32_blocks"] == int((prec == 1).sum())
    assert st.stop_reason == gk.STOP_CONVERGED
    r = b - orc.spmv(A, x)
    assert np.linalg.norm(r) <= 1.2e-12 * np.linalg.norm(b)


def test_ir_host_loop_equals_graph_loop(gk, orc):
    """The refinement launched from the host (check_every > 0) runs the same
    kernels as the device-controlled graph loop: bit-identical results."""
    A = W.stencil27(20)
    n = A[0].size - 1
    b = orc.spmv(A, W.uniform_vector(n, 4))
    for prec in (1, 8):
        s1, x1, _ = _gk_ir(gk, A, b, "ell", prec, max_iters=20000, reduction_factor=1e-10)
        s2, x2, _ = _gk_ir(gk, A, b, "ell", prec, max_iters=20000, reduction_factor=1e-10, check_every=7)
        assert s1.iters == s2.iters and s1.outer_iters == s2.outer_iters
        np.testing.assert_array_equal(x1, x2)
