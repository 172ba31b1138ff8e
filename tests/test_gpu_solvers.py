"""GPU parity of the CG and BiCGSTAB solver operators (Section 3.1) against
the oracle, and the stopping criteria of Section 2.5.

The GPU sums dot products in a fixed tree order and the oracle sequentially,
so iterates differ by rounding.  What is compared: the stop reason; the
iteration count within max(2, 3%) of the oracle's; the true relative residual
(<= 1e-10 * 1.5 at a 1e-10 target); and the solution against the oracle's and
the manufactured one to kappa * tol.  Invariants that hold bit for bit on the
GPU itself are checked bit for bit.
"""
import math

import numpy as np
import pytest

import workloads as W
from helpers import to_dev, to_np

pytestmark = pytest.mark.gpu


def _kappa_poisson2d(m):
    lmin = 4 - 4 * math.cos(math.pi / (m + 1))
    lmax = 4 + 4 * math.cos(math.pi / (m + 1))
    return lmax / lmin


def _solve(gk, A, b, x0=None, fmt="csr", prec=None, kind="cg", **crit):
    n = A[0].size - 1
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt=fmt)
    P = gk.Precond(M, prec) if prec else None
    S = gk.Solver(M, P, kind, **crit)
    x = to_dev(np.zeros(n) if x0 is None else x0)
    st = gk.solve(S, to_dev(b), x)
    return st, to_np(x)


def _iters_close(a, b):
    return abs(a - b) <= max(2, int(0.03 * max(a, b)))


@pytest.mark.parametrize("fmt", ["csr", "csr_merge", "ell", "hyb"])
@pytest.mark.parametrize("prec", [None, 1, 8])
def test_cg_poisson_matches_oracle(gk, orc, fmt, prec):
    A = W.poisson2d(64)
    xs = W.uniform_vector(4096, 1)
    b = orc.spmv(A, xs)
    st, x = _solve(gk, A, b, fmt=fmt, prec=prec, max_iters=2000, reduction_factor=1e-10)
    P = orc.precond(A, {None: "none", 1: "jacobi", 8: "block_jacobi"}[prec], 8)
    ref = orc.cg(A, b, P=P, tol=1e-10, max_iters=2000)
    assert st.stop_reason == gk.STOP_CONVERGED == ref.stop_reason
    assert _iters_close(st.iters, ref.iters), (st.iters, ref.iters)
    assert st.spmvs == st.iters + 2
    assert st.rel_res <= 1e-10 and st.rel_res_true <= 1.5e-10
    kappa = _kappa_poisson2d(64)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= kappa * 2e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 2e-10


def test_cg_jacobi_bit_identical_to_plain_on_poisson(gk):
    """a_ii = 4: scaling by 1/4 is exact in every product and sum of the GPU
    kernels too, so Jacobi-PCG must reproduce plain CG bit for bit; block
    Jacobi with bs = 1 is the same operator."""
    A = W.poisson2d(64)
    b = W.uniform_vector(4096, 2)
    s0, x0 = _solve(gk, A, b, prec=None)
    s1, x1 = _solve(gk, A, b, prec=1)
    assert s0.iters == s1.iters and np.array_equal(x0, x1)


def test_host_loop_equals_graph_loop(gk):
    A = W.poisson2d(48)
    b = W.uniform_vector(48 * 48, 3)
    for kind in ("cg", "bicgstab"):
        s0, x0 = _solve(gk, A, b, kind=kind, prec=1, check_every=-1)
        s1, x1 = _solve(gk, A, b, kind=kind, prec=1, check_every=7)
        assert s0.iters == s1.iters and np.array_equal(x0, x1), kind
        # kernels launched after the stop: the graph runs whole passes of four
        # CG iterations (one pass at least), the host loop whole groups of 7
        if kind == "cg":
            assert 0 <= s0.idle_iters < 4 and (s0.iters + s0.idle_iters) % 4 == 0, (s0.iters, s0.idle_iters)
        else:
            assert s0.idle_iters == 0
        assert 0 <= s1.idle_iters < 7 and (s1.iters + s1.idle_iters) % 7 == 0, (s1.iters, s1.idle_iters)


@pytest.mark.parametrize("max_iters", [0, 1, 5, 6, 7])
@pytest.mark.parametrize("prec", [None, 1, 4])
def test_graph_passes_stop_mid_pass(gk, prec, max_iters):
    """The graph's loop body holds four CG iterations; a stop inside a pass
    (here the iteration limit, and an exact x0 that stops at k = 0) leaves
    the rest of the pass without effect: iterations, status and x equal the
    host loop's with a status read after every iteration."""
    A = W.poisson2d(40)
    b = W.uniform_vector(1600, 8)
    s0, x0 = _solve(gk, A, b, prec=prec, check_every=-1, max_iters=max_iters, reduction_factor=1e-12)
    s1, x1 = _solve(gk, A, b, prec=prec, check_every=1, max_iters=max_iters, reduction_factor=1e-12)
    assert s0.stop_reason == s1.stop_reason == gk.STOP_MAX_ITERS
    assert s0.iters == s1.iters == max_iters
    assert s0.rel_res == s1.rel_res and np.array_equal(x0, x1)
    assert s0.idle_iters == (4 if max_iters == 0 else -max_iters % 4), s0.idle_iters
    _, xs = _solve(gk, A, b, prec=prec, check_every=-1, max_iters=500, reduction_factor=1e-12)
    s2, x2 = _solve(gk, A, b, x0=xs, prec=prec, check_every=-1, max_iters=50, reduction_factor=1e-2)
    assert s2.stop_reason == gk.STOP_CONVERGED and s2.iters == 0 and s2.idle_iters == 4
    assert np.array_equal(x2, xs)


@pytest.mark.parametrize("prec", [None, 1, 4, 16])
@pytest.mark.parametrize("fmt", ["csr", "csr_merge", "hyb"])
def test_bicgstab_nonsymmetric_matches_oracle(gk, orc, prec, fmt):
    A = W.convdiff2d(40, wind=2.0)
    D = W.csr_to_dense(A)
    xs = W.uniform_vector(1600, 4)
    b = orc.spmv(A, xs)
    st, x = _solve(gk, A, b, fmt=fmt, prec=prec, kind="bicgstab", max_iters=3000, reduction_factor=1e-10)
    P = orc.precond(A, {None: "none", 1: "jacobi"}.get(prec, "block_jacobi"), prec or 1)
    ref = orc.bicgstab(A, b, P=P, tol=1e-10, max_iters=3000)
    assert st.stop_reason == gk.STOP_CONVERGED == ref.stop_reason
    assert _iters_close(st.iters, ref.iters), (st.iters, ref.iters)
    assert st.rel_res_true <= 2e-10
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 2e-10


def test_cg_powerlaw_matches_oracle(gk, orc):
    A = W.powerlaw(20000, seed=5)
    b = W.uniform_vector(20000, 6)
    for fmt in ("csr_merge", "hyb", "csr"):
        st, x = _solve(gk, A, b, fmt=fmt, prec=1, max_iters=500)
        ref = orc.cg(A, b, P=orc.precond(A, "jacobi"), tol=1e-10, max_iters=500)
        assert st.stop_reason == gk.STOP_CONVERGED
        assert _iters_close(st.iters, ref.iters)
        assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-8


def test_powerlaw_csr_graph_form_matches_oracle(gk, orc):
    """GK_CSR inside the large-system solve graph on a power-law matrix whose
    longest rows are summed in pieces (the pieces' second launch finishes the
    fused dot and residual reductions): Jacobi-CG and block-Jacobi (bs 4)
    BiCGSTAB against the oracle, with 300,000 rows (past the one-launch forms)."""
    A = W.powerlaw(300_000, seed=7)
    n = A[0].size - 1
    assert (np.diff(A[0]) > 512).sum() > 100
    xs = W.uniform_vector(n, 8)
    b = orc.spmv(A, xs)
    for kind, bs in (("cg", 1), ("bicgstab", 4)):
        st, x = _solve(gk, A, b, fmt="csr", prec=bs, kind=kind, max_iters=2000, reduction_factor=1e-10)
        assert st.stop_reason == gk.STOP_CONVERGED, kind
        assert np.linalg.norm(b - orc.spmv(A, x)) <= 1.5e-10 * np.linalg.norm(b), kind
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-8, kind
        P = orc.precond(A, "jacobi" if bs == 1 else "block_jacobi", bs)
        ref = (orc.cg if kind == "cg" else orc.bicgstab)(A, b, P=P, tol=1e-10, max_iters=2000)
        slack = max(2, ref.iters * 3 // 100) if kind == "cg" else max(3, ref.iters // 4)
        assert abs(st.iters - ref.iters) <= slack, (kind, st.iters, ref.iters)


def test_criteria_edge_cases(gk, orc):
    A = W.poisson2d(8)
    xs = W.uniform_vector(64, 5)
    b = orc.spmv(A, xs)
    # max_iters = 0: nothing changes
    x0 = W.uniform_vector(64, 6)
    st, x = _solve(gk, A, b, x0=x0, max_iters=0)
    assert st.iters == 0 and st.stop_reason == gk.STOP_MAX_ITERS and np.array_equal(x, x0)
    # x0 = exact solution: r_0 = b - A x* = 0 exactly (binned rows sum in the oracle's order)
    st, x = _solve(gk, A, b, x0=xs)
    assert st.iters == 0 and st.stop_reason == gk.STOP_CONVERGED and np.array_equal(x, xs)
    # NaN right-hand side (Section 7.2's set-up) ends with NAN, never hangs
    for kind in ("cg", "bicgstab"):
        st, _ = _solve(gk, A, np.full(64, np.nan), kind=kind, max_iters=1000)
        assert st.stop_reason == gk.STOP_NAN and st.iters == 0
    # n = 1
    st, x = _solve(gk, W.diagonal([3.0]), np.array([6.0]))
    assert st.iters == 1 and x[0] == 2.0
    # iteration limit
    st, _ = _solve(gk, A, b, max_iters=3, reduction_factor=1e-14)
    assert st.iters == 3 and st.stop_reason == gk.STOP_MAX_ITERS
    # breakdown on an indefinite matrix
    st, _ = _solve(gk, W.diagonal([1.0, -1.0]), np.array([1.0, 1.0]))
    assert st.stop_reason == gk.STOP_BREAKDOWN
    # BiCGSTAB half step on c*I
    st, x = _solve(gk, W.scaled_identity(50, 3.0), np.ones(50), kind="bicgstab")
    assert st.iters == 1 and st.spmvs == 3 and st.stop_reason == gk.STOP_CONVERGED


def test_time_criterion_on_device(gk):
    A = W.stencil27(40)
    b = W.uniform_vector(64000, 7)
    st, _ = _solve(gk, A, b, max_iters=100000, reduction_factor=1e-300, time_limit_s=0.002)
    assert st.stop_reason == gk.STOP_TIME and 0 < st.iters < 100000


def test_host_vectors_in_solve(gk, orc):
    A = W.poisson2d(32)
    b = W.uniform_vector(1024, 8)
    M = gk.Matrix(A[0], A[1], A[2])
    S = gk.Solver(M, gk.Precond(M, 1), "cg")
    x = np.zeros(1024)
    st = gk.solve(S, b, x)
    assert st.stop_reason == gk.STOP_CONVERGED and st.rel_res_true <= 1.5e-10
    ref = orc.cg(A, b, tol=1e-10)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= _kappa_poisson2d(32) * 2e-10


def test_cg_full_size_stencil27(gk):
    """The benchmark's CG: 27-point stencil on 128^3 to 1e-10, manufactured
    solution; kappa from the closed-form spectrum 27 - prod_d (1 + 2 cos(k_d pi/129))."""
    N = 128
    A = W.stencil27(N)
    n = N ** 3
    xs = W.uniform_vector(n, 2)
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt="csr")
    bt = to_dev(np.zeros(n))
    gk.apply(M, to_dev(xs), bt)
    S = gk.Solver(M, gk.Precond(M, 1), "cg", max_iters=2000, reduction_factor=1e-10)
    x = to_dev(np.zeros(n))
    st = gk.solve(S, bt, x)
    c = 1 + 2 * math.cos(math.pi / (N + 1))
    lmin = 27 - c ** 3
    lmax = 27 + c * c  # two factors near 3 and one near -1
    kappa = lmax / lmin
    assert st.stop_reason == gk.STOP_CONVERGED and st.rel_res_true <= 1.5e-10
    err = np.linalg.norm(to_np(x) - xs) / np.linalg.norm(xs)
    assert err <= kappa * 2e-10, (err, kappa)


def test_powerlaw_full_size_solves(gk, orc):
    """The benchmark's solves on (b), the power-law matrix with 10^6 rows, in
    the benchmark's formats and preconditioners: Jacobi-CG and block-Jacobi
    (bs 4) BiCGSTAB on HYB to 1e-10 from b = A x*.  Iteration counts against
    the oracle's (max(2, 3 %) for CG, max(3, 25 %) for BiCGSTAB), the true
    residual with the oracle's SpMV, and the forward error (the matrix is
    strictly diagonally dominant, so well conditioned)."""
    A = W.powerlaw(1_000_000, seed=3)
    n = A[0].size - 1
    xs = W.uniform_vector(n, 5)
    b = orc.spmv(A, xs)
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt="hyb")
    for kind, bs in (("cg", 1), ("bicgstab", 4)):
        S = gk.Solver(M, gk.Precond(M, bs), kind, max_iters=5000, reduction_factor=1e-10)
        x = to_dev(np.zeros(n))
        st = gk.solve(S, to_dev(b), x)
        x = to_np(x)
        assert st.stop_reason == gk.STOP_CONVERGED, kind
        assert np.linalg.norm(b - orc.spmv(A, x)) <= 1.5e-10 * np.linalg.norm(b), kind
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-8, kind
        P = orc.precond(A, "jacobi" if bs == 1 else "block_jacobi", bs)
        ref = (orc.cg if kind == "cg" else orc.bicgstab)(A, b, P=P, tol=1e-10, max_iters=5000)
        slack = max(2, ref.iters * 3 // 100) if kind == "cg" else max(3, ref.iters // 4)
        assert abs(st.iters - ref.iters) <= slack, (kind, st.iters, ref.iters)


@pytest.mark.parametrize("kind", ["cg", "bicgstab"])
@pytest.mark.parametrize("every", [0, -1])
def test_reduction_relative_to_initial_residual(gk, orc, kind, every):
    """ResidualNormReduction against ||r_0|| (Section 2.5's reading, rel_to_b
    off) from a nonzero x0, in the one-launch form (check_every 0) and the
    graph (-1): ref is ||b - A x0||, the stop is ||r_k|| <= 1e-8 ||r_0||, and
    the iteration count follows the oracle's under the same criterion."""
    A = W.poisson2d(48) if kind == "cg" else W.convdiff2d(40, wind=1.0)
    n = A[0].size - 1
    xs = W.uniform_vector(n, 21)
    b = orc.spmv(A, xs)
    x0 = xs + 0.1 * W.uniform_vector(n, 22)
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]))
    S = gk.Solver(M, gk.Precond(M, 1), kind, max_iters=3000, reduction_factor=1e-8, rel_to_b=False,
                  check_every=every)
    x = to_dev(x0.copy())
    st = gk.solve(S, to_dev(b), x)
    r0 = np.linalg.norm(b - orc.spmv(A, x0))
    assert st.stop_reason == gk.STOP_CONVERGED
    assert abs(st.ref_norm - r0) <= 1e-12 * r0
    assert st.rel_res <= 1e-8 and st.rel_res_true <= 1.5e-8
    P = orc.precond(A, "jacobi")
    ref = (orc.cg if kind == "cg" else orc.bicgstab)(A, b, x0=x0, P=P, tol=1e-8, max_iters=3000, rel_to_b=False)
    slack = max(2, ref.iters * 3 // 100) if kind == "cg" else max(3, ref.iters // 4)
    assert abs(st.iters - ref.iters) <= slack, (st.iters, ref.iters)
    if every == 0:
        assert st.form == gk.FORM_CLUSTER


# The benchmark step's solves on (a), the 27-point stencil on 128^3: format,
# preconditioner (block size, 0 = none) and method, exactly as the step runs
# them, each against the oracle's run of the same method.
STEP_SOLVES_A = {
    "cg_plain_csr": ("csr", 0, "cg"),
    "cg_jacobi_ell": ("ell", 1, "cg"),
    "cg_bj8_ell": ("ell", 8, "cg"),
    "ircg_jacobi_ell": ("ell", 1, "ir_cg"),
    "ircg_bj8_ell": ("ell", 8, "ir_cg"),
}


@pytest.fixture(scope="module")
def stencil27_full(orc):
    """(a) with the benchmark's right-hand side b = A x*, x* uniform (seed 4),
    and kappa from the closed-form spectrum 27 - prod_d (1 + 2 cos(k_d pi/129))."""
    N = 128
    A = W.stencil27(N)
    xs = W.uniform_vector(N ** 3, 4)
    b = orc.spmv(A, xs)
    c = 1 + 2 * math.cos(math.pi / (N + 1))
    kappa = (27 + c * c) / (27 - c ** 3)
    return {"A": A, "xs": xs, "b": b, "kappa": kappa, "mats": {}}


@pytest.mark.parametrize("name", list(STEP_SOLVES_A))
def test_stencil27_full_size_step_solves_match_oracle(gk, orc, stencil27_full, name):
    """Every solve of the benchmark step on (a) at its full size (n =
    2,097,152, nnz = 55,742,968), in the step's format and preconditioner,
    to 1e-10 against the oracle: the same stop reason; iterations within
    max(2, 3 %) (CG), or refinement steps within 1 and inner iterations no
    more than the oracle's + max(5, 1/8) (refinement: see below); the true residual <= 1.5e-10 by the oracle's SpMV; and the
    solution within kappa * 2e-10 of the oracle's and of x*."""
    D = stencil27_full
    A, b, xs, kappa = D["A"], D["b"], D["xs"], D["kappa"]
    fmt, bs, kind = STEP_SOLVES_A[name]
    n = A[0].size - 1
    if fmt not in D["mats"]:
        D["mats"][fmt] = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt=fmt)
    M = D["mats"][fmt]
    S = gk.Solver(M, gk.Precond(M, bs) if bs else None, kind, max_iters=5000, reduction_factor=1e-10)
    xt = to_dev(np.zeros(n))
    st = gk.solve(S, to_dev(b), xt)
    x = to_np(xt)
    P = orc.precond(A, {0: "none", 1: "jacobi", 8: "block_jacobi"}[bs], max(bs, 1))
    if kind == "cg":
        ref = orc.cg(A, b, P=P, tol=1e-10, max_iters=5000)
        assert _iters_close(st.iters, ref.iters), (name, st.iters, ref.iters)
    else:
        # The oracle sums the FP32 inner dot products sequentially; over n =
        # 2,097,152 terms that sum's error reaches ~n u_32 of the sum of
        # magnitudes, which slows its FP32 CG (347 inner iterations with
        # Jacobi), while the GPU's blocked tree sums converge like FP32 CG
        # with accurate sums (263; a copy of the oracle with 1024-term
        # blocked float sums also takes 263).  So the inner count may be
        # lower than the oracle's, not higher.
        ref, outer = orc.ir_cg(A, b, P=P, tol=1e-10)
        assert abs(st.outer_iters - outer) <= 1, (name, st.outer_iters, outer)
        assert ref.iters // 2 <= st.iters <= ref.iters + max(5, ref.iters // 8), (name, st.iters, ref.iters)
    assert st.stop_reason == gk.STOP_CONVERGED == ref.stop_reason, name
    assert st.rel_res_true <= 1.5e-10, name
    assert np.linalg.norm(b - orc.spmv(A, x)) <= 1.5e-10 * np.linalg.norm(b), name
    assert np.linalg.norm(x - ref.x) <= kappa * 2e-10 * np.linalg.norm(ref.x), name
    assert np.linalg.norm(x - xs) <= kappa * 2e-10 * np.linalg.norm(xs), name
