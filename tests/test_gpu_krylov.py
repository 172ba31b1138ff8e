"""GPU parity of flexible CG, CGS and restarted GMRES (Section 3.1) against
the oracle.  Reductions are tree-ordered on the GPU and sequential in the
oracle, so the comparison is: the stop reason, the iteration count (within
max(2, 3 %) for FCG and GMRES, within max(3, 15 %) for CGS, whose residual
is irregular), the true relative residual at the 1e-10 target, and the
solution against the oracle's and the manufactured one."""
import numpy as np
import pytest

import workloads as W
from helpers import to_dev, to_np

pytestmark = pytest.mark.gpu


def _solve(gk, A, b, kind, fmt="csr", prec=None, x0=None, **crit):
    n = A[0].size - 1
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt=fmt)
    P = gk.Precond(M, prec) if prec else None
    S = gk.Solver(M, P, kind, **crit)
    x = to_dev(np.zeros(n) if x0 is None else x0)
    st = gk.solve(S, to_dev(b), x)
    return st, to_np(x)


def _oprec(orc, A, prec):
    return orc.precond(A, {None: "none", 1: "jacobi"}.get(prec, "block_jacobi"), prec or 1)


@pytest.mark.parametrize("fmt", ["csr", "ell", "hyb", "csr_merge"])
@pytest.mark.parametrize("prec", [None, 1, 8])
def test_fcg_matches_oracle(gk, orc, fmt, prec):
    A = W.poisson2d(64)
    xs = W.uniform_vector(4096, 1)
    b = orc.spmv(A, xs)
    st, x = _solve(gk, A, b, "fcg", fmt, prec, max_iters=2000, reduction_factor=1e-10)
    ref = orc.fcg(A, b, P=_oprec(orc, A, prec), tol=1e-10, max_iters=2000)
    cg = orc.cg(A, b, P=_oprec(orc, A, prec), tol=1e-10, max_iters=2000)
    assert st.stop_reason == ref.stop_reason == gk.STOP_CONVERGED
    assert abs(st.iters - ref.iters) <= max(2, ref.iters // 33), (st.iters, ref.iters)
    assert abs(st.iters - cg.iters) <= max(2, cg.iters // 33)
    assert st.rel_res_true <= 1.5e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1712 * 2e-10


@pytest.mark.parametrize("fmt", ["csr", "ell", "hyb"])
@pytest.mark.parametrize("prec", [None, 1, 4])
def test_cgs_matches_oracle(gk, orc, fmt, prec):
    A = W.convdiff2d(48, 0.5)
    n = A[0].size - 1
    xs = W.uniform_vector(n, 2)
    b = orc.spmv(A, xs)
    st, x = _solve(gk, A, b, "cgs", fmt, prec, max_iters=2000, reduction_factor=1e-10)
    ref = orc.cgs(A, b, P=_oprec(orc, A, prec), tol=1e-10, max_iters=2000)
    assert st.stop_reason == ref.stop_reason == gk.STOP_CONVERGED
    assert abs(st.iters - ref.iters) <= max(3, ref.iters * 15 // 100), (st.iters, ref.iters)
    assert st.spmvs == 2 * st.iters + 2
    assert st.rel_res_true <= 5e-10
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-7


@pytest.mark.parametrize("fmt", ["csr", "ell", "hyb"])
@pytest.mark.parametrize("prec", [None, 1, 4])
@pytest.mark.parametrize("m", [10, 30])
def test_gmres_matches_oracle(gk, orc, fmt, prec, m):
    A = W.convdiff2d(48, 0.5)
    n = A[0].size - 1
    xs = W.uniform_vector(n, 3)
    b = orc.spmv(A, xs)
    st, x = _solve(gk, A, b, "gmres", fmt, prec, max_iters=5000, reduction_factor=1e-10, krylov_dim=m)
    ref = orc.gmres(A, b, P=_oprec(orc, A, prec), tol=1e-10, max_iters=5000, krylov_dim=m)
    assert st.stop_reason == ref.stop_reason == gk.STOP_CONVERGED
    assert abs(st.iters - ref.iters) <= max(2, ref.iters // 33), (st.iters, ref.iters)
    assert st.rel_res_true <= 1e-10 * 1.0001
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-8


def test_gmres_unrestarted_finite_termination(gk, orc):
    """Five distinct eigenvalues: at most five Arnoldi steps, x = b / d."""
    d = np.repeat([1.0, -2.0, 3.0, 7.0, 0.5], 60)
    b = W.uniform_vector(d.size, 4)
    st, x = _solve(gk, W.diagonal(d), b, "gmres", max_iters=100, reduction_factor=1e-12, krylov_dim=50)
    assert st.stop_reason == gk.STOP_CONVERGED and st.iters <= 5
    np.testing.assert_allclose(x, b / d, rtol=1e-10)


@pytest.mark.parametrize("kind", ["fcg", "cgs", "gmres"])
def test_criteria_edge_cases(gk, orc, kind):
    A = W.convdiff2d(16, 0.3) if kind != "fcg" else W.poisson2d(16)
    xs = W.uniform_vector(256, 5)
    b = orc.spmv(A, xs)
    # exact initial guess: nothing to do
    st, x = _solve(gk, A, b, kind, x0=xs, reduction_factor=1e-10)
    assert st.stop_reason == gk.STOP_CONVERGED and st.iters == 0
    # iteration limit
    st, _ = _solve(gk, A, b, kind, max_iters=3, reduction_factor=1e-14)
    assert st.stop_reason == gk.STOP_MAX_ITERS and st.iters == 3
    # NaN right-hand side
    st, _ = _solve(gk, A, np.full(256, np.nan), kind, max_iters=50)
    assert st.stop_reason == gk.STOP_NAN


def test_gmres_krylov_dim_limit(gk):
    A = W.poisson2d(8)
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]))
    with pytest.raises(gk.GkError):
        gk.Solver(M, None, "gmres", krylov_dim=129)


@pytest.mark.parametrize("every", [1, 7])
@pytest.mark.parametrize("prec", [None, 1, 4])
def test_gmres_host_driven_steps_identical(gk, prec, every):
    """The host-driven cycle (check_every > 0: the same kernels launched one
    by one, the end flag read after every `every` steps) gives the graph's
    result bit for bit, including restarts and the iteration count."""
    A = W.convdiff2d(40, 0.5)
    n = A[0].size - 1
    b = W.uniform_vector(n, 8)
    st0, x0 = _solve(gk, A, b, "gmres", "ell", prec, max_iters=3000, reduction_factor=1e-10, krylov_dim=12)
    st1, x1 = _solve(gk, A, b, "gmres", "ell", prec, max_iters=3000, reduction_factor=1e-10, krylov_dim=12,
                     check_every=every)
    assert st0.stop_reason == st1.stop_reason == gk.STOP_CONVERGED
    assert st0.iters == st1.iters and st0.spmvs == st1.spmvs and st0.iters > 12
    np.testing.assert_array_equal(x0, x1)
