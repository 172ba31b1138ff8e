"""CPU pins of the oracle's CGS, flexible CG and restarted GMRES (the rest of
the Krylov family of Section 3.1): dense LAPACK solves, closed forms,
finite termination and the minimal-residual property."""
import numpy as np
import pytest

import workloads as W


def _dense_solution(A, b):
    return np.linalg.solve(W.csr_to_dense(A), b)


@pytest.mark.parametrize("prec", ["none", "jacobi", "block_jacobi"])
def test_cgs_nonsymmetric_matches_lapack(orc, prec):
    A = W.convdiff2d(16, 0.5)
    b = W.uniform_vector(256, 2)
    res = orc.cgs(A, b, P=orc.precond(A, prec, 4), tol=1e-11)
    assert res.stop_reason == 1
    xd = _dense_solution(A, b)
    assert np.linalg.norm(res.x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert res.rel_res_true <= 1e-10


def test_cgs_scaled_identity_one_step(orc):
    """A = c I: u = p = r, v^ = c r, alpha = 1/c, q = 0, x = r / c: exact in
    one iteration."""
    b = W.uniform_vector(50, 3)
    res = orc.cgs(W.scaled_identity(50, 4.0), b, tol=1e-14)
    assert res.iters == 1 and res.stop_reason == 1
    np.testing.assert_array_equal(res.x, b / 4.0)


@pytest.mark.parametrize("prec", ["none", "jacobi", "block_jacobi"])
def test_fcg_equals_cg_for_a_fixed_preconditioner(orc, prec):
    """With a fixed SPD preconditioner the flexible beta equals CG's in exact
    arithmetic: the same iteration count (within 1) and the same iterates."""
    A = W.poisson2d(32)
    b = W.uniform_vector(1024, 4)
    P = orc.precond(A, prec, 8)
    r1 = orc.cg(A, b, P=P, tol=1e-10)
    r2 = orc.fcg(A, b, P=P, tol=1e-10)
    assert r2.stop_reason == 1 and abs(r1.iters - r2.iters) <= 1
    assert np.linalg.norm(r1.x - r2.x) <= 1e-9 * np.linalg.norm(r1.x)


def test_fcg_finite_termination(orc):
    d = np.repeat([1.0, 2.0, 5.0, 11.0], 40)
    res = orc.fcg(W.diagonal(d), W.uniform_vector(d.size, 5), tol=1e-12)
    assert res.stop_reason == 1 and res.iters <= 4


def test_gmres_finite_termination_and_monotone_residual(orc):
    """Unrestarted GMRES on a diagonal matrix with 5 distinct values ends in
    at most 5 steps, and its residual never grows (minimal residual)."""
    d = np.repeat([1.0, -2.0, 3.0, 7.0, 0.5], 30)
    b = W.uniform_vector(d.size, 6)
    res = orc.gmres(W.diagonal(d), b, tol=1e-12, krylov_dim=50, history=True)
    assert res.stop_reason == 1 and res.iters <= 5
    np.testing.assert_allclose(res.x, b / d, rtol=1e-10)
    A = W.convdiff2d(12, 0.8)
    r = orc.gmres(A, W.uniform_vector(144, 7), tol=1e-12, krylov_dim=200, max_iters=144, history=True)
    h = r.history
    assert np.all(np.diff(h) <= 1e-12 * h[:-1] + 1e-300)


@pytest.mark.parametrize("prec", ["none", "jacobi", "block_jacobi"])
def test_gmres_restarted_matches_lapack(orc, prec):
    A = W.convdiff2d(16, 0.5)
    b = W.uniform_vector(256, 8)
    res = orc.gmres(A, b, P=orc.precond(A, prec, 4), tol=1e-11, krylov_dim=20, max_iters=2000)
    assert res.stop_reason == 1
    xd = _dense_solution(A, b)
    assert np.linalg.norm(res.x - xd) <= 1e-8 * np.linalg.norm(xd)
    # the criterion was met on the true residual of the final cycle
    assert res.rel_res_true <= 1e-11 * 1.0000001


def test_gmres_rotated_residual_is_the_true_residual(orc):
    """After one cycle (no restart), the rotated residual |g_{j+1}| equals
    ||b - A x|| of the updated iterate up to rounding."""
    A = W.convdiff2d(10, 0.3)
    b = W.uniform_vector(100, 9)
    res = orc.gmres(A, b, tol=1e-30, krylov_dim=15, max_iters=15, history=True)
    assert res.iters == 15 and res.stop_reason == 2
    est = res.history[15]
    assert res.rel_res_true == pytest.approx(est, rel=1e-6)
