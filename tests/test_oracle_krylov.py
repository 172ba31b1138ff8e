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


def _nonsymmetric_block_preconditioner(orc, A, bs, seed):
    """A fixed but nonsymmetric preconditioner: the block-Jacobi inverse
    blocks of A plus a skew-symmetric part of comparable size.  x^T (B + K) x
    = x^T B x > 0, so it stays positive real, but M^{-1} != M^{-T}."""
    P = orc.precond(A, "block_jacobi", bs)
    blocks = P.blocks.copy()
    n = A[0].size - 1
    rng = np.random.default_rng(seed)
    off = 0
    for k in range((n + bs - 1) // bs):
        m = min(bs, n - k * bs)
        B = blocks[off:off + m * m].reshape(m, m)
        S = rng.standard_normal((m, m))
        B += 0.5 * np.abs(B).max() * (S - S.T)
        off += m * m
    return type(P)(P.kind, bs, None, blocks)


def _local_conjugacy(A, xs):
    """|d_{k+1}^T A d_k| / (||d_{k+1}||_A ||d_k||_A) for the steps d_k =
    x_{k+1} - x_k of an iterate sequence (d_k is alpha_k p_k)."""
    D = W.csr_to_dense(A)
    d = [xs[k + 1] - xs[k] for k in range(len(xs) - 1)]
    out = []
    for k in range(len(d) - 1):
        num = abs(d[k + 1] @ D @ d[k])
        den = np.sqrt((d[k + 1] @ D @ d[k + 1]) * (d[k] @ D @ d[k]))
        out.append(num / den)
    return np.array(out)


def test_fcg_flexible_beta_keeps_directions_conjugate_under_a_nonsymmetric_preconditioner(orc):
    """The flexible (Polak-Ribiere) beta = z_{k+1}.(r_{k+1} - r_k)/rho_k
    equals -(z_{k+1}.A p_k)/(p_k.A p_k) (since r_{k+1} - r_k = -alpha_k A p_k),
    so p_{k+1} is A-conjugate to p_k for ANY preconditioner, symmetric or
    not (Notay 2000).  The Fletcher-Reeves beta rho_{k+1}/rho_k of plain PCG
    coincides with it only when M^{-1} is symmetric.  With a fixed
    nonsymmetric M^{-1} on an SPD matrix, the oracle's successive steps
    x_{k+1} - x_k (= alpha_k p_k, read from runs stopped after k iterations)
    must be locally A-conjugate to rounding; the same loop with the
    Fletcher-Reeves beta (written out below on the CPU, as a planted mistake)
    is not, so this pin tells the two apart."""
    A = W.poisson2d(12)
    n = 144
    b = W.uniform_vector(n, 31)
    P = _nonsymmetric_block_preconditioner(orc, A, 4, seed=32)
    J = 7
    xs = [np.zeros(n)] + [orc.fcg(A, b, P=P, tol=1e-300, max_iters=j).x for j in range(1, J + 1)]
    assert _local_conjugacy(A, xs).max() <= 1e-9
    # the planted mistake: the same iteration with Fletcher-Reeves' beta
    D = W.csr_to_dense(A)
    x, r = np.zeros(n), b.copy()
    z = orc.precond_apply(P, r)
    p, rho = z.copy(), r @ z
    fr = [x.copy()]
    for _ in range(J):
        q = D @ p
        alpha = rho / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        z = orc.precond_apply(P, r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
        fr.append(x.copy())
    assert _local_conjugacy(A, fr).max() >= 1e-3
    # and with the symmetric block-Jacobi preconditioner the two betas agree
    Ps = orc.precond(A, "block_jacobi", 4)
    ys = [np.zeros(n)] + [orc.fcg(A, b, P=Ps, tol=1e-300, max_iters=j).x for j in range(1, J + 1)]
    cg = [np.zeros(n)] + [orc.cg(A, b, P=Ps, tol=1e-300, max_iters=j).x for j in range(1, J + 1)]
    for u, v in zip(ys, cg):
        assert np.linalg.norm(u - v) <= 1e-10 * max(np.linalg.norm(v), 1e-300)
