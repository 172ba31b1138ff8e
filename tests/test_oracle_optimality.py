"""Pins of the oracle's CG and GMRES to the property that defines each
method, checked by brute force on small dense problems (no recurrence of the
methods is retyped here):

* CG after j steps (x0 = 0) is the point of the Krylov space
  K_j(M^-1 A, M^-1 b) with the least A-norm error (the Galerkin condition
  Q^T (b - A x_j) = 0 on an orthonormal basis Q of that space);
* GMRES after j < m steps with right preconditioning (x0 = 0) is
  x_j = M^-1 u_j, where u_j in K_j(A M^-1, b) minimises ||b - A M^-1 u||.

The Krylov spaces come from numpy QR of the power basis; the optimum from a
dense solve or least squares."""
import numpy as np
import pytest

import workloads as W


def _csr(D):
    rows, cols = np.nonzero(D)
    rowptr = np.zeros(D.shape[0] + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows, minlength=D.shape[0]), out=rowptr[1:])
    return rowptr, cols.astype(np.int32), D[rows, cols].astype(np.float64)


def _krylov_basis(B, v, j):
    K = np.empty((v.size, j))
    K[:, 0] = v / np.linalg.norm(v)
    for i in range(1, j):
        w = B @ K[:, i - 1]
        K[:, i] = w / np.linalg.norm(w)
    Q, _ = np.linalg.qr(K)
    return Q


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(1.0, 12.0, n)
    D = (Q * lam) @ Q.T
    D = (D + D.T) / 2
    s = np.exp(rng.uniform(-1, 1, n))       # uneven diagonal, so Jacobi matters
    return D * np.outer(s, s)


@pytest.mark.parametrize("prec", ["none", "jacobi"])
@pytest.mark.parametrize("j", [1, 2, 3, 5, 7])
def test_cg_is_the_a_norm_optimum_of_its_krylov_space(orc, prec, j):
    n = 40
    D = _spd(n, 3)
    A = _csr(D)
    b = W.uniform_vector(n, 4)
    Minv = np.diag(1.0 / np.diag(D)) if prec == "jacobi" else np.eye(n)
    r = orc.cg(A, b, P=orc.precond(A, prec), max_iters=j, tol=1e-300)
    assert r.iters == j
    Q = _krylov_basis(Minv @ D, Minv @ b, j)
    y = np.linalg.solve(Q.T @ D @ Q, Q.T @ b)
    x_opt = Q @ y
    xs = np.linalg.solve(D, b)
    err = lambda x: np.sqrt((x - xs) @ D @ (x - xs))
    assert np.linalg.norm(r.x - x_opt) <= 1e-9 * np.linalg.norm(x_opt)
    assert err(r.x) <= err(x_opt) * (1 + 1e-9)


@pytest.mark.parametrize("prec", ["none", "jacobi"])
@pytest.mark.parametrize("j", [1, 2, 4, 6, 9])
def test_gmres_is_the_minimal_residual_of_its_krylov_space(orc, prec, j):
    A = W.convdiff2d(6, wind=1.5)                 # nonsymmetric, n = 36
    D = W.csr_to_dense(A)
    n = D.shape[0]
    rng = np.random.default_rng(5)
    D = D * np.exp(rng.uniform(-0.5, 0.5, n))[:, None]   # uneven row scaling
    A = _csr(D)
    b = W.uniform_vector(n, 6)
    Minv = np.diag(1.0 / np.diag(D)) if prec == "jacobi" else np.eye(n)
    r = orc.gmres(A, b, P=orc.precond(A, prec), max_iters=j, tol=1e-300, krylov_dim=30)
    assert r.iters == j
    AM = D @ Minv
    Q = _krylov_basis(AM, b, j)
    y, *_ = np.linalg.lstsq(AM @ Q, b, rcond=None)
    x_opt = Minv @ (Q @ y)
    res_opt = np.linalg.norm(b - D @ x_opt)
    res = np.linalg.norm(b - D @ r.x)
    assert abs(res - res_opt) <= 1e-9 * np.linalg.norm(b)
    assert np.linalg.norm(r.x - x_opt) <= 1e-8 * np.linalg.norm(x_opt)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_cgs_residual_is_the_squared_cg_polynomial(orc, k):
    """On SPD A with r^ = r_0 = b, BiCG's residual polynomial phi_k is CG's,
    and CGS's residual after k steps is phi_k(A)^2 b (Sonneveld 1989).
    phi_k(t) = 1 - t p(t), with x_k = p(A) b CG's A-norm optimum over
    K_k(A, b) (computed here by brute force, as above)."""
    n = 30
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    D = (Q * np.linspace(1.0, 4.0, n)) @ Q.T
    D = (D + D.T) / 2
    A = _csr(D)
    b = W.uniform_vector(n, 9)
    Kb = _krylov_basis(D, b, k)
    x_cg = Kb @ np.linalg.solve(Kb.T @ D @ Kb, Kb.T @ b)
    P = np.empty((n, k))                      # the power basis b, A b, ..., A^(k-1) b
    P[:, 0] = b
    for i in range(1, k):
        P[:, i] = D @ P[:, i - 1]
    c, *_ = np.linalg.lstsq(P, x_cg, rcond=None)

    def phi(v):
        pv = np.zeros(n)
        w = v.copy()
        for i in range(k):
            pv += c[i] * w
            w = D @ w
        return v - D @ pv

    r = orc.cgs(A, b, max_iters=k, tol=1e-300)
    assert r.iters == k
    res = b - D @ r.x
    want = phi(phi(b))
    assert np.linalg.norm(res - want) <= 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_bicgstab_residual_from_cg_polynomials_and_local_minimisation(orc, k):
    """On SPD A with r^ = r_0 = b, BiCGSTAB's residual after k steps is
    psi_k(A) phi_k(A) b (van der Vorst 1992): phi_k is CG's residual
    polynomial (brute force, as above) and psi_k(t) = prod_i (1 - omega_i t),
    each omega_i minimising ||s_i - omega A s_i|| for
    s_i = psi_{i-1}(A) phi_i(A) b.  Rebuilt here from those definitions."""
    n = 30
    rng = np.random.default_rng(10)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    D = (Q * np.linspace(1.0, 4.0, n)) @ Q.T
    D = (D + D.T) / 2
    A = _csr(D)
    b = W.uniform_vector(n, 11)

    def phi_b(i):
        Kb = _krylov_basis(D, b, i)
        x_cg = Kb @ np.linalg.solve(Kb.T @ D @ Kb, Kb.T @ b)
        return b - D @ x_cg                   # phi_i(A) b = the CG residual

    omegas = []
    r_want = None
    for i in range(1, k + 1):
        s = phi_b(i)
        for w in omegas:                      # psi_{i-1}(A) phi_i(A) b
            s = s - w * (D @ s)
        t = D @ s
        w = (t @ s) / (t @ t)
        omegas.append(w)
        r_want = s - w * t
    r = orc.bicgstab(A, b, max_iters=k, tol=1e-300)
    assert r.iters == k
    res = b - D @ r.x
    assert np.linalg.norm(res - r_want) <= 1e-8 * np.linalg.norm(b)
