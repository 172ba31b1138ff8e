"""CPU pins of the mixed-precision oracle: the adaptive block precision rule
(closed-form condition numbers) and FP64 iterative refinement around an FP32
CG inner solver (Sections 2.2.3, 3.1, 3.2)."""
import numpy as np
import pytest

import workloads as W


def _tridiag_inv_colsum_max(m):
    i = np.arange(1, m + 1)
    T = np.minimum.outer(i, i) * (m + 1 - np.maximum.outer(i, i)) / (m + 1)
    return T.sum(axis=0).max()


@pytest.mark.parametrize("m,expect", [(2, 0), (4, 0), (8, 1), (16, 1)])
def test_precision_rule_on_tridiagonal_blocks(orc, m, expect):
    """kappa_1(tridiag(-1, 2, -1)_m) = ||D||_1 * max column sum of the
    closed-form inverse; FP16 storage iff kappa_1 * 2^-11 <= 1e-2
    (kappa_1 <= 20.48): m = 2 gives 3, m = 4 gives 12, m = 8 gives 40."""
    A = W.poisson1d(3 * m)
    P = orc.precond(A, "block_jacobi", m)
    prec, kappa = orc.block_jacobi_precision(A, m, P.blocks)
    # ||D||_1 = 4 (a column holding -1, 2, -1) once m >= 3; for m = 2 both
    # columns hold only 2 and -1
    norm_d = 4.0 if m >= 3 else 3.0
    k_exact = norm_d * _tridiag_inv_colsum_max(m)
    assert kappa[1] == pytest.approx(k_exact, rel=1e-12)
    assert prec[1] == expect


def test_precision_rule_uses_one_norm(orc):
    """D = [[1, a], [0, 1]] has ||D||_1 = ||D^{-1}||_1 = 1 + a: kappa_1 = 2.25
    for a = 0.5 (FP16) and 169 for a = 12 (FP32); diagonal blocks have
    kappa_1 = max|d| / min|d|."""
    for a, expect in ((0.5, 0), (12.0, 1)):
        rowptr = np.array([0, 2, 3], np.int32)
        col = np.array([0, 1, 1], np.int32)
        val = np.array([1.0, a, 1.0])
        A = (rowptr, col, val)
        P = orc.precond(A, "block_jacobi", 2)
        prec, kappa = orc.block_jacobi_precision(A, 2, P.blocks)
        assert kappa[0] == pytest.approx((1 + a) ** 2)
        assert prec[0] == expect
    # diagonal blocks: kappa = max|d| / min|d| per block
    A = W.diagonal([1.0, 2.0, 4.0, 1.0, 100.0, 1.0])
    P = orc.precond(A, "block_jacobi", 3)
    prec, kappa = orc.block_jacobi_precision(A, 3, P.blocks)
    assert kappa.tolist() == [4.0, 100.0] and prec.tolist() == [0, 1]


@pytest.mark.parametrize("prec", ["none", "jacobi", "block_jacobi"])
@pytest.mark.parametrize("name", ["poisson64", "stencil27_16"])
def test_ir_reaches_fp64_accuracy(orc, prec, name):
    A = W.poisson2d(64) if name == "poisson64" else W.stencil27(16)
    n = A[0].size - 1
    xs = W.uniform_vector(n, 1)
    b = orc.spmv(A, xs)
    P = orc.precond(A, prec, 4)
    r, outer = orc.ir_cg(A, b, P=P, tol=1e-10)
    c = orc.cg(A, b, P=P, tol=1e-10)
    assert r.stop_reason == orc.STOP_CONVERGED
    assert r.rel_res_true <= 1e-10  # the FP64 residual itself decides
    assert 1 <= outer <= 4
    # an FP32 inner solve restarts the Krylov space at every outer step, but
    # must not need more than about twice the FP64 iterations
    assert c.iters <= r.iters <= 2 * c.iters + 10
    kappa = 1711.7 if name == "poisson64" else 250.0
    assert np.linalg.norm(r.x - xs) / np.linalg.norm(xs) <= kappa * 2e-10


def test_ir_more_outer_steps_when_inner_is_loose(orc):
    A = W.poisson2d(32)
    b = W.uniform_vector(1024, 2)
    tight, o1 = orc.ir_cg(A, b, inner_reduction=1e-6)
    loose, o2 = orc.ir_cg(A, b, inner_reduction=1e-2)
    assert tight.stop_reason == loose.stop_reason == orc.STOP_CONVERGED
    assert o2 > o1 >= 2
    # an inner solve that cannot reach its target stops at inner_max and the
    # outer loop still converges
    capped, o3 = orc.ir_cg(A, b, inner_reduction=1e-12, inner_max=40)
    assert capped.stop_reason == orc.STOP_CONVERGED and o3 > o1


def test_varcoef3d_unit_coefficients_is_poisson7():
    """Unit cell coefficients give the 7-point Poisson stencil (6 on the
    diagonal, -1 per neighbour, Dirichlet)."""
    A = W.varcoef3d_from(np.ones((3, 4, 5)))
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    P = W._from_offsets((3, 4, 5), offs, [-1, -1, -1, 6, -1, -1, -1])
    for a, p in zip(A, P):
        np.testing.assert_array_equal(a, p)


def test_varcoef3d_faces_and_spd():
    """a_ij = -2 c_i c_j / (c_i + c_j) for face neighbours along each axis;
    a_ii = the six faces with boundary faces carrying c_i; symmetric positive
    definite; the 256^3 size of the mixed-precision workload has
    7 n - 6 * 256^2 nonzeros."""
    rng = np.random.default_rng(2)
    coef = np.exp(rng.standard_normal((3, 4, 5)))
    D = W.csr_to_dense(W.varcoef3d_from(coef))
    c = coef.ravel()
    hm = lambda a, b: 2 * a * b / (a + b)
    i = 1 * 20 + 2 * 5 + 3  # interior cell (z=1, y=2, x=3)
    for j in (i - 1, i + 1, i - 5, i + 5, i - 20, i + 20):
        assert D[i, j] == pytest.approx(-hm(c[i], c[j]), rel=1e-15)
    assert D[i, i] == pytest.approx(-(D[i].sum() - D[i, i]), rel=1e-14)  # interior: diag = sum of faces
    # corner cell 0: three boundary faces (c_0) + three interior faces
    assert D[0, 0] == pytest.approx(3 * c[0] - (D[0, 1] + D[0, 5] + D[0, 20]), rel=1e-14)
    np.testing.assert_array_equal(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0
    assert 7 * 256 ** 3 - 6 * 256 ** 2 == 117_047_296
