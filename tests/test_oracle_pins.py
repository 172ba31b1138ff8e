"""CPU pins of the oracle against brute force, closed forms and invariants.

Each test is chosen so that a plausible slip in the oracle (a transposed
operand, a dropped term, a wrong sign, a wrong index, r.r in place of r.z, a
mis-ordered criterion) fails at least one of them.  None of them calls the
CUDA library.
"""
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

U = 2.0 ** -53  # unit roundoff of binary64


def _rows_bound(A, x):
    rowptr, col, val = A
    rows = np.repeat(np.arange(rowptr.size - 1), np.diff(rowptr))
    return np.bincount(rows, weights=np.abs(val) * np.abs(x[col]), minlength=rowptr.size - 1)


# --------------------------------------------------------------------------
# SpMV (Section 4.2, simple and advanced apply)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m,n,seed", [(1, 1, 0), (37, 53, 1), (64, 64, 2), (50, 20, 3)])
def test_spmv_matches_dense_brute_force(orc, m, n, seed):
    A = W.random_csr(m, n, seed=seed, long_rows=1)
    D = W.csr_to_dense(A, n)
    x = W.uniform_vector(n, seed + 100)
    y = orc.spmv(A, x)
    ref = D @ x
    k = max(1, int(np.diff(A[0]).max()))
    bound = _rows_bound(A, x)
    assert np.all(np.abs(y - ref) <= 2 * k * U * bound + 1e-300)
    # a transposed operand would not even have the right length when m != n
    assert y.shape == (m,)


def test_spmv_advanced_apply(orc):
    A = W.random_csr(40, 30, seed=7)
    D = W.csr_to_dense(A, 30)
    x = W.uniform_vector(30, 8)
    y0 = W.uniform_vector(40, 9)
    y = orc.spmv(A, x, alpha=-2.5, beta=0.75, y=y0)
    ref = -2.5 * (D @ x) + 0.75 * y0
    bound = 2.5 * _rows_bound(A, x) + 0.75 * np.abs(y0)
    assert np.all(np.abs(y - ref) <= 200 * U * bound)
    # simple apply == advanced(alpha=1, beta=0), and beta=0 never reads y
    ynan = np.full(40, np.nan)
    assert np.array_equal(orc.spmv(A, x, 1.0, 0.0, ynan), orc.spmv(A, x))
    # empty rows give beta*y
    empty = np.diff(A[0]) == 0
    assert empty.any()
    assert np.array_equal(y[empty], 0.75 * y0[empty])


def test_spmv_dot2_is_accurate(orc):
    rng = np.random.default_rng(11)
    # ill-conditioned rows: large cancelling terms plus small ones
    n = 30
    rowptr = np.arange(0, 6 * n + 1, 6)
    col = np.tile(np.arange(6), n)
    big = rng.uniform(1e8, 1e9, size=n)
    val = np.stack([big, -big, rng.standard_normal(n), rng.standard_normal(n) * 1e-8,
                    big * 0.5, -big * 0.5], axis=1).ravel()
    A = (rowptr.astype(np.int32), col.astype(np.int32), val)
    x = np.array([1.0 + 2 ** -30, 1.0, 0.3, 1.7, 1.0 - 2 ** -40, 1.0])
    xx = np.zeros(6)
    xx[:] = x
    y, b = orc.spmv_accurate(A, xx)
    for i in range(n):
        exact = sum(Fraction(float(v)) * Fraction(float(xx[c]))
                    for v, c in zip(val[6 * i:6 * i + 6], col[6 * i:6 * i + 6]))
        assert abs(Fraction(float(y[i])) - exact) <= Fraction(2 * U) * abs(exact) + Fraction(1e-290)
        absum = sum(abs(Fraction(float(v)) * Fraction(float(xx[c])))
                    for v, c in zip(val[6 * i:6 * i + 6], col[6 * i:6 * i + 6]))
        assert abs(Fraction(float(b[i])) - absum) <= Fraction(8 * U) * absum


def test_spmv_poisson2d_eigenvectors(orc):
    """Closed form: v_jk(x, y) = sin(j pi x/65) sin(k pi y/65) on the 64x64 grid
    (x, y = 1..64) has eigenvalue 4 - 2cos(j pi/65) - 2cos(k pi/65)."""
    A = W.poisson2d(64)
    g = np.arange(1, 65)
    for j, k in [(1, 1), (3, 7), (64, 64), (20, 45)]:
        # reduce j*g modulo the period 130 in integers first, so the sine
        # arguments stay below 2 pi and carry no large rounding error
        sx = np.sin(np.pi * ((j * g) % 130) / 65)
        sy = np.sin(np.pi * ((k * g) % 130) / 65)
        v = np.outer(sy, sx).ravel()
        lam = 4 - 2 * np.cos(j * np.pi / 65) - 2 * np.cos(k * np.pi / 65)
        y = orc.spmv(A, v)
        assert np.all(np.abs(y - lam * v) <= 1e-13 * _rows_bound(A, v) + 1e-15)


# --------------------------------------------------------------------------
# Jacobi and block-Jacobi (Sections 3.2, 7.5)
# --------------------------------------------------------------------------

def test_block_jacobi_tridiagonal_closed_form(orc):
    """(T_m^{-1})_{ij} = min(i,j) (m+1-max(i,j)) / (m+1) for T_m = tridiag(-1,2,-1),
    1-based.  n = 3*m + 3 also checks the shorter last block (m' = 3)."""
    for m in (4, 8, 13, 32):
        n = 3 * m + 3
        A = W.poisson1d(n)
        blocks = orc.block_jacobi(A, m)
        off = 0
        for size in [m, m, m, 3]:
            i = np.arange(1, size + 1)
            T = np.minimum.outer(i, i) * (size + 1 - np.maximum.outer(i, i)) / (size + 1)
            got = blocks[off:off + size * size].reshape(size, size)
            assert np.allclose(got, T, rtol=0, atol=64 * size * size * U * np.abs(T).max())
            off += size * size
        assert off == blocks.size


def test_block_jacobi_matches_lapack_inverse_with_pivoting(orc):
    """Random blocks with tiny diagonals force row exchanges; compare with
    numpy's LAPACK inverse, and check D D^{-1} = I to a condition-scaled
    bound."""
    rng = np.random.default_rng(5)
    n, bs = 64, 16
    D = np.zeros((n, n))
    for b0 in range(0, n, bs):
        blk = rng.standard_normal((bs, bs))
        blk[np.arange(bs), np.arange(bs)] *= 1e-3
        D[b0:b0 + bs, b0:b0 + bs] = blk
    # couplings that cross block boundaries must be ignored by the extraction
    D += np.diag(np.full(n - 1, 0.25), 1)
    rows, cols = np.nonzero(D)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    A = (rowptr.astype(np.int32), cols.astype(np.int32), D[rows, cols])
    blocks = orc.block_jacobi(A, bs)
    for k, b0 in enumerate(range(0, n, bs)):
        blk = D[b0:b0 + bs, b0:b0 + bs]
        inv = blocks[k * bs * bs:(k + 1) * bs * bs].reshape(bs, bs)
        ref = np.linalg.inv(blk)
        kappa = np.linalg.cond(blk, 1)
        assert np.abs(inv - ref).max() <= 100 * bs * kappa * U * np.abs(ref).max()
        assert np.abs(blk @ inv - np.eye(bs)).max() <= 100 * bs * kappa * U


def test_block_jacobi_bs1_equals_scalar_jacobi(orc):
    A = W.stencil27(6)
    d = orc.jacobi_scalar(A)
    blocks = orc.block_jacobi(A, 1)
    assert np.array_equal(d, blocks)
    r = W.uniform_vector(d.size, 3)
    z1 = orc.precond_apply(orc.precond(A, "jacobi"), r)
    z2 = orc.precond_apply(orc.precond(A, "block_jacobi", 1), r)
    assert np.array_equal(z1, z2)
    assert np.array_equal(z1, r * (1.0 / 26.0))


def test_block_jacobi_apply_matches_dense(orc):
    A = W.convdiff2d(7)  # n = 49, blocks of 8 and a last block of 1
    P = orc.precond(A, "block_jacobi", 8)
    r = W.uniform_vector(49, 4)
    z = orc.precond_apply(P, r)
    D = W.csr_to_dense(A)
    ref = np.zeros(49)
    for b0 in range(0, 49, 8):
        e = min(49, b0 + 8)
        ref[b0:e] = np.linalg.solve(D[b0:e, b0:e], r[b0:e])
    assert np.allclose(z, ref, rtol=1e-13, atol=1e-14)


def test_jacobi_singular(orc):
    A = W.diagonal([1.0, 0.0, 2.0])
    with pytest.raises(ZeroDivisionError):
        orc.jacobi_scalar(A)
    with pytest.raises(ZeroDivisionError):
        orc.block_jacobi(A, 1)
    # a missing diagonal entry is singular for scalar Jacobi
    A2 = (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([1.0, 1.0]))
    with pytest.raises(ZeroDivisionError):
        orc.jacobi_scalar(A2)
    # but the 2x2 block [[0,1],[1,0]] is invertible with pivoting
    blk = orc.block_jacobi(A2, 2)
    assert np.array_equal(blk, [0.0, 1.0, 1.0, 0.0])


# --------------------------------------------------------------------------
# CG (Section 3.1, Listing 1) and criteria (Section 2.5)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 5, 10])
def test_cg_terminates_in_distinct_eigenvalue_steps(orc, d):
    """In exact arithmetic CG on a diagonal matrix with d distinct eigenvalues
    finds the solution in at most d steps; d = 1 takes exactly one."""
    n = 1000
    rng = np.random.default_rng(d)
    eig = np.linspace(1.0, 10.0, d)
    A = W.diagonal(eig[rng.integers(0, d, size=n)])
    b = W.uniform_vector(n, 17)
    r = orc.cg(A, b, tol=1e-10, max_iters=100)
    assert r.stop_reason == orc.STOP_CONVERGED
    assert r.iters <= d
    if d == 1:
        assert r.iters == 1


def _poisson_kappa():
    lmin = 4 - 4 * np.cos(np.pi / 65)
    lmax = 4 + 4 * np.cos(np.pi / 65)
    return lmax / lmin


def test_cg_manufactured_solution_and_chebyshev_bound(orc):
    A = W.poisson2d(64)
    kappa = _poisson_kappa()
    assert abs(kappa - 1711.66) < 0.01
    xs = W.uniform_vector(4096, 1)
    b = orc.spmv(A, xs)
    r = orc.cg(A, b, tol=1e-10, max_iters=2000)
    assert r.stop_reason == orc.STOP_CONVERGED
    assert r.rel_res <= 1e-10 and r.rel_res_true <= 2e-10
    assert np.linalg.norm(r.x - xs) / np.linalg.norm(xs) <= kappa * 1e-10
    # ||r_k||/||r_0|| <= 2 sqrt(kappa) ((sqrt(kappa)-1)/(sqrt(kappa)+1))^k
    sk = np.sqrt(kappa)
    kmax = int(np.ceil(np.log(2 * sk / 1e-10) / np.log((sk + 1) / (sk - 1))))
    assert kmax == 568
    assert r.iters <= kmax
    # the recorded history is monotone on average and ends below the tolerance
    rh = orc.cg(A, b, tol=1e-10, max_iters=2000, history=True).history
    assert rh.size == r.iters + 1 and rh[-1] <= 1e-10 and rh[0] == pytest.approx(1.0)


def test_cg_scalar_jacobi_bit_identical_on_poisson(orc):
    """With a_ii = 4 (a power of two), M^{-1} = I/4 scales exactly, so
    Jacobi-PCG reproduces plain CG bit for bit."""
    A = W.poisson2d(64)
    b = orc.spmv(A, W.uniform_vector(4096, 1))
    r0 = orc.cg(A, b)
    r1 = orc.cg(A, b, P=orc.precond(A, "jacobi"))
    r2 = orc.cg(A, b, P=orc.precond(A, "block_jacobi", 1))
    assert r0.iters == r1.iters == r2.iters
    assert np.array_equal(r0.x, r1.x) and np.array_equal(r1.x, r2.x)


def test_cg_jacobi_helps_on_badly_scaled_matrix(orc):
    """Diagonal scaling removes a row-scaling ill-conditioning exactly: for
    A = S T S with T = poisson2d(16) and S diagonal, Jacobi-PCG takes the same
    number of iterations as CG on T (within rounding), plain CG many more."""
    T = W.poisson2d(16)
    s = 10.0 ** np.linspace(-3, 3, 256)
    rowptr, col, val = T
    rows = np.repeat(np.arange(256), np.diff(rowptr))
    A = (rowptr, col, val * s[rows] * s[col])
    b = W.uniform_vector(256, 2)
    plain = orc.cg(A, b, tol=1e-8, max_iters=5000)
    jac = orc.cg(A, b, tol=1e-8, max_iters=5000, P=orc.precond(A, "jacobi"))
    assert jac.stop_reason == orc.STOP_CONVERGED
    assert jac.iters < plain.iters / 3


def test_cg_one_block_converges_in_one_step(orc):
    A = W.poisson2d(6)
    b = W.uniform_vector(36, 3)
    r = orc.cg(A, b, P=orc.precond(A, "block_jacobi", 36), tol=1e-12)
    assert r.iters == 1 and r.stop_reason == orc.STOP_CONVERGED


def test_cg_criteria_edge_cases(orc):
    A = W.poisson2d(8)
    xs = W.uniform_vector(64, 5)
    b = orc.spmv(A, xs)
    # max_iters = 0: no iteration, x unchanged
    x0 = W.uniform_vector(64, 6)
    r = orc.cg(A, b, x0=x0, max_iters=0)
    assert r.iters == 0 and r.stop_reason == orc.STOP_MAX_ITERS and np.array_equal(r.x, x0)
    # x0 = exact solution: r_0 = b - A x* is exactly zero with the same row sums
    r = orc.cg(A, b, x0=xs)
    assert r.iters == 0 and r.stop_reason == orc.STOP_CONVERGED and np.array_equal(r.x, xs)
    # NaN right-hand side (Section 7.2's overhead set-up) ends the solve
    r = orc.cg(A, np.full(64, np.nan), max_iters=1000)
    assert r.stop_reason == orc.STOP_NAN and r.iters == 0
    # n = 1: one iteration
    r = orc.cg(W.diagonal([3.0]), np.array([6.0]))
    assert r.iters == 1 and r.x[0] == 2.0
    # iteration limit hit before the tolerance
    r = orc.cg(A, b, max_iters=3, tol=1e-14)
    assert r.iters == 3 and r.stop_reason == orc.STOP_MAX_ITERS
    # rel_to_b=False measures against ||r_0||: with x0 = 0 both agree
    r1 = orc.cg(A, b, rel_to_b=False)
    r2 = orc.cg(A, b, rel_to_b=True)
    assert r1.iters == r2.iters
    # a nonzero x0 makes ||r_0|| < ||b|| here, so the r_0-relative test is stricter
    x0 = xs + 1e-3 * W.uniform_vector(64, 9)
    r3 = orc.cg(A, b, x0=x0, rel_to_b=False, tol=1e-6)
    r4 = orc.cg(A, b, x0=x0, rel_to_b=True, tol=1e-6)
    assert r3.iters >= r4.iters and r3.ref_norm < r4.ref_norm


def test_cg_breakdown_on_indefinite(orc):
    A = W.diagonal([1.0, -1.0])
    r = orc.cg(A, np.array([1.0, 1.0]))
    assert r.stop_reason == orc.STOP_BREAKDOWN


# --------------------------------------------------------------------------
# BiCGSTAB (Section 3.1, Listing 3)
# --------------------------------------------------------------------------

def test_bicgstab_scaled_identity_half_step(orc):
    A = W.scaled_identity(50, 3.0)
    b = W.uniform_vector(50, 1)
    r = orc.bicgstab(A, b)
    assert r.iters == 1 and r.spmvs == 3  # initial residual, v = A p^, final check
    assert r.stop_reason == orc.STOP_CONVERGED
    assert np.allclose(r.x, b / 3.0, rtol=1e-15, atol=0)


@pytest.mark.parametrize("prec", ["none", "jacobi", "block_jacobi"])
def test_bicgstab_nonsymmetric_vs_dense_solve(orc, prec):
    A = W.convdiff2d(20, wind=2.0)
    D = W.csr_to_dense(A)
    xs = W.uniform_vector(400, 2)
    b = D @ xs
    P = orc.precond(A, prec, 8)
    r = orc.bicgstab(A, b, P=P, tol=1e-10, max_iters=2000)
    assert r.stop_reason == orc.STOP_CONVERGED and r.rel_res_true <= 2e-10
    ref = np.linalg.solve(D, b)
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(r.x - ref) / np.linalg.norm(ref) <= kappa * 2e-10


def test_bicgstab_spd_agrees_with_cg(orc):
    A = W.poisson2d(64)
    b = orc.spmv(A, W.uniform_vector(4096, 1))
    c = orc.cg(A, b)
    s = orc.bicgstab(A, b)
    assert s.stop_reason == orc.STOP_CONVERGED
    assert np.linalg.norm(c.x - s.x) / np.linalg.norm(c.x) <= _poisson_kappa() * 2e-10


def test_bicgstab_nan_and_limits(orc):
    A = W.convdiff2d(5)
    r = orc.bicgstab(A, np.full(25, np.nan))
    assert r.stop_reason == orc.STOP_NAN
    r = orc.bicgstab(A, W.uniform_vector(25, 1), max_iters=0)
    assert r.iters == 0 and r.stop_reason == orc.STOP_MAX_ITERS


# --------------------------------------------------------------------------
# Hybrid split
# --------------------------------------------------------------------------

def test_hyb_width_closed_forms(orc):
    # uniform rows of length L: ELL alone is optimal, K = L
    A = W.stencil27(5)
    inner = np.diff(A[0]).max()
    assert inner == 27
    # all rows length 3 -> K = 3
    n = 100
    rowptr = np.arange(0, 3 * n + 1, 3)
    col = np.tile([0, 1, 2], n)
    assert orc.hyb_width((rowptr, col, np.ones(3 * n))) == 3
    # rows of length 2 plus one row of length 1000: a slot in every row costs
    # 12 n = 1200 bytes, one COO entry 16, so the long row goes to COO: K = 2
    lens = np.full(n, 2)
    lens[7] = 1000
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    col = np.concatenate([np.arange(l) for l in lens])
    assert orc.hyb_width((rowptr, col, np.ones(col.size))) == 2
    # half the rows have 10 entries, half have 2: K = 10 costs 12*10*n, K = 2
    # costs 12*2*n + 16*8*(n/2) = 88 n < 120 n -> K = 2
    lens = np.array([10, 2] * 50)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    col = np.concatenate([np.arange(l) for l in lens])
    assert orc.hyb_width((rowptr, col, np.ones(col.size))) == 2


def test_spmv_thread_count_changes_no_bit(orc):
    """The SpMV row loops may run on several threads: each row is still
    summed in increasing k by one thread, so y and a solve that uses the
    SpMV are bit-identical on one thread and on all of them."""
    A = W.powerlaw(20000, seed=3)
    n = A[0].size - 1
    x = W.uniform_vector(n, 5)
    try:
        orc.set_threads(1)
        y1 = orc.spmv(A, x)
        r1 = orc.cg(A, y1, P=orc.precond(A, "jacobi"), tol=1e-10)
        orc.set_threads(0)
        yn = orc.spmv(A, x)
        rn = orc.cg(A, yn, P=orc.precond(A, "jacobi"), tol=1e-10)
    finally:
        orc.set_threads(0)
    assert np.array_equal(y1, yn)
    assert r1.iters == rn.iters and np.array_equal(r1.x, rn.x)
