"""The mid-size form of CG: the whole solve in one cooperative launch (one
CTA per SM, grid-wide barriers in global memory), chosen by default for CG
without a preconditioner or with scalar Jacobi on 32,769 .. 262,144 rows of
at most 64 entries.  Checked against the graph form and the oracle's SpMV
(Section 3.1's CG, Section 2.5's criteria): stop reason, iteration count
within max(2, 3 %), true residual; every exit of the loop; selection."""
import numpy as np
import pytest

import workloads as W
from helpers import to_dev, to_np

pytestmark = pytest.mark.gpu


def _solve(gk, A, b, x0=None, prec=None, **crit):
    n = A[0].size - 1
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt="csr")
    P = gk.Precond(M, prec) if prec else None
    S = gk.Solver(M, P, "cg", **crit)
    x = to_dev(np.zeros(n) if x0 is None else x0)
    st = gk.solve(S, to_dev(b), x)
    return st, to_np(x)


def _close(a, b):
    return abs(a - b) <= max(2, int(0.03 * max(a, b)))


@pytest.mark.parametrize("shape", [(182, 181), (256, 256), (317, 331), (512, 512)])
@pytest.mark.parametrize("prec", [None, 1])
def test_against_graph_form(gk, orc, shape, prec):
    """n from 32,942 to 262,144 (rows per thread 1 .. 8, a ragged last CTA):
    variable-coefficient diffusion, same stop reason and iterations within
    max(2, 3 %) of the graph form, x checked with the oracle's SpMV."""
    ny, nx = shape
    coef = np.exp(0.5 * np.random.default_rng(ny * nx).standard_normal((ny, nx)))
    A = W.varcoef2d(coef)
    n = ny * nx
    b = W.uniform_vector(n, 4)
    s1, x1 = _solve(gk, A, b, prec=prec, max_iters=20000, reduction_factor=1e-10)
    s0, x0 = _solve(gk, A, b, prec=prec, max_iters=20000, reduction_factor=1e-10, check_every=-1)
    assert s1.form == gk.FORM_GRID and s0.form == gk.FORM_GRAPH
    assert s1.stop_reason == s0.stop_reason == gk.STOP_CONVERGED
    assert _close(s1.iters, s0.iters), (s1.iters, s0.iters)
    assert s1.spmvs == s1.iters + 2
    assert s1.device_error == 0
    r = b - orc.spmv(A, x1)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)


def test_deterministic_and_jacobi_exact(gk):
    """Run to run bit-identical; a_ii = 4 (Poisson): Jacobi reproduces plain
    CG bit for bit."""
    A = W.poisson2d(256)
    b = W.uniform_vector(65536, 2)
    s0, x0 = _solve(gk, A, b)
    s1, x1 = _solve(gk, A, b)
    s2, x2 = _solve(gk, A, b, prec=1)
    assert s0.form == s2.form == gk.FORM_GRID
    assert s0.iters == s1.iters == s2.iters
    assert np.array_equal(x0, x1) and np.array_equal(x0, x2)


def test_exits(gk, orc):
    """Exact initial guess, zero right-hand side, iteration limits 0 and 3,
    NaN in b: as the graph form (stop reason, iterations, SpMV count)."""
    A = W.poisson2d(200)
    n = 40000
    xs = W.uniform_vector(n, 5)
    b = orc.spmv(A, xs)
    cases = [dict(b=b, x0=xs), dict(b=np.zeros(n)), dict(b=b, max_iters=0), dict(b=b, max_iters=3),
             dict(b=np.full(n, np.nan), max_iters=50)]
    for c in cases:
        c = dict(c)
        bb, x0 = c.pop("b"), c.pop("x0", None)
        c.setdefault("reduction_factor", 1e-10)
        s1, x1 = _solve(gk, A, bb, x0=x0, **c)
        s0, x0g = _solve(gk, A, bb, x0=x0, check_every=-1, **c)
        assert s1.form == gk.FORM_GRID
        assert (s1.stop_reason, s1.iters, s1.spmvs) == (s0.stop_reason, s0.iters, s0.spmvs), c
        if s1.stop_reason != gk.STOP_NAN:
            np.testing.assert_allclose(x1, x0g, rtol=0, atol=1e-12 * max(1.0, np.abs(x0g).max()))
    D = W.diagonal(np.linspace(-3.0, 1.0, 40000))  # mostly negative: p.Ap < 0 at once
    s1, _ = _solve(gk, D, W.uniform_vector(40000, 6), max_iters=100)
    s0, _ = _solve(gk, D, W.uniform_vector(40000, 6), max_iters=100, check_every=-1)
    assert s1.form == gk.FORM_GRID
    assert s1.stop_reason == s0.stop_reason == gk.STOP_BREAKDOWN and s1.iters == s0.iters


def test_form_selection(gk):
    """Not above 262,144 rows, not with a row of more than 64 entries, not
    with block Jacobi or a Time criterion."""
    A = W.poisson2d(200)
    b = W.uniform_vector(40000, 7)
    assert _solve(gk, A, b, max_iters=3)[0].form == gk.FORM_GRID
    assert _solve(gk, A, b, max_iters=3, time_limit_s=5.0)[0].form == gk.FORM_GRAPH
    assert _solve(gk, A, b, max_iters=3, prec=4)[0].form == gk.FORM_GRAPH
    big = W.poisson2d(513, 512)
    assert _solve(gk, big, W.uniform_vector(513 * 512, 8), max_iters=3)[0].form == gk.FORM_GRAPH
    # one dense row of 100 entries (symmetric arrow matrix, diagonally dominant)
    n = 40000
    rows, cols, vals = [], [], []
    for i in range(n):
        rows.append(i); cols.append(i); vals.append(200.0 if i < 100 else 2.0)
    for j in range(1, 100):
        rows += [0, j]; cols += [j, 0]; vals += [-1.0, -1.0]
    import scipy.sparse as sp
    M = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    M.sort_indices()
    arrow = (M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))
    assert _solve(gk, arrow, W.uniform_vector(n, 9), max_iters=3)[0].form == gk.FORM_GRAPH


@pytest.mark.parametrize("side,staged", [(40, True), (60, False)])
def test_27_point_staged_and_not(gk, orc, side, staged):
    """27-point stencils: on 40^3 each CTA's rows fit shared memory, on 60^3
    (n = 216,000, ~38,000 entries per CTA) they do not and the kernel reads
    the matrix from global memory; both as the graph form."""
    A = W.stencil27(side)
    n = side ** 3
    b = W.uniform_vector(n, 13)
    s1, x1 = _solve(gk, A, b, prec=1, max_iters=2000, reduction_factor=1e-10)
    s0, x0 = _solve(gk, A, b, prec=1, max_iters=2000, reduction_factor=1e-10, check_every=-1)
    assert s1.form == gk.FORM_GRID
    assert s1.stop_reason == s0.stop_reason == gk.STOP_CONVERGED
    assert _close(s1.iters, s0.iters), (s1.iters, s0.iters)
    assert np.linalg.norm(b - orc.spmv(A, x1)) <= 1.5e-10 * np.linalg.norm(b)
