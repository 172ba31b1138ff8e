"""The small-system form of CG: the whole solve in one launch of a 16-CTA
thread-block cluster (direction vector in distributed shared memory, cluster
barriers between the phases), chosen by default for CG without a
preconditioner or with scalar Jacobi on up to 32,768 rows.  Checked against
the oracle (Section 3.1's CG, the criteria of Section 2.5) like the graph
form -- stop reason, iteration count within max(2, 3 %), true residual,
solution -- and against the graph form itself on every edge of the row
partition (n below, at and above multiples of 16 and 256, the largest
size) and every exit of the loop."""
import math

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


@pytest.mark.parametrize("prec", [None, 1])
def test_poisson64_matches_oracle(gk, orc, prec):
    """Poisson-2D 64 x 64 (the small configuration), b = A x*."""
    A = W.poisson2d(64)
    xs = W.uniform_vector(4096, 1)
    b = orc.spmv(A, xs)
    st, x = _solve(gk, A, b, prec=prec, max_iters=2000, reduction_factor=1e-10)
    assert st.form == gk.FORM_CLUSTER
    ref = orc.cg(A, b, P=orc.precond(A, "jacobi" if prec else "none", 1), tol=1e-10, max_iters=2000)
    assert st.stop_reason == gk.STOP_CONVERGED == ref.stop_reason
    assert _close(st.iters, ref.iters), (st.iters, ref.iters)
    assert st.spmvs == st.iters + 2
    assert st.rel_res <= 1e-10 and st.rel_res_true <= 1.5e-10
    lmin, lmax = 4 - 4 * math.cos(math.pi / 65), 4 + 4 * math.cos(math.pi / 65)
    kappa = lmax / lmin
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= kappa * 2e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 2e-10


@pytest.mark.parametrize("side", [1, 3, 4, 17, 31, 64, 100, 128, 181])
@pytest.mark.parametrize("prec", [None, 1])
def test_against_graph_form_over_sizes(gk, orc, side, prec):
    """n = side^2 from 1 to 32,761 (rows per CTA 1 .. 2,048, rows per thread
    1 .. 8, CTAs left without rows): same stop reason, iterations within
    max(2, 3 %) of the graph form's, both within the tolerance, and the
    cluster form's x checked with the oracle's SpMV."""
    A = W.varcoef2d(np.exp(0.5 * np.random.default_rng(side).standard_normal((side, side))))
    n = side * side
    b = W.uniform_vector(n, 4)
    s1, x1 = _solve(gk, A, b, prec=prec, max_iters=20000, reduction_factor=1e-10)
    s0, x0 = _solve(gk, A, b, prec=prec, max_iters=20000, reduction_factor=1e-10, check_every=-1)
    assert s1.form == gk.FORM_CLUSTER and s0.form == gk.FORM_GRAPH
    assert s1.stop_reason == s0.stop_reason == gk.STOP_CONVERGED
    assert _close(s1.iters, s0.iters), (s1.iters, s0.iters)
    assert s1.spmvs == s1.iters + 2
    r = b - orc.spmv(A, x1)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(b)
    assert s1.rel_res_true <= 1.5e-10


def test_deterministic_and_jacobi_exact_on_poisson(gk):
    """Run to run bit-identical; with a_ii = 4 Jacobi-PCG reproduces plain CG
    bit for bit (exact power-of-two scaling in every step)."""
    A = W.poisson2d(64)
    b = W.uniform_vector(4096, 2)
    s0, x0 = _solve(gk, A, b)
    s1, x1 = _solve(gk, A, b)
    s2, x2 = _solve(gk, A, b, prec=1)
    assert s0.form == s2.form == gk.FORM_CLUSTER
    assert s0.iters == s1.iters == s2.iters
    assert np.array_equal(x0, x1) and np.array_equal(x0, x2)


def test_exits(gk, orc):
    """Every exit of the loop agrees with the graph form: exact initial
    guess (0 iterations), zero right-hand side, iteration limits 0 and 3,
    NaN in b, and an indefinite matrix (p.Ap <= 0: breakdown)."""
    A = W.poisson2d(20)
    n = 400
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
        assert s1.form == gk.FORM_CLUSTER
        assert (s1.stop_reason, s1.iters, s1.spmvs) == (s0.stop_reason, s0.iters, s0.spmvs), c
        if s1.stop_reason != gk.STOP_NAN:
            np.testing.assert_allclose(x1, x0g, rtol=0, atol=1e-12 * max(1.0, np.abs(x0g).max()))
    assert _solve(gk, A, b, x0=xs)[0].iters == 0
    D = W.diagonal(np.linspace(-3.0, 1.0, 300))  # mostly negative: p.Ap < 0 at once
    s1, _ = _solve(gk, D, W.uniform_vector(300, 6), max_iters=100)
    s0, _ = _solve(gk, D, W.uniform_vector(300, 6), max_iters=100, check_every=-1)
    assert s1.stop_reason == s0.stop_reason == gk.STOP_BREAKDOWN
    assert s1.iters == s0.iters


def test_form_selection(gk):
    """The cluster form is taken only where it applies: CG (or BiCGSTAB), no or scalar
    Jacobi preconditioning, n <= 32,768, no Time criterion, check_every 0."""
    A = W.poisson2d(8)
    b = W.uniform_vector(64, 7)
    assert _solve(gk, A, b)[0].form == gk.FORM_CLUSTER
    assert _solve(gk, A, b, time_limit_s=10.0)[0].form == gk.FORM_GRAPH
    assert _solve(gk, A, b, check_every=3)[0].form == gk.FORM_HOST
    assert _solve(gk, A, b, prec=4)[0].form == gk.FORM_GRAPH
    edge = W.poisson2d(128, 256)  # n = 32,768: the largest size of the form
    assert _solve(gk, edge, W.uniform_vector(32768, 8), max_iters=5)[0].form == gk.FORM_CLUSTER
    big = W.poisson2d(182)  # above the cluster form's size: the cooperative-grid form
    assert _solve(gk, big, W.uniform_vector(182 * 182, 8), max_iters=5)[0].form == gk.FORM_GRID


def test_rows_not_staged(gk, orc):
    """The 27-point stencil on 32^3 (n = 32,768): a CTA's 2,048 rows hold
    ~55,000 entries, more than fit shared memory, so the kernel reads the
    matrix from global memory -- same results as the graph form."""
    A = W.stencil27(32)
    n = 32768
    b = W.uniform_vector(n, 12)
    s1, x1 = _solve(gk, A, b, prec=1, max_iters=2000, reduction_factor=1e-10)
    s0, x0 = _solve(gk, A, b, prec=1, max_iters=2000, reduction_factor=1e-10, check_every=-1)
    assert s1.form == gk.FORM_CLUSTER
    assert s1.stop_reason == s0.stop_reason == gk.STOP_CONVERGED
    assert _close(s1.iters, s0.iters), (s1.iters, s0.iters)
    assert np.linalg.norm(b - orc.spmv(A, x1)) <= 1.5e-10 * np.linalg.norm(b)


def _solve_kind(gk, A, b, kind, x0=None, prec=None, **crit):
    n = A[0].size - 1
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt="csr")
    P = gk.Precond(M, prec) if prec else None
    S = gk.Solver(M, P, kind, **crit)
    x = to_dev(np.zeros(n) if x0 is None else x0)
    st = gk.solve(S, to_dev(b), x)
    return st, to_np(x)


@pytest.mark.parametrize("side", [48, 64, 100, 128])
@pytest.mark.parametrize("prec", [None, 1])
def test_bicgstab_cluster_against_graph_form(gk, orc, side, prec):
    """BiCGSTAB in the cluster form (n up to 16,384: rows per thread 1 .. 4)
    on the nonsymmetric upwind convection-diffusion matrix: same stop
    reason, iterations within max(3, 25 %) of the graph form's (BiCGSTAB's
    iteration count is sensitive to rounding), SpMV count 2 per full
    iteration, x checked with the oracle's SpMV; and against the oracle's
    BiCGSTAB."""
    A = W.convdiff2d(side, 0.5)
    n = side * side
    xs = W.uniform_vector(n, 14)
    b = orc.spmv(A, xs)
    s1, x1 = _solve_kind(gk, A, b, "bicgstab", prec=prec, max_iters=5000, reduction_factor=1e-10)
    s0, x0 = _solve_kind(gk, A, b, "bicgstab", prec=prec, max_iters=5000, reduction_factor=1e-10, check_every=-1)
    assert s1.form == gk.FORM_CLUSTER and s0.form == gk.FORM_GRAPH
    assert s1.stop_reason == s0.stop_reason == gk.STOP_CONVERGED
    assert abs(s1.iters - s0.iters) <= max(3, s0.iters // 4), (s1.iters, s0.iters)
    assert s1.spmvs in (2 * s1.iters + 2, 2 * s1.iters + 1)
    assert np.linalg.norm(b - orc.spmv(A, x1)) <= 1.5e-10 * np.linalg.norm(b)
    ref = orc.bicgstab(A, b, P=orc.precond(A, "jacobi" if prec else "none", 1), tol=1e-10, max_iters=5000)
    assert ref.stop_reason == gk.STOP_CONVERGED
    assert abs(s1.iters - ref.iters) <= max(3, ref.iters // 4), (s1.iters, ref.iters)


def test_bicgstab_cluster_exits(gk, orc):
    """A = c I converges at the first half step (x = b / c, one SpMV in the
    iteration); exact initial guess, zero right-hand side, iteration limits,
    NaN: as the graph form."""
    D = W.scaled_identity(3000, 2.5)
    b = W.uniform_vector(3000, 15)
    s1, x1 = _solve_kind(gk, D, b, "bicgstab", max_iters=50, reduction_factor=1e-10)
    assert s1.form == gk.FORM_CLUSTER and s1.stop_reason == gk.STOP_CONVERGED
    assert s1.iters == 1 and s1.spmvs == 3
    np.testing.assert_allclose(x1, b / 2.5, rtol=1e-14)
    A = W.convdiff2d(40, 0.5)
    n = 1600
    xs = W.uniform_vector(n, 16)
    bb = orc.spmv(A, xs)
    cases = [dict(b=bb, x0=xs), dict(b=np.zeros(n)), dict(b=bb, max_iters=0), dict(b=bb, max_iters=3),
             dict(b=np.full(n, np.nan), max_iters=50)]
    for c in cases:
        c = dict(c)
        bv, x0 = c.pop("b"), c.pop("x0", None)
        c.setdefault("reduction_factor", 1e-10)
        s1, x1 = _solve_kind(gk, A, bv, "bicgstab", x0=x0, **c)
        s0, x0g = _solve_kind(gk, A, bv, "bicgstab", x0=x0, check_every=-1, **c)
        assert s1.form == gk.FORM_CLUSTER
        assert (s1.stop_reason, s1.iters, s1.spmvs) == (s0.stop_reason, s0.iters, s0.spmvs), c
        if s1.stop_reason != gk.STOP_NAN:
            np.testing.assert_allclose(x1, x0g, rtol=0, atol=1e-11 * max(1.0, np.abs(x0g).max()))


def test_bicgstab_cluster_selection(gk):
    A = W.convdiff2d(128, 0.5)  # n = 16,384: the largest size of the form
    assert _solve_kind(gk, A, W.uniform_vector(16384, 17), "bicgstab", max_iters=3)[0].form == gk.FORM_CLUSTER
    A2 = W.convdiff2d(129, 0.5)
    assert _solve_kind(gk, A2, W.uniform_vector(129 * 129, 17), "bicgstab", max_iters=3)[0].form == gk.FORM_GRAPH
    assert _solve_kind(gk, A, W.uniform_vector(16384, 17), "bicgstab", max_iters=3,
                       prec=4)[0].form == gk.FORM_GRAPH


def test_bicgstab_cluster_rows_not_staged(gk, orc):
    """BiCGSTAB on the 27-point stencil on 25^3 (n = 15,625): a CTA's 1,024
    rows hold ~27,000 entries, more than are staged, so the kernel reads the
    matrix from global memory -- as the graph form."""
    A = W.stencil27(25)
    n = 25 ** 3
    b = W.uniform_vector(n, 18)
    s1, x1 = _solve_kind(gk, A, b, "bicgstab", prec=1, max_iters=2000, reduction_factor=1e-10)
    s0, x0 = _solve_kind(gk, A, b, "bicgstab", prec=1, max_iters=2000, reduction_factor=1e-10, check_every=-1)
    assert s1.form == gk.FORM_CLUSTER
    assert s1.stop_reason == s0.stop_reason == gk.STOP_CONVERGED
    assert abs(s1.iters - s0.iters) <= max(3, s0.iters // 4), (s1.iters, s0.iters)
    assert np.linalg.norm(b - orc.spmv(A, x1)) <= 1.5e-10 * np.linalg.norm(b)
