"""GPU parity of the Jacobi preconditioners (Section 3.2) against the oracle.

Generation and apply perform the oracle's operations in the oracle's order
(the reciprocal of the diagonal; Gauss-Jordan with the same pivot choice and
the same fma updates; the block matvec summed in increasing column order), so
the comparison is bit for bit.
"""
import numpy as np
import pytest

import workloads as W
from helpers import to_dev, to_np

pytestmark = pytest.mark.gpu


def _pivoting_matrix(n=200, seed=3):
    """Random dense-ish blocks with small diagonals (row exchanges happen) plus
    couplings across block boundaries."""
    rng = np.random.default_rng(seed)
    D = np.zeros((n, n))
    for b0 in range(0, n, 32):
        e = min(n, b0 + 32)
        blk = rng.standard_normal((e - b0, e - b0))
        blk[np.arange(e - b0), np.arange(e - b0)] *= 1e-2
        D[b0:e, b0:e] = blk
    D += np.diag(rng.standard_normal(n - 1), 1) + np.diag(rng.standard_normal(n - 1), -1)
    D[np.arange(n), np.arange(n)] += 0.0
    rows, cols = np.nonzero(D)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return rowptr.astype(np.int32), cols.astype(np.int32), D[rows, cols]


def _nan_block_matrix():
    """A NaN on a diagonal entry and a NaN below a pivot: the pivot choice
    takes no NaN (the strict comparison of the elimination), so the NaN
    spreads through its block instead of stopping the generation."""
    D = np.diag([2.0, 3.0, 4.0, 5.0, 1.0, 2.0, 3.0, 4.0, 6.0, 7.0])
    D[1, 1] = np.nan
    D[6, 5] = np.nan
    D[0, 2] = 1.0
    rows, cols = np.nonzero(D)
    rowptr = np.zeros(11, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=10), out=rowptr[1:])
    return rowptr.astype(np.int32), cols.astype(np.int32), D[rows, cols]


CASES = {
    "nan_blocks": _nan_block_matrix(),
    "stencil27_12": W.stencil27(12),
    "convdiff_30": W.convdiff2d(30, wind=1.5),
    "pivoting_200": _pivoting_matrix(),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("bs", [1, 2, 4, 7, 8, 13, 16, 32])
def test_jacobi_generate_and_apply_bit_exact(gk, orc, name, bs):
    A = CASES[name]
    n = A[0].size - 1
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt="csr")
    try:
        P = gk.Precond(M, bs)
    except gk.GkError as e:
        with pytest.raises(ZeroDivisionError):
            orc.precond(A, "jacobi" if bs == 1 else "block_jacobi", bs)
        assert e.code == 7
        return
    ref = orc.precond(A, "jacobi" if bs == 1 else "block_jacobi", bs)
    got = P.blocks()
    want = ref.dinv if bs == 1 else ref.blocks
    assert got.shape == want.shape
    assert np.array_equal(got, want, equal_nan=True), f"max diff {np.abs(got - want).max()}"
    if name == "nan_blocks":
        return
    r = W.uniform_vector(n, 9)
    z = to_dev(np.zeros(n))
    gk.precond_apply(P, to_dev(r), z)
    assert np.array_equal(to_np(z), orc.precond_apply(ref, r))


def test_singular_reported(gk):
    A = W.diagonal([1.0, 0.0, 2.0, 3.0])
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]))
    for bs in (1, 2, 4):
        with pytest.raises(gk.GkError) as ei:
            gk.Precond(M, bs)
        assert ei.value.code == 7
    # the 2x2 anti-diagonal block is invertible only with pivoting
    A2 = (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([1.0, 1.0]))
    M2 = gk.Matrix(to_dev(A2[0]), to_dev(A2[1]), to_dev(A2[2]))
    with pytest.raises(gk.GkError):
        gk.Precond(M2, 1)
    assert np.array_equal(gk.Precond(M2, 2).blocks(), [0.0, 1.0, 1.0, 0.0])


def test_bad_block_size(gk):
    A = W.poisson2d(4)
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]))
    for bs in (0, 33, -1):
        with pytest.raises(gk.GkError) as ei:
            gk.Precond(M, bs)
        assert ei.value.code == 1


@pytest.fixture(scope="module")
def bench_mats():
    return {"stencil27_128": W.stencil27(128), "powerlaw_1M": W.powerlaw(1_000_000, seed=3)}


@pytest.mark.parametrize("which,bs", [("stencil27_128", 1), ("stencil27_128", 8), ("stencil27_128", 16),
                                      ("powerlaw_1M", 1), ("powerlaw_1M", 4), ("powerlaw_1M", 32)])
def test_generate_full_size_bit_exact(gk, orc, bench_mats, which, bs):
    """The benchmark's generations at full size -- scalar and block Jacobi of
    the 27-point matrix on 128^3 (bs 8: 262,144 blocks) and of the power-law
    matrix with 10^6 rows (bs 4), plus one size each of the shared-memory
    form (bs 16, 32) -- every inverse block bit for bit against the oracle,
    including the blocks of the longest rows (10^4 entries), whose in-block
    entries the kernel finds by binary search."""
    A = bench_mats[which]
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt="csr")
    got = gk.Precond(M, bs).blocks()
    ref = orc.precond(A, "jacobi" if bs == 1 else "block_jacobi", bs)
    want = ref.dinv if bs == 1 else ref.blocks
    assert got.shape == want.shape
    assert np.array_equal(got, want), f"{int((got != want).sum())} entries differ"
    if which == "powerlaw_1M" and bs > 1:
        # the blocks holding the longest rows were among those compared
        lens = np.diff(A[0])
        assert lens.max() > 4096
