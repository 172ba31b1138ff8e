"""CPU checks of the seeded input generators against the input recipe: sizes,
stencil values, symmetry, diagonal dominance and the CSR invariants every
matrix handed to the library must satisfy (sorted, unique, in-range columns)."""
import numpy as np
import pytest

import workloads as W


def _csr_ok(A, n_cols=None):
    rowptr, col, val = A
    n = rowptr.size - 1
    n_cols = n if n_cols is None else n_cols
    assert rowptr.dtype == np.int32 and col.dtype == np.int32 and val.dtype == np.float64
    assert rowptr[0] == 0 and rowptr[-1] == col.size and np.all(np.diff(rowptr) >= 0)
    assert col.size == 0 or (col.min() >= 0 and col.max() < n_cols)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    same_row = rows[1:] == rows[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row]), "columns not sorted and unique"
    return rows


def _dense(A):
    return W.csr_to_dense(A)


@pytest.mark.parametrize("N", [3, 5, 8])
def test_stencil27_sizes_and_values(N):
    A = W.stencil27(N)
    rows = _csr_ok(A)
    n = N ** 3
    assert A[0].size - 1 == n and A[1].size == (3 * N - 2) ** 3
    diag = A[1] == rows
    assert np.all(A[2][diag] == 26.0) and np.all(A[2][~diag] == -1.0) and diag.sum() == n
    D = _dense(A)
    assert np.array_equal(D, D.T)
    # the interior point of a 3^3 grid has all 26 neighbours
    if N == 3:
        assert np.count_nonzero(D[13]) == 27


def test_stencil27_benchmark_size_formula():
    # n and nnz of the 128^3 benchmark matrix, from the same count
    assert 128 ** 3 == 2_097_152 and (3 * 128 - 2) ** 3 == 55_742_968


def test_poisson2d_64():
    A = W.poisson2d(64)
    rows = _csr_ok(A)
    assert A[0].size - 1 == 4096 and A[1].size == 20_224
    assert np.all(A[2][A[1] == rows] == 4.0)
    D = _dense(A)
    assert np.array_equal(D, D.T)


def test_convdiff2d_upwind_rows():
    w = 0.5
    A = W.convdiff2d(6, w)
    _csr_ok(A)
    D = _dense(A)
    i = 2 * 6 + 2                       # an interior point
    assert D[i, i] == 4 + w and D[i, i - 1] == -1 - w and D[i, i + 1] == -1
    assert D[i, i - 6] == -1 and D[i, i + 6] == -1
    assert abs(D[i].sum()) == 0.0       # interior rows sum to zero
    assert not np.array_equal(D, D.T)


def test_powerlaw_symmetric_strictly_dominant():
    A = W.powerlaw(3000, seed=7)
    rows = _csr_ok(A)
    D = _dense(A)
    assert np.array_equal(D, D.T)
    off = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
    # a_ii = sum_j |a_ij| + 1, up to the order of the row sum's rounding
    assert np.all(np.abs(np.diag(D) - (off + 1.0)) <= 1e-14 * np.diag(D) * (np.diff(A[0]) + 1))
    lens = np.diff(A[0])
    assert lens.max() > 10 * np.median(lens)   # heavy-tailed row lengths
    # same seed, same matrix
    B = W.powerlaw(3000, seed=7)
    assert all(np.array_equal(a, b) for a, b in zip(A, B))


def test_uniform_vector_range_and_seed():
    a = W.uniform_vector(10_000, 1)
    assert a.min() >= -1.0 and a.max() < 1.0 and abs(a.mean()) < 0.05
    assert np.array_equal(a, W.uniform_vector(10_000, 1))
    assert not np.array_equal(a, W.uniform_vector(10_000, 2))
