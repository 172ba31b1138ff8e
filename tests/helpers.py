"""Shared helpers for the GPU parity tests: tensors on cuda:0, the oracle's
per-row accuracy bound, and sub-matrices for sampled full-size checks."""
import numpy as np

U = 2.0 ** -53


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def to_np(t):
    return t.detach().cpu().numpy()


def row_bound(A, x):
    """(|A||x|)_i."""
    rowptr, col, val = A
    rows = np.repeat(np.arange(rowptr.size - 1), np.diff(rowptr))
    return np.bincount(rows, weights=np.abs(val) * np.abs(x[col]), minlength=rowptr.size - 1)


def assert_rows_within(y, y_ref, bound, tol=1e-13, what=""):
    """|y - y_ref|_i <= tol * bound_i (rows with bound 0 must match exactly)."""
    err = np.abs(y - y_ref)
    bad = ~(err <= tol * bound)
    if bad.any():
        i = int(np.flatnonzero(bad)[0])
        raise AssertionError(f"{what}: {int(bad.sum())} rows exceed {tol}*(|A||x|)_i; first row {i}: "
                             f"y={y[i]!r} ref={y_ref[i]!r} bound={bound[i]!r}")


def sub_rows(A, rows):
    """CSR of the selected rows (same columns)."""
    rowptr, col, val = A
    rows = np.asarray(rows, dtype=np.int64)
    lens = (rowptr[rows + 1] - rowptr[rows]).astype(np.int64)
    rp = np.zeros(rows.size + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.concatenate([np.arange(rowptr[r], rowptr[r + 1]) for r in rows]) if rows.size else \
        np.zeros(0, dtype=np.int64)
    return rp.astype(np.int32), col[idx], val[idx]
