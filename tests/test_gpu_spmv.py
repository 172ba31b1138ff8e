"""GPU parity of the SpMV kernels (all formats) against the CPU oracle.

Rows that a kernel sums in the oracle's order (one thread per row, fma in
increasing column position: GK_CSR rows of up to 256 entries, GK_ELL) must be bit-identical;
every row of every format must satisfy |y - y_acc|_i <= 1e-13 (|A||x|)_i with
y_acc the oracle's Dot2-accurate row sum.
"""
import numpy as np
import pytest

import workloads as W
from helpers import U, assert_rows_within, row_bound, sub_rows, to_dev, to_np

pytestmark = pytest.mark.gpu

FORMATS = ["csr", "csr_merge", "ell", "hyb", "auto"]


def _matrices():
    """name -> (CSR, n_cols)."""
    return {
        "poisson2d_64": (W.poisson2d(64), 4096),
        "stencil27_20": (W.stencil27(20), 8000),
        "ragged_3000x2500": (W.random_csr(3000, 2500, seed=4, max_len=60, empty_frac=0.2, long_rows=3,
                                          long_len=2400), 2500),
        "powerlaw_20000": (W.powerlaw(20000, seed=5), 20000),
        "single_long_row": (W.random_csr(1, 9000, seed=6, max_len=9000, empty_frac=0.0, long_rows=1), 9000),
        "all_empty": ((np.zeros(101, np.int32), np.zeros(0, np.int32), np.zeros(0)), 101),
    }


MATS = _matrices()


def _gk_matrix(gk, A, fmt, n_cols=None):
    return gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), n_cols=n_cols, fmt=fmt)


def _ordered_rows(info, A):
    """Rows whose GPU sum follows the oracle's order exactly."""
    lens = np.diff(A[0])
    f = info["format_name"]
    if f == "csr":
        return lens <= 256
    if f == "ell":
        return np.ones(lens.size, dtype=bool)
    return np.zeros(lens.size, dtype=bool)


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("fmt", FORMATS)
def test_spmv_parity(gk, orc, name, fmt):
    A, n_cols = MATS[name]
    n_rows = A[0].size - 1
    try:
        M = _gk_matrix(gk, A, fmt, n_cols)
    except gk.GkError as e:
        assert fmt == "ell" and e.code == 6, e  # ELL refuses heavy padding
        lens = np.diff(A[0])
        assert lens.max() * n_rows > 8 * A[1].size + n_rows
        return
    info = M.info()
    x = W.uniform_vector(n_cols, 7)
    y = to_dev(np.full(n_rows, np.nan))
    gk.apply(M, to_dev(x), y)
    y = to_np(y)
    y_ord = orc.spmv(A, x)
    y_acc, bnd = orc.spmv_accurate(A, x)
    assert_rows_within(y, y_acc, bnd, 1e-13, f"{name}/{fmt}")
    exact = _ordered_rows(info, A)
    assert np.array_equal(y[exact], y_ord[exact]), f"{name}/{fmt}: ordered rows not bit-identical"
    # run-to-run reproducibility
    y2 = to_dev(np.zeros(n_rows))
    gk.apply(M, to_dev(x), y2)
    assert np.array_equal(to_np(y2), y)


@pytest.mark.parametrize("fmt", ["csr", "csr_merge", "ell", "hyb"])
def test_apply_adv_and_beta_zero(gk, orc, fmt):
    A, n_cols = MATS["ragged_3000x2500"] if fmt != "ell" else MATS["stencil27_20"]
    n_rows = A[0].size - 1
    M = _gk_matrix(gk, A, fmt, n_cols)
    x = W.uniform_vector(n_cols, 1)
    y0 = W.uniform_vector(n_rows, 2)
    y = to_dev(y0)
    gk.apply_adv(-1.5, M, to_dev(x), 0.25, y)
    ref_acc, bnd = orc.spmv_accurate(A, x)
    ref = -1.5 * ref_acc + 0.25 * y0
    assert_rows_within(to_np(y), ref, 1.5 * bnd + 0.25 * np.abs(y0) + 1e-300, 2e-13, fmt)
    # beta = 0 never reads x: NaN there must not propagate
    ynan = to_dev(np.full(n_rows, np.nan))
    gk.apply_adv(2.0, M, to_dev(x), 0.0, ynan)
    assert np.all(np.isfinite(to_np(ynan)))
    # simple apply == advanced(1, 0), bit for bit
    ya, yb = to_dev(np.zeros(n_rows)), to_dev(np.zeros(n_rows))
    gk.apply(M, to_dev(x), ya)
    gk.apply_adv(1.0, M, to_dev(x), 0.0, yb)
    assert np.array_equal(to_np(ya), to_np(yb))


def test_host_vectors_are_staged(gk, orc):
    A, _ = MATS["poisson2d_64"]
    M = gk.Matrix(A[0], A[1], A[2], fmt="csr")  # host arrays, copied by the library
    x = W.uniform_vector(4096, 3)
    y = np.zeros(4096)
    gk.apply(M, x, y)  # host in, host out
    assert np.array_equal(y, orc.spmv(A, x))


def test_hyb_width_matches_oracle(gk, orc):
    for name in ("powerlaw_20000", "ragged_3000x2500", "poisson2d_64"):
        A, n_cols = MATS[name]
        M = _gk_matrix(gk, A, "hyb", n_cols)
        info = M.info()
        assert info["ell_width"] == orc.hyb_width(A)
        lens = np.diff(A[0])
        K = info["ell_width"]
        assert info["tail_rows"] == int((lens > K).sum())
        assert info["tail_nnz"] == int(np.maximum(lens - K, 0).sum())


def test_invalid_csr_rejected(gk):
    rp = np.array([0, 2, 3], np.int32)
    val = np.ones(3)
    for col, what in ((np.array([1, 0, 0], np.int32), "unsorted"),
                      (np.array([0, 0, 1], np.int32), "repeated"),
                      (np.array([0, 5, 1], np.int32), "out of range")):
        with pytest.raises(gk.GkError) as ei:
            gk.Matrix(to_dev(rp), to_dev(col), to_dev(val))
        assert ei.value.code == 5, what
    with pytest.raises(gk.GkError) as ei:
        gk.Matrix(to_dev(np.array([0, 2, 1], np.int32)), to_dev(np.array([0, 1], np.int32)), to_dev(np.ones(2)))
    assert ei.value.code == 5
    M = gk.Matrix(to_dev(rp), to_dev(np.array([0, 1, 1], np.int32)), to_dev(val))
    v = to_dev(np.ones(2))
    with pytest.raises(gk.GkError) as ei:
        gk.apply(M, v, v)
    assert ei.value.code == 1


def test_empty_matrix(gk):
    M = gk.Matrix(to_dev(np.zeros(1, np.int32)), to_dev(np.zeros(0, np.int32)), to_dev(np.zeros(0)))
    gk.apply(M, to_dev(np.zeros(0)), to_dev(np.zeros(0)))
    assert M.info()["nnz"] == 0


@pytest.mark.parametrize("fmt", ["csr", "csr_merge", "hyb", "ell"])
@pytest.mark.parametrize("which", ["stencil27_128", "powerlaw_1M"])
def test_full_size_sampled_rows(gk, orc, big_mats, fmt, which):
    """The benchmark's sizes and launch shapes: rows against the Dot2 bound
    on a sample of 4000 random rows, the first and last, and every row with
    more than 256 entries -- all rows of GK_CSR's warp-per-row (257..4096)
    and block-per-row (> 4096) bins, which are also the rows that the
    merge-path tiles and the HYB overflow split."""
    A = big_mats[which]
    n = A[0].size - 1
    if fmt == "ell" and which == "powerlaw_1M":
        with pytest.raises(gk.GkError):
            _gk_matrix(gk, A, fmt)
        return
    M = _gk_matrix(gk, A, fmt)
    x = W.uniform_vector(n, 11)
    y = to_dev(np.zeros(n))
    gk.apply(M, to_dev(x), y)
    y = to_np(y)
    rng = np.random.default_rng(12)
    lens_all = np.diff(A[0])
    long_rows = np.flatnonzero(lens_all > 256)
    if which == "powerlaw_1M":
        # the sample must reach both long-row bins
        assert long_rows.size > 1000 and (lens_all > 4096).any()
    rows = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 4000), long_rows]))
    S = sub_rows(A, rows)
    y_acc, bnd = orc.spmv_accurate(S, x)
    assert_rows_within(y[rows], y_acc, bnd, 1e-13, f"{which}/{fmt}")
    if M.info()["format_name"] in ("csr", "ell"):
        lens = np.diff(S[0])
        exact = lens <= 256 if fmt == "csr" else np.ones(lens.size, bool)
        assert np.array_equal(y[rows][exact], orc.spmv(S, x)[exact])


@pytest.fixture(scope="module")
def big_mats():
    return {"stencil27_128": W.stencil27(128), "powerlaw_1M": W.powerlaw(1_000_000, seed=3)}


@pytest.mark.parametrize("fmt", ["csr", "csr_merge", "ell", "hyb"])
def test_apply_dot_fuses_the_dot(gk, orc, fmt):
    """x = A b equals gk_apply bit for bit, and result = u . x within the
    rounding of a length-n dot product; run to run bit-identical."""
    import torch
    A = W.poisson2d(70)
    n = 4900
    b, u = W.uniform_vector(n, 1), W.uniform_vector(n, 2)
    M = _gk_matrix(gk, A, fmt)
    x1 = to_dev(np.zeros(n))
    x2 = to_dev(np.zeros(n))
    r = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    gk.apply(M, to_dev(b), x1)
    gk.apply_dot(M, to_dev(b), x2, to_dev(u), r[0:1])
    gk.apply_dot(M, to_dev(b), x2, to_dev(u), r[1:2])
    np.testing.assert_array_equal(to_np(x1), to_np(x2))
    rv = to_np(r)
    assert rv[0] == rv[1]
    x = to_np(x2)
    ref = float(np.dot(u, x))
    assert abs(rv[0] - ref) <= 1e-13 * float(np.dot(np.abs(u), np.abs(x)))


def test_apply_dot_long_row_pieces(gk, big_mats):
    """GK_CSR on the power-law matrix with 10^6 rows: its rows of more than
    512 entries are summed in pieces, added by a second launch that also
    finishes the fused dot's reduction.  x = A b through the fused-dot apply
    equals the plain apply bit for bit, the dot is within the rounding of a
    length-n dot product of u . x, and both are identical from run to run."""
    import torch
    A = big_mats["powerlaw_1M"]
    n = A[0].size - 1
    lens = np.diff(A[0])
    assert (lens > 512).sum() > 1000
    b, u = W.uniform_vector(n, 31), W.uniform_vector(n, 32)
    M = _gk_matrix(gk, A, "csr")
    assert M.info()["long_rows"] == int((lens > 256).sum())
    assert M.info()["split_rows"] == int((lens > 512).sum())
    x1, x2 = to_dev(np.zeros(n)), to_dev(np.zeros(n))
    r = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    gk.apply(M, to_dev(b), x1)
    gk.apply_dot(M, to_dev(b), x2, to_dev(u), r[0:1])
    x = to_np(x2)
    np.testing.assert_array_equal(to_np(x1), x)
    gk.apply_dot(M, to_dev(b), x2, to_dev(u), r[1:2])
    np.testing.assert_array_equal(to_np(x2), x)
    rv = to_np(r)
    assert rv[0] == rv[1]
    assert abs(rv[0] - float(np.dot(u, x))) <= 1e-13 * float(np.dot(np.abs(u), np.abs(x)))
