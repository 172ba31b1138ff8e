"""The benchmark's byte accounting against the paper's Table 2 (Section 7.3).

`tests/golden/table2_memory_volume.txt` restates the table's read and write
volumes as expressions; this test evaluates them on its own and compares
them with `bench.table2_bytes` for every solver, on iteration counts that
are even and odd and GMRES counts below, at and past a restart."""
import math
import os

import pytest

import bench

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_memory_volume.txt")


def _table():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            solver, side, expr = (p.strip() for p in line.split("|"))
            rows[(solver, side)] = expr
    return rows


def _eval(expr, n, nnz, it_count, k, vt, it):
    q, r = divmod(it_count, k)
    env = {"n": n, "nnz": nnz, "VT": vt, "IT": it, "iter": it_count, "k": k, "r": r, "q": q,
           "iter_r": q * (k - 1) * k / 2 + (r - 1) * r / 2,
           "ceil2": math.ceil(it_count / 2), "floor2": it_count // 2}
    return eval(expr, {"__builtins__": {}}, env)


def test_golden_has_every_solver():
    rows = _table()
    for s in ("cg", "fcg", "bicgstab", "cgs", "gmres"):
        assert (s, "read") in rows and (s, "write") in rows


@pytest.mark.parametrize("solver", ["cg", "fcg", "bicgstab", "cgs", "gmres"])
@pytest.mark.parametrize("iters", [0, 1, 2, 7, 99, 100, 101, 250])
@pytest.mark.parametrize("vt,it", [(8, 4), (4, 4), (8, 8)])
def test_table2_bytes_matches_the_table(solver, iters, vt, it):
    rows = _table()
    n, nnz, k = 2_097_152, 55_742_968, 100
    rd, wr = bench.table2_bytes(solver, iters, nnz, n, vt, it, k=k)
    assert rd == pytest.approx(_eval(rows[(solver, "read")], n, nnz, iters, k, vt, it), rel=1e-15, abs=1e-6)
    assert wr == pytest.approx(_eval(rows[(solver, "write")], n, nnz, iters, k, vt, it), rel=1e-15, abs=1e-6)


def test_table2_cg_per_iteration_volume():
    """Per CG iteration the table's volume is 20 n VT + 2 nnz (VT + IT) + 2 VT;
    the setup is 9 n VT + 2 nnz (VT + IT) + 2 VT."""
    n, nnz = 1000, 5000
    t0 = sum(bench.table2_bytes("cg", 0, nnz, n))
    t1 = sum(bench.table2_bytes("cg", 1, nnz, n))
    assert t0 == 9 * n * 8 + 2 * nnz * 12 + 16
    assert t1 - t0 == 20 * n * 8 + 2 * nnz * 12 + 16
    assert bench.table2_cg_bytes(3, nnz, n) == t0 + 3 * (t1 - t0)


def test_spmv_bytes_of_the_benchmark_matrix():
    """The 27-point matrix on 128^3: nnz (8 + 4) + (n + 1) 4 + 8 n (x, read
    once) + 8 n (y) = 710.9 MB; with the fused dot's second vector, 727.6 MB
    (the roofline kernel's algorithmic bytes per launch)."""
    n, nnz = 128 ** 3, 55_742_968
    assert bench.spmv_bytes(nnz, n, n) == 710_858_660
    assert bench.spmv_bytes(nnz, n, n) + 8 * n == 727_635_876


@pytest.mark.parametrize("prec,bs,vec", [("none", 1, 72), ("jacobi", 1, 88), ("block", 8, 80 + 8 * 8),
                                         ("block", 32, 80 + 8 * 32)])
def test_cg_bytes_per_iteration(prec, bs, vec):
    """Per CG iteration the model moves one SpMV plus the fused vector
    kernels' bytes: 72 n unpreconditioned, 88 n with scalar Jacobi,
    80 n + 8 bs n with block Jacobi (the inverse blocks once)."""
    n, nnz = 1000, 27_000
    per = bench.cg_bytes(1, nnz, n, prec, bs) - bench.cg_bytes(0, nnz, n, prec, bs)
    assert per == bench.spmv_bytes(nnz, n, n) + vec * n
    assert bench.cg_bytes(5, nnz, n, prec, bs) - bench.cg_bytes(0, nnz, n, prec, bs) == 5 * per


def test_bicgstab_bytes_half_step_is_cheaper():
    """A BiCGSTAB iteration that ends at its half step does one SpMV instead
    of two: with the same iteration count, one SpMV fewer means fewer bytes."""
    n, nnz = 1000, 5000
    full = bench.bicgstab_bytes(10, 2 + 20, nnz, n, "jacobi")
    half = bench.bicgstab_bytes(10, 2 + 19, nnz, n, "jacobi")
    assert half < full
    assert full - half >= bench.spmv_bytes(nnz, n, n)


def test_spmv_bytes_per_format():
    """The stored operator's bytes follow the format: CSR reads row pointers,
    ELL does not (nnz (VT + IT) + 2 n VT: 702.5 MB on the 27-point matrix,
    719.2 MB with the fused dot's second vector -- the roofline kernel's
    algorithmic bytes per launch), and HYB's COO part carries a row index
    per entry (nnz_ell (VT + IT) + nnz_coo (VT + 2 IT) + 2 n VT)."""
    n, nnz = 128 ** 3, 55_742_968
    assert bench.spmv_bytes(nnz, n, n, fmt="ell") == nnz * 12 + 16 * n == 702_470_048
    assert bench.spmv_bytes(nnz, n, n, fmt="ell") + 8 * n == 719_247_264
    assert bench.spmv_bytes(nnz, n, n, fmt="csr_merge") == bench.spmv_bytes(nnz, n, n)
    assert bench.spmv_bytes(1000, 100, 100, fmt="hyb", tail_nnz=300) == 700 * 12 + 300 * 16 + 1600
    assert bench.spmv_bytes(1000, 100, 100, fmt="hyb", tail_nnz=0) == bench.spmv_bytes(1000, 100, 100, fmt="ell")
    # a CG iteration carries the format's SpMV
    d = bench.cg_bytes(1, nnz, n, "jacobi", fmt="ell") - bench.cg_bytes(0, nnz, n, "jacobi", fmt="ell")
    assert d == bench.spmv_bytes(nnz, n, n, fmt="ell") + 88 * n


def test_solve_launches_counts_idle_iterations():
    """CG launches init, the set-up SpMV and start, three kernels per
    iteration (the SpMV, update and direction; a GK_CSR matrix's SpMV is one
    kernel when no row has more than 512 entries, else two) including the
    iterations launched after the stop (idle_iters), and the final SpMV."""
    assert bench.solve_launches("cg", 251, 253, 1) == 2 + 1 + 251 * 3 + 1
    assert bench.solve_launches("cg", 251, 253, 1, idle=1) == 2 + 1 + 252 * 3 + 1
    # HYB with an overflow: 3 kernels per SpMV
    assert bench.solve_launches("cg", 14, 16, 3, idle=2) == 2 + 3 + 16 * 5 + 3


def test_inference_byte_model():
    """The warm-start inference moves 596 bytes per pixel (2 FP32 features
    in, four 32-channel BF16 activations out and back in, nine FP32 tap
    planes of the folded last layer out and back in, one FP32 output) for
    2 x 37,728 flops: about 127 flops per byte, below the ridge of a GPU
    with ~1.9 PFLOP/s BF16 and ~6.7 TB/s, so HBM bounds it."""
    bpp = bench.infer_bytes_per_pixel()
    assert bpp == 2 * 4 + 4 * 32 * 2 * 2 + 9 * 4 * 2 + 4 == 596
    macs = sum(a * b * 9 for a, b in zip((2, 32, 32, 32, 32, 32), (32, 32, 32, 32, 32, 1)))
    assert macs == 37728
    assert 2 * macs / bpp < 1.9e15 / 6.7e12


def test_spmv_launch_counts_per_format():
    """One kernel per GK_CSR apply, two when rows of more than 512 entries are
    summed in pieces (their second launch adds the pieces); two for the merge
    path (tiles and fix-up); three for HYB with an overflow (COO, its fix-up,
    ELL), one without; one for ELL."""
    assert bench.spmv_launches({"format_name": "csr", "split_rows": 0}) == 1
    assert bench.spmv_launches({"format_name": "csr", "split_rows": 4165}) == 2
    assert bench.spmv_launches({"format_name": "csr_merge"}) == 2
    assert bench.spmv_launches({"format_name": "hyb", "tail_rows": 10}) == 3
    assert bench.spmv_launches({"format_name": "hyb", "tail_rows": 0}) == 1
    assert bench.spmv_launches({"format_name": "ell"}) == 1
