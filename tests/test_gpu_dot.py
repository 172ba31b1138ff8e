"""gk_dot, the library's fixed-order reduction (the dot products of every
Krylov step), against the oracle's sequential sum on random data.

The GPU sums per thread, per warp, per block and then over the block
partials in a fixed order; the oracle sums in increasing index order.  Both
are FP64 sums of the same n products, so they differ by rounding only:
|gk_dot - or_dot| <= 1e-13 * sum_i |x_i y_i| (the workload's stated
tolerance; the worst-case bound of either order is about n u sum |x_i y_i|,
and for random signs the error grows like sqrt(n) u).  Repeated calls are
bit-identical."""
import numpy as np
import pytest

import workloads as W
from helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 7, 255, 256, 257, 4095, 65_537, 1_000_000, 1_000_003, 4_194_305])
def test_dot_against_oracle(gk, orc, n):
    import torch
    xh = W.uniform_vector(n, 100 + n % 97)
    yh = W.uniform_vector(n, 200 + n % 89)
    if n > 100:
        # a few large entries, so that the sum is dominated by some terms
        xh[:: max(1, n // 17)] *= 1e3
    x, y = to_dev(xh), to_dev(yh)
    r = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    gk.dot(x, y, r[0:1])
    gk.dot(x, y, r[1:2])
    got = r.cpu().numpy()
    assert got[0] == got[1]
    ref = orc.dot(xh, yh)
    bound = float(np.sum(np.abs(xh * yh)))
    assert abs(got[0] - ref) <= 1e-13 * bound, (n, got[0], ref, bound)


def test_dot_empty(gk):
    import torch
    r = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda:0")
    z = torch.zeros(0, dtype=torch.float64, device="cuda:0")
    gk.dot(z, z, r)
    assert r.item() == 0.0


@pytest.mark.parametrize("n", [0, 1, 1000, 2_000_003])
def test_gather_dot_against_oracle(gk, orc, n):
    """gk_gather_dot = sum_k v_k x[c_k] within 1e-13 sum |v_k x[c_k]| of the
    oracle's sequential dot of v with the gathered x; an index outside
    [0, len(x)) contributes 0; repeated calls are bit-identical."""
    import torch
    nx = 100_003
    rng = np.random.default_rng(40 + n % 7)
    c = rng.integers(0, nx, n).astype(np.int32)
    if n > 10:
        c[3] = -1
        c[7] = nx
    v = W.uniform_vector(n, 41)
    x = W.uniform_vector(nx, 42)
    xg = np.where((c >= 0) & (c < nx), x[np.clip(c, 0, nx - 1)], 0.0)
    r = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    cd = torch.from_numpy(c).to("cuda:0")
    gk.gather_dot(cd, to_dev(v), to_dev(x), r[0:1])
    gk.gather_dot(cd, to_dev(v), to_dev(x), r[1:2])
    got = r.cpu().numpy()
    assert got[0] == got[1]
    ref = orc.dot(v, xg)
    assert abs(got[0] - ref) <= 1e-13 * float(np.sum(np.abs(v * xg))), (got[0], ref)


def test_fp64_rate_is_measured(gk):
    """gk_fp64_rate times FP64 fused multiply-adds on the device: a positive
    rate below the nominal FP64 peak of a GB300 (1.25 TFLOP/s) with some
    margin, and more iterations give about the same rate."""
    r1 = gk.fp64_rate(5000)
    r2 = gk.fp64_rate(20000)
    assert 0.05 < r1 < 1.5 and 0.05 < r2 < 1.5, (r1, r2)
    assert abs(r1 - r2) <= 0.25 * max(r1, r2), (r1, r2)
