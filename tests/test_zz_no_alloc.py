"""gk_dot_noalloc against gk_dot and the oracle's dot product.

gk_dot_noalloc serves callers that cannot allocate device memory (their GPU
memory is reserved by another allocator, or their host application forbids
libraries from owning device allocations); it keeps its reduction scratch in
a static device array.  It runs gk_dot's kernel on gk_dot's grid, so on two
calls in a row (the second one reuses the scratch the first one left behind)
its result must equal gk_dot's bit for bit, and both must be within
1e-13 * sum_i |x_i y_i| of the oracle's sequential sum.  Collected last so
that a failure here does not hide the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_dot_on_two_calls(gk, orc):
    import torch
    L = gk.load()
    rng = np.random.default_rng(21)
    for n in (1_000_003, 4096, 1):
        xh, yh = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
        x = torch.from_numpy(xh).cuda()
        y = torch.from_numpy(yh).cuda()
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        assert L.gk_dot(n, x.data_ptr(), y.data_ptr(), ref.data_ptr(), None) == 0
        torch.cuda.synchronize()
        bound = float(np.sum(np.abs(xh * yh)))
        oracle_dot = orc.dot(xh, yh)
        assert abs(ref.item() - oracle_dot) <= 1e-13 * bound, (n, ref.item(), oracle_dot)
        for call in range(2):
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            rc = L.gk_dot_noalloc(n, x.data_ptr(), y.data_ptr(), out.data_ptr(), None)
            assert rc == 0, L.gk_last_error()
            torch.cuda.synchronize()
            assert out.item() == ref.item(), (n, call, out.item(), ref.item())


def test_dot_noalloc_argument_errors(gk):
    L = gk.load()
    assert L.gk_dot_noalloc(-1, None, None, None, None) == 1
    host = np.zeros(4)
    p = host.ctypes.data
    assert L.gk_dot_noalloc(4, p, p, p, None) == 4
