"""gk_dot_noalloc against gk_dot.

gk_dot_noalloc serves callers that cannot allocate device memory (their GPU
memory is reserved by another allocator, or their host application forbids
libraries from owning device allocations); it keeps its reduction scratch in
a static device array.  It must give gk_dot's result, here within the 1e-13
relative tolerance the other parity tests use, on two calls in a row (the
second one reuses the scratch the first one left behind).  Collected last so
that a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_dot_on_two_calls(gk):
    import torch
    L = gk.load()
    rng = np.random.default_rng(21)
    for n in (1_000_003, 4096):
        x = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
        y = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        assert L.gk_dot(n, x.data_ptr(), y.data_ptr(), ref.data_ptr(), None) == 0
        bound = float((x.abs() * y.abs()).sum())
        for call in range(2):
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            rc = L.gk_dot_noalloc(n, x.data_ptr(), y.data_ptr(), out.data_ptr(), None)
            assert rc == 0, L.gk_last_error()
            torch.cuda.synchronize()
            assert abs(out.item() - ref.item()) <= 1e-13 * bound, (call, out.item(), ref.item())


def test_dot_noalloc_argument_errors(gk):
    L = gk.load()
    assert L.gk_dot_noalloc(-1, None, None, None, None) == 1
    host = np.zeros(4)
    p = host.ctypes.data
    assert L.gk_dot_noalloc(4, p, p, p, None) == 4
