"""Failure detection on the GPU without a fault: a bounded device-side wait
that nothing satisfies gives up, reports the timeout through the device
error word, and leaves the context usable for the next call."""
import time

import numpy as np
import pytest

from helpers import to_dev

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_device_stays_usable(gk):
    import torch
    t0 = time.perf_counter()
    err = gk.wait_selftest()
    dt = time.perf_counter() - t0
    assert err == 1                 # the timeout bit, and not "the phase completed"
    assert 0.5 < dt < 60.0          # the ~2 s clock limit, whatever the SM clock
    # the context survived: a reduction and an SpMV still give exact results
    x = torch.arange(1000, dtype=torch.float64, device="cuda:0")
    r = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    gk.dot(x, x, r)
    assert r.item() == float(sum(i * i for i in range(1000)))
    import workloads as W
    A = W.poisson2d(16)
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]))
    y = torch.zeros(256, dtype=torch.float64, device="cuda:0")
    gk.apply(M, torch.ones(256, dtype=torch.float64, device="cuda:0"), y)
    D = W.csr_to_dense(A)
    assert np.array_equal(y.cpu().numpy(), D @ np.ones(256))
