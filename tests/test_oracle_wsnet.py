"""CPU pins of the warm-start network oracle (oracle/wsnet.py): the dilated
convolution against scipy's correlation with a zero-dilated kernel, its
gradients against central finite differences, Adam's first step in closed
form, BF16 rounding against its definition, and the problem generator."""
import numpy as np
import pytest

import workloads as W
from oracle import wsnet as N

scipy_signal = pytest.importorskip("scipy.signal")


def _dilated(k, d):
    """A 3x3 kernel spread to (2d+1)x(2d+1) with zeros between the taps."""
    out = np.zeros((2 * d + 1, 2 * d + 1))
    out[::d, ::d] = k
    return out


@pytest.mark.parametrize("dil", [1, 2, 5])
def test_conv_matches_scipy_correlation(dil):
    """y[o] = bias[o] + sum_c correlate(x[c], dilated w[o, c]) with zero
    padding ('same'), for every output channel."""
    rng = np.random.default_rng(dil)
    x = rng.standard_normal((2, 3, 9, 11))
    w = rng.standard_normal((4, 3, 3, 3))
    bias = rng.standard_normal(4)
    y = N.conv_forward(x, w, bias, dil)
    for bb in range(2):
        for o in range(4):
            ref = bias[o] + sum(scipy_signal.correlate2d(x[bb, c], _dilated(w[o, c], dil), mode="same",
                                                         boundary="fill", fillvalue=0.0) for c in range(3))
            np.testing.assert_allclose(y[bb, o], ref, rtol=1e-12, atol=1e-12)


def test_conv_identity_kernel():
    x = np.random.default_rng(0).standard_normal((1, 2, 5, 6))
    w = np.zeros((2, 2, 3, 3))
    w[0, 0, 1, 1] = w[1, 1, 1, 1] = 1.0
    np.testing.assert_array_equal(N.conv_forward(x, w, np.zeros(2), 3), x)


def _num_grad(f, arr, idx, eps=1e-6):
    old = arr[idx]
    arr[idx] = old + eps
    fp = f()
    arr[idx] = old - eps
    fm = f()
    arr[idx] = old
    return (fp - fm) / (2 * eps)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 6, 7))
    w = rng.standard_normal((4, 3, 3, 3))
    bias = rng.standard_normal(4)
    dy = rng.standard_normal((2, 4, 6, 7))
    f = lambda: float(np.sum(dy * N.conv_forward(x, w, bias, 2)))
    dx, dw, db = N.conv_backward(x, w, 2, dy)
    for idx in [(0, 0, 0, 0), (1, 2, 3, 4), (0, 1, 5, 6), (1, 0, 2, 0)]:
        assert dx[idx] == pytest.approx(_num_grad(f, x, idx), rel=1e-6, abs=1e-8)
    for idx in [(0, 0, 0, 0), (3, 2, 1, 2), (2, 1, 2, 0)]:
        assert dw[idx] == pytest.approx(_num_grad(f, w, idx), rel=1e-6, abs=1e-8)
    for o in range(4):
        assert db[o] == pytest.approx(_num_grad(f, bias, (o,)), rel=1e-6, abs=1e-8)


def test_network_gradients_finite_differences():
    """Every parameter group of a small network (the same code path as the
    full one) against central differences of the MSE loss."""
    ch, dil = (2, 4, 4, 1), (1, 2, 1)
    params = N.init_params(3, ch)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 2, 7, 6))
    t = rng.standard_normal((2, 1, 7, 6))

    def loss():
        out, _ = N.forward(params, x, dil)
        return N.mse(out, t)[0]

    out, acts = N.forward(params, x, dil)
    _, dout = N.mse(out, t)
    grads = N.backward(params, acts, dout, dil)
    for l, (w, b) in enumerate(params):
        gw, gb = grads[l]
        for idx in [(0, 0, 0, 0), (w.shape[0] - 1, w.shape[1] - 1, 2, 1), (0, w.shape[1] - 1, 1, 1)]:
            assert gw[idx] == pytest.approx(_num_grad(loss, w, idx), rel=1e-5, abs=1e-9)
        assert gb[0] == pytest.approx(_num_grad(loss, b, (0,)), rel=1e-5, abs=1e-9)


def test_flatten_round_trip_and_size():
    params = N.init_params(0)
    v = N.flatten(params)
    assert v.size == 2 * 32 * 9 + 32 + 4 * (32 * 32 * 9 + 32) + 32 * 9 + 1
    for (w0, b0), (w1, b1) in zip(params, N.unflatten(v)):
        np.testing.assert_array_equal(w0, w1)
        np.testing.assert_array_equal(b0, b1)


def test_adam_first_step_closed_form():
    """From m = v = 0 the bias-corrected first step is lr * g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = N.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_bf16_rounding():
    """Nearest bfloat16 (8 significant bits), ties to even, against the
    definition: the closer of the two neighbouring BF16 values."""
    one = 1.0
    assert N.bf16(one) == 1.0
    assert N.bf16(1.0 + 2.0 ** -8) == 1.0                    # tie -> even (1.0)
    assert N.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6    # tie -> even (1 + 2^-6)
    assert N.bf16(np.pi) == 3.140625
    rng = np.random.default_rng(5)
    v = (rng.standard_normal(2000) * np.exp(rng.uniform(-20, 20, 2000))).astype(np.float32)
    v64 = v.astype(np.float64)
    r = N.bf16(v)
    lo = (v.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)  # toward zero
    ulp = 2.0 ** (np.floor(np.log2(np.abs(lo))) - 7)
    hi = lo + np.sign(v64) * ulp
    best = np.minimum(np.abs(lo - v64), np.abs(hi - v64))
    assert np.all(np.abs(r - v64) <= best)
    assert np.all((r == lo) | (r == hi))


def test_bf16_inference_is_the_forward_at_bf16_inputs():
    """With weights and inputs already BF16 values and activations that the
    rounding leaves alone, BF16 inference equals the FP64 forward."""
    ch, dil = (2, 4, 1), (1, 2)
    params = [(N.bf16(w), N.bf16(b)) for w, b in N.init_params(6, ch)]
    x = N.bf16(np.random.default_rng(7).standard_normal((1, 2, 5, 5)))
    out, acts = N.forward(params, x, dil)
    inf = N.infer_bf16(params, x, dil)
    # the hidden activation is the only extra rounding
    h = N.bf16(acts[1])
    ref = N.conv_forward(h, params[1][0], params[1][1], dil[1])
    np.testing.assert_allclose(inf, ref, rtol=1e-15, atol=0)


def test_grf_problem_statistics():
    """The coefficient field has zero mean and unit variance over the
    ensemble, the source is a sum of four bumps, and b = h^2 f."""
    gs = np.stack([W.grf_field(32, (6, i, 0)) for i in range(200)])
    assert abs(gs.mean()) < 0.1 and abs(gs.var() - 1.0) < 0.15
    g, A, b = W.grf_problem(32, 3)
    assert A[0].size == 32 * 32 + 1 and b.shape == (1024,)
    f = W.gaussian_bumps(32, (6, 3, 1))
    np.testing.assert_allclose(b, f.ravel() / 33.0 ** 2, rtol=1e-15)
    D = W.csr_to_dense(A)
    np.testing.assert_array_equal(D, D.T)


def test_energy_loss_is_the_operator_norm(orc):
    """(1 / N) sum e.(A e) with A = varcoef2d(exp(g)) applied by the CSR
    oracle, and its gradient 2 A e / N."""
    rng = np.random.default_rng(8)
    g = rng.standard_normal((2, 7, 9))
    out = rng.standard_normal((2, 1, 7, 9))
    t = rng.standard_normal((2, 1, 7, 9))
    loss, grad = N.energy(out, t, g)
    tot, n = 0.0, out.size
    for b in range(2):
        A = W.varcoef2d(np.exp(g[b]))
        e = (out[b, 0] - t[b, 0]).ravel()
        ae = orc.spmv(A, e)
        tot += float(e @ ae)
        np.testing.assert_allclose(grad[b, 0].ravel(), 2.0 * ae / n, rtol=1e-12, atol=1e-14)
    assert loss == pytest.approx(tot / n, rel=1e-12)
