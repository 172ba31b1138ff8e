"""GPU parity of the warm-start network (gk_wsnet_*) against the CPU oracle
(oracle/wsnet.py): FP32 forward, loss and every gradient, the Adam step, BF16
inference; determinism of the training step; and the gain of the trained
network over zero-start CG on held-out problems."""
import numpy as np
import pytest

import workloads as W
from helpers import to_dev, to_np
from oracle import wsnet as ON

pytestmark = pytest.mark.gpu

DIL = (1, 2, 4, 8, 16, 32)


def _net(gk, H, W_, B, seed=0):
    net = gk.WsNet(H, W_, B, DIL)
    params = ON.init_params(seed)
    net.set_params(ON.flatten(params).astype(np.float32))
    # the oracle works on the FP32 values the GPU holds
    return net, ON.unflatten(ON.flatten(params).astype(np.float32).astype(np.float64))


def _data(B, H, W_, seed=1):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, 2, H, W_)).astype(np.float32)
    t = rng.standard_normal((B, 1, H, W_)).astype(np.float32)
    return x, t


def test_forward_matches_oracle(gk):
    net, params = _net(gk, 24, 20, 2)
    x, _ = _data(2, 24, 20)
    y = to_dev(np.zeros((2, 1, 24, 20), dtype=np.float32))
    net.forward(to_dev(x), y)
    ref, _ = ON.forward(params, x.astype(np.float64), DIL)
    got = to_np(y)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    np.testing.assert_allclose(got, ref, rtol=1e-3, atol=1e-4 * np.abs(ref).max())


def test_gradients_match_oracle(gk):
    """Loss and the gradient of every layer's weights and biases (relative
    error of each group <= 1e-4: FP32 sums of up to 2 * 24 * 20 terms)."""
    net, params = _net(gk, 24, 20, 2)
    x, t = _data(2, 24, 20)
    loss, g = net.gradients(to_dev(x), to_dev(t))
    out, acts = ON.forward(params, x.astype(np.float64), DIL)
    ref_loss, dout = ON.mse(out, t.astype(np.float64))
    grads = ON.backward(params, acts, dout, DIL)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    gl = ON.unflatten(g.astype(np.float64))
    for l, ((gw, gb), (rw, rb)) in enumerate(zip(gl, grads)):
        assert np.linalg.norm(gw - rw) <= 1e-4 * np.linalg.norm(rw), l
        assert np.linalg.norm(gb - rb) <= 1e-4 * np.linalg.norm(rb) + 1e-12, l


def test_energy_loss_gradients_match_oracle(gk):
    """The energy-norm loss of the sample's operator: loss and gradients."""
    net, params = _net(gk, 24, 20, 2)
    net.set_loss("energy")
    x, t = _data(2, 24, 20)
    loss, g = net.gradients(to_dev(x), to_dev(t))
    out, acts = ON.forward(params, x.astype(np.float64), DIL)
    ref_loss, dout = ON.energy(out, t.astype(np.float64), x[:, 0].astype(np.float64))
    grads = ON.backward(params, acts, dout, DIL)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    gl = ON.unflatten(g.astype(np.float64))
    for l, ((gw, gb), (rw, rb)) in enumerate(zip(gl, grads)):
        assert np.linalg.norm(gw - rw) <= 1e-4 * np.linalg.norm(rw), l
        assert np.linalg.norm(gb - rb) <= 1e-4 * np.linalg.norm(rb) + 1e-12, l


def test_gradients_are_deterministic(gk):
    net, _ = _net(gk, 32, 32, 4)
    x, t = _data(4, 32, 32)
    l1, g1 = net.gradients(to_dev(x), to_dev(t))
    l2, g2 = net.gradients(to_dev(x), to_dev(t))
    assert l1 == l2
    np.testing.assert_array_equal(g1, g2)


def test_adam_step_matches_oracle(gk):
    """One training step = the oracle's Adam update applied to the GPU's
    gradient (t = 1, lr 1e-3)."""
    net, params = _net(gk, 16, 16, 2)
    x, t = _data(2, 16, 16)
    p0 = net.get_params().astype(np.float64)
    _, g = net.gradients(to_dev(x), to_dev(t))
    net.train_step(to_dev(x), to_dev(t), 1e-3)
    p1 = net.get_params().astype(np.float64)
    ref, _, _ = ON.adam_step(p0, g.astype(np.float64), np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    np.testing.assert_allclose(p1, ref, rtol=1e-5, atol=1e-7)


def test_training_fits_a_batch(gk):
    net, _ = _net(gk, 16, 16, 4)
    x, t = _data(4, 16, 16)
    dx, dt = to_dev(x), to_dev(t)
    l0, _ = net.gradients(dx, dt)
    for _ in range(60):
        net.train_step(dx, dt, 3e-3)
    l1, _ = net.gradients(dx, dt)
    assert l1 < 0.5 * l0


def test_bf16_inference_matches_oracle(gk):
    """BF16 weights, inputs and activations with FP32 sums against the
    oracle's BF16 inference (float64 sums): they round the same values to
    BF16 except where an FP32 and an FP64 sum straddle a rounding boundary."""
    net, params = _net(gk, 24, 20, 2)
    x, _ = _data(2, 24, 20)
    y = to_dev(np.zeros((2, 1, 24, 20), dtype=np.float32))
    net.infer_bf16(to_dev(x), y)
    net.check()
    ref = ON.infer_bf16(params, x.astype(np.float64), DIL)
    got = to_np(y)
    assert np.linalg.norm(got - ref) <= 1e-2 * np.linalg.norm(ref)
    full, _ = ON.forward(params, x.astype(np.float64), DIL)
    # and BF16 stays close to the FP64 network
    assert np.linalg.norm(got - full) <= 5e-2 * np.linalg.norm(full)


@pytest.mark.parametrize("H,W_,B,dil", [(5, 300, 3, (1, 64, 3, 64, 2, 1)), (9, 128, 2, (2, 1, 7, 16, 5, 3)),
                                         (3, 1, 1, (1, 1, 1, 1, 1, 1)), (1, 257, 1, (1, 64, 64, 64, 64, 1))])
def test_bf16_inference_tiles_and_edges(gk, H, W_, B, dil):
    """The tensor-core layers over several 128-pixel tiles per image row,
    a ragged last tile, a one-pixel-wide and a one-row image, and dilations
    up to 64 (the staged window's full width, taps falling outside the
    image on both sides), per element against the oracle's BF16 inference:
    an element may differ by the BF16 rounding of its inputs, so the bound
    is 2 % of the output's scale plus 1 % of the element."""
    net = gk.WsNet(H, W_, B, dil)
    params = ON.init_params(5)
    net.set_params(ON.flatten(params).astype(np.float32))
    p32 = ON.unflatten(ON.flatten(params).astype(np.float32).astype(np.float64))
    rng = np.random.default_rng(9)
    x = rng.standard_normal((B, 2, H, W_)).astype(np.float32)
    y = to_dev(np.full((B, 1, H, W_), np.nan, dtype=np.float32))
    net.infer_bf16(to_dev(x), y)
    net.check()
    got = to_np(y)
    ref = ON.infer_bf16(p32, x.astype(np.float64), dil)
    assert np.all(np.isfinite(got))
    scale = np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= 2e-2 * scale + 1e-2 * np.abs(ref))
    assert np.linalg.norm(got - ref) <= 1e-2 * np.linalg.norm(ref)
    # run to run identical
    y2 = to_dev(np.zeros((B, 1, H, W_), dtype=np.float32))
    net.infer_bf16(to_dev(x), y2)
    np.testing.assert_array_equal(to_np(y2), got)


def test_features_and_targets(gk):
    """[g, b / rms(b)] and x / (rms(b) s) from FP64 arrays."""
    import torch
    net = gk.WsNet(8, 8, 1, DIL)
    rng = np.random.default_rng(3)
    g, b, x = rng.standard_normal(64), rng.standard_normal(64), rng.standard_normal(64)
    feat = torch.zeros((2, 8, 8), dtype=torch.float32, device="cuda:0")
    tgt = torch.zeros((1, 8, 8), dtype=torch.float32, device="cuda:0")
    net.features(to_dev(g), to_dev(b), feat, x=to_dev(x), target=tgt, out_scale=7.0)
    rms = np.sqrt(np.mean(b * b))
    np.testing.assert_allclose(to_np(feat)[0].ravel(), g.astype(np.float32), rtol=0)
    np.testing.assert_allclose(to_np(feat)[1].ravel(), b / rms, rtol=1e-6)
    np.testing.assert_allclose(to_np(tgt).ravel(), x / (rms * 7.0), rtol=1e-6)


def test_warm_start_against_zero_start(gk, orc):
    """Train on 2,048 problems of the family at 64 x 64 (solutions from the
    library's CG, energy-norm loss), then solve 12 held-out problems from the
    network's x0 and from zero.  What the network gains: x0 is much closer to
    the solution than x0 = 0 in the A-norm CG minimises (relative energy error
    < 0.5, against 1 for zero).  What it does not: its residual b - A x0 is
    larger than b itself (its error is broadband and A amplifies the high
    frequencies), so CG to ||r|| <= 1e-10 ||b|| needs as many iterations as
    from zero -- asserted as measured: within 2 % of the zero start, every
    warm-started solve meeting the criterion (the oracle's SpMV)."""
    from paper_2006_16852_gb300 import learned as LN
    net = gk.WsNet(64, 64, 16, LN.dilations_for(64))
    net.set_params(LN.init_params(0))
    net.set_loss("energy")
    feats, tgts, scale, _ = LN.make_training_data(net, 2048, start=0, stack=512, tol=1e-8)
    hist, _ = LN.train(net, feats, tgts, epochs=15, batch=16, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    res = LN.evaluate(net, range(100000, 100012), scale)
    s = LN.summarize(res)
    print(s)
    assert s["x0_energy_error_mean"] < 0.5
    assert s["x0_rel_residual_mean"] > 1.0
    assert s["iters_warm"] <= 1.02 * s["iters_zero"]
    for i, r in zip(range(100000, 100012), res):
        assert r["zero"]["stop_reason"] == r["warm"]["stop_reason"] == gk.STOP_CONVERGED
        assert r["warm"]["rel_res_true"] <= 1.05e-10
    # one solution checked independently
    g, A, b = W.grf_problem(64, 100000)
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt="ell")
    S = gk.Solver(M, gk.Precond(M, 1), "cg", max_iters=20000, reduction_factor=1e-10)
    x = to_dev(np.zeros(4096))
    net.warm_start(to_dev(g.reshape(-1)), to_dev(b), x, scale, A=M)
    gk.solve(S, to_dev(b), x)
    r = b - orc.spmv(A, to_np(x))
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(b)


def test_committed_network_on_held_out_problems(gk, orc):
    """The trained 256 x 256 network shipped with the package: on held-out
    problems its x0 is closer to the solution than zero in the A-norm while
    its residual exceeds ||b|| (7.5-10.8 ||b|| measured on held-out
    problems), and CG from it meets the criterion (checked with the
    oracle's SpMV)."""
    import os
    from paper_2006_16852_gb300 import learned as LN
    path = os.path.join(LN.DATA_DIR, "wsnet_256.npz")
    net, scale, meta = LN.load(path)
    assert meta["samples"] == 20000 and net.dilations == tuple(meta["dilations"])
    res = LN.evaluate(net, [1_000_100, 1_000_101], scale)
    for i, r in zip((1_000_100, 1_000_101), res):
        assert r["x0_energy_error"] < 0.6
        assert r["x0_rel_residual"] > 1.0
        assert r["warm"]["stop_reason"] == gk.STOP_CONVERGED
    g, A, b = W.grf_problem(256, 1_000_100)
    M = gk.Matrix(to_dev(A[0]), to_dev(A[1]), to_dev(A[2]), fmt="ell")
    S = gk.Solver(M, gk.Precond(M, 1), "cg", max_iters=20000, reduction_factor=1e-10)
    x = to_dev(np.zeros(65536))
    net.warm_start(to_dev(g.reshape(-1)), to_dev(b), x, scale, A=M)
    gk.solve(S, to_dev(b), x)
    r = b - orc.spmv(A, to_np(x))
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(b)
