"""The learned warm start: training data from the library's own solver,
training of the warm-start network through its C ABI (``gk_wsnet_*``), and
the comparison of CG from the predicted x0 with CG from zero.

Not in the paper: an extension of the method.  The network, its kernels and
its definition are in ``csrc/wsnet.cu`` and ``include/gk.h``; this module only
orchestrates calls (every arithmetic step runs in the library's kernels, the
problems come from ``workloads``)."""
from __future__ import annotations

import ast
import math
import os
import time

import numpy as np

import paper_2006_16852_gb300 as gk

CHANNELS = (2, 32, 32, 32, 32, 32, 1)
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
# Dilations per grid size: the receptive field 1 + 2 * sum(d) spans most of
# the grid, and the last layers use dilation 1 so that the output is smooth.
DILATIONS = {64: (1, 4, 16, 4, 1, 1), 256: (1, 4, 16, 64, 4, 1)}


def dilations_for(side: int):
    return DILATIONS.get(side, (1, 4, 16, 4, 1, 1))


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (9 c_in)); the last layer
    sqrt(1 / (9 c_in))), zero biases, in the flat parameter layout."""
    rng = np.random.default_rng(seed)
    parts = []
    L = len(CHANNELS) - 1
    for l in range(L):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        std = math.sqrt((1.0 if l == L - 1 else 2.0) / (9.0 * ci))
        parts.append(rng.normal(0.0, std, size=co * ci * 9))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def solve_stack(side: int, indices, dev, tol: float = 1e-8, max_iters: int = 20000):
    """Solutions of problems `indices` by Jacobi-CG on their block-diagonal
    stack (one global criterion ||r|| <= tol ||b||).  Returns device arrays
    (g (S, side^2), b (S, side^2), x (S, side^2)) in FP64 and the status."""
    import torch
    import workloads as W
    gs, bs, A = W.grf_stack(side, list(indices))
    dA = [_t(a, dev) for a in A]
    M = gk.Matrix(*dA, fmt="ell")
    P = gk.Precond(M, 1)
    S = gk.Solver(M, P, "cg", max_iters=max_iters, reduction_factor=tol)
    b = _t(bs.reshape(-1), dev)
    x = torch.zeros_like(b)
    st = gk.solve(S, b, x)
    n = side * side
    return _t(gs.reshape(len(indices), n), dev), b.view(len(indices), n), x.view(len(indices), n), st


def make_training_data(net: gk.WsNet, count: int, start: int = 0, stack: int = 64, tol: float = 1e-8,
                       out_scale: float | None = None, dev="cuda:0", log=None):
    """Inputs (count, 2, H, W) and targets (count, 1, H, W) float32 on the
    device for problems start .. start + count - 1, their solutions computed
    by the library's CG.  out_scale (x / (rms(b) out_scale) ~ O(1)) is taken
    from the first stack when not given."""
    import torch
    side = net.H
    feats = torch.empty((count, 2, side, side), dtype=torch.float32, device=dev)
    tgts = torch.empty((count, 1, side, side), dtype=torch.float32, device=dev)
    t0 = time.time()
    iters = []
    for k0 in range(0, count, stack):
        idx = range(start + k0, start + min(count, k0 + stack))
        g, b, x, st = solve_stack(side, idx, dev, tol)
        iters.append(st.iters)
        if out_scale is None:
            xr = x.norm(dim=1) / b.norm(dim=1)
            out_scale = float(xr.median().item())
        for j in range(len(idx)):
            net.features(g[j], b[j], feats[k0 + j], x=x[j], target=tgts[k0 + j], out_scale=out_scale)
        if log:
            log(f"data {k0 + len(idx)}/{count}: stacked CG {st.iters} iterations, {time.time() - t0:.1f} s")
    torch.cuda.synchronize()
    return feats, tgts, out_scale, {"seconds": time.time() - t0, "stack_iters": iters}


def train(net: gk.WsNet, feats, tgts, epochs: int = 3, batch: int = 16, lr: float = 1e-3, log=None):
    """Adam over the samples in order (the problems are i.i.d.), cosine decay
    of the learning rate to lr / 20.  Returns the mean loss of every epoch."""
    import torch
    count = feats.shape[0]
    steps_per_epoch = count // batch
    total = epochs * steps_per_epoch
    losses = torch.zeros(total, dtype=torch.float32, device=feats.device)
    t0 = time.time()
    hist = []
    step = 0
    for ep in range(epochs):
        for k in range(steps_per_epoch):
            frac = step / max(total - 1, 1)
            cur = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * frac)))
            sl = slice(k * batch, (k + 1) * batch)
            net.train_step(feats[sl], tgts[sl], cur, loss_out=losses[step:step + 1])
            step += 1
        ep_loss = float(losses[ep * steps_per_epoch:(ep + 1) * steps_per_epoch].mean().item())
        hist.append(ep_loss)
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {ep_loss:.4e}, {time.time() - t0:.1f} s")
    return hist, time.time() - t0


def energy_error(M: gk.Matrix, x, xs) -> float:
    """||x - xs||_A / ||xs||_A with the library's SpMV and dot."""
    import torch
    e = x - xs
    ae = torch.zeros_like(e)
    gk.apply(M, e, ae)
    ax = torch.zeros_like(xs)
    gk.apply(M, xs, ax)
    d = torch.zeros(2, dtype=torch.float64, device=x.device)
    gk.dot(e, ae, d[0:1])
    gk.dot(xs, ax, d[1:2])
    v = d.cpu().numpy()
    return float(np.sqrt(max(v[0], 0.0) / v[1]))


def rel_residual(M: gk.Matrix, x, b) -> float:
    """||b - A x|| / ||b|| with the library's advanced apply and dot."""
    import torch
    r = b.clone()
    gk.apply_adv(-1.0, M, x, 1.0, r)
    d = torch.zeros(2, dtype=torch.float64, device=x.device)
    gk.dot(r, r, d[0:1])
    gk.dot(b, b, d[1:2])
    v = d.cpu().numpy()
    return float(np.sqrt(v[0] / v[1]))


def evaluate(net: gk.WsNet, indices, out_scale: float, tol: float = 1e-10, dev="cuda:0", project: bool = True):
    """Jacobi-CG from zero and from the network's x0 on problems `indices`:
    iterations, true residuals and device time (the warm start's time includes
    the feature construction, the BF16 inference and the A-norm scaling)."""
    import torch
    import workloads as W
    side = net.H
    out = []
    stream = torch.cuda.current_stream(dev)
    for i in indices:
        g, A, b = W.grf_problem(side, int(i))
        dA = [_t(a, dev) for a in A]
        M = gk.Matrix(*dA, fmt="ell")
        P = gk.Precond(M, 1)
        S = gk.Solver(M, P, "cg", max_iters=20000, reduction_factor=tol)
        gd, bd = _t(g.reshape(-1), dev), _t(b, dev)
        rec = {}
        for mode in ("zero", "warm", "zero", "warm"):  # the second round is timed warm
            x = torch.zeros_like(bd)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if mode == "warm":
                net.warm_start(gd, bd, x, out_scale, A=M if project else None)
            st = gk.solve(S, bd, x)
            e1.record(stream)
            e1.synchronize()
            rec[mode] = {"iters": st.iters, "ms": e0.elapsed_time(e1), "rel_res_true": st.rel_res_true,
                         "stop_reason": st.stop_reason}
            if mode == "zero":
                xs = x
        x0 = torch.zeros_like(bd)
        net.warm_start(gd, bd, x0, out_scale, A=M if project else None)
        rec["x0_energy_error"] = energy_error(M, x0, xs)
        rec["x0_rel_residual"] = rel_residual(M, x0, bd)
        out.append(rec)
    return out


def summarize(res):
    z = sum(r["zero"]["iters"] for r in res)
    w = sum(r["warm"]["iters"] for r in res)
    zm = sum(r["zero"]["ms"] for r in res)
    wm = sum(r["warm"]["ms"] for r in res)
    return {"problems": len(res), "iters_zero": z, "iters_warm": w, "iters_ratio": round(w / z, 4),
            "ms_zero": round(zm, 3), "ms_warm": round(wm, 3), "time_ratio": round(wm / zm, 4),
            "x0_energy_error_mean": round(float(np.mean([r["x0_energy_error"] for r in res])), 4),
            "x0_rel_residual_mean": round(float(np.mean([r["x0_rel_residual"] for r in res])), 4),
            "max_rel_res_true_warm": max(r["warm"]["rel_res_true"] for r in res)}


def main(argv=None):
    """Train the warm-start network on the GPU and save it:
    python -m paper_2006_16852_gb300.learned --side 256 --samples 20000 --out wsnet_256.npz"""
    import argparse
    import json
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--side", type=int, default=256)
    ap.add_argument("--samples", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--stack", type=int, default=64)
    ap.add_argument("--loss", default="energy", choices=["energy", "mse"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--eval", type=int, default=12, help="held-out problems to evaluate")
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    gk.load()
    log = lambda m: print(m, flush=True)
    net = gk.WsNet(a.side, a.side, a.batch, dilations_for(a.side))
    net.set_params(init_params(a.seed))
    net.set_loss(a.loss)
    feats, tgts, scale, dinfo = make_training_data(net, a.samples, stack=a.stack, log=log)
    hist, secs = train(net, feats, tgts, epochs=a.epochs, batch=a.batch, lr=a.lr, log=log)
    del feats, tgts
    summ = summarize(evaluate(net, range(1_000_000, 1_000_000 + a.eval), scale))
    meta = {"side": a.side, "samples": a.samples, "epochs": a.epochs, "batch": a.batch, "lr": a.lr,
            "loss": a.loss, "dilations": list(dilations_for(a.side)), "data_seconds": round(dinfo["seconds"], 1),
            "train_seconds": round(secs, 1), "loss_history": [round(h, 6) for h in hist], "eval": summ}
    save(a.out, net, scale, meta)
    print(json.dumps(meta))



def save(path: str, net: gk.WsNet, out_scale: float, meta: dict):
    np.savez(path, params=net.get_params(), out_scale=np.float64(out_scale), side=np.int64(net.H),
             dilations=np.array(net.dilations, dtype=np.int64), meta=np.array(repr(meta)))


def load(path: str, batch_max: int = 1):
    z = np.load(path)
    side = int(z["side"])
    net = gk.WsNet(side, side, batch_max, tuple(int(v) for v in z["dilations"]))
    net.set_params(z["params"])
    return net, float(z["out_scale"]), ast.literal_eval(str(z["meta"]))
if __name__ == "__main__":
    main()
