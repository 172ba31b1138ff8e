"""CPU oracle of the learned warm start: the convolutional network that
predicts an initial guess for the variable-coefficient diffusion solves, its
gradients, its loss, the Adam update and its BF16 inference.

TEST INFRASTRUCTURE ONLY: used by ``tests/`` and ``bench.py``'s CPU legs;
the product library never imports it and shares no code with it.  Plain
numpy in float64 (the BF16 inference rounds to BF16 where the kernel does and
sums in float64).

The network (not in the paper: the warm start extends the method; its
definition is this project's):
  * input  (B, 2, H, W): the log-coefficient field g and the right-hand side
    divided by its root mean square;
  * 6 layers of 3x3 convolutions with dilation d_l and zero padding,
    channels 2 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1:
        y[b, o, i, j] = bias[o] + sum_{c, ky, kx} w[o, c, ky, kx]
                        * x[b, c, i + d (ky - 1), j + d (kx - 1)]
    with ReLU after every layer but the last;
  * output (B, 1, H, W): the solution divided by (rms(b) * out_scale).
Loss: the mean squared error over all output entries, or the energy norm of
the error in the sample's own operator (energy()).
"""
from __future__ import annotations

import numpy as np

CHANNELS = (2, 32, 32, 32, 32, 32, 1)
DILATIONS = (1, 2, 4, 8, 16, 32)


def init_params(seed, channels=CHANNELS):
    """He-normal weights (std sqrt(2 / (9 c_in))), the last layer with std
    sqrt(1 / (9 c_in)), zero biases.  Returns a list of (w, bias) float64."""
    rng = np.random.default_rng(seed)
    params = []
    L = len(channels) - 1
    for l in range(L):
        ci, co = channels[l], channels[l + 1]
        std = np.sqrt((1.0 if l == L - 1 else 2.0) / (9.0 * ci))
        params.append((rng.normal(0.0, std, size=(co, ci, 3, 3)), np.zeros(co)))
    return params


def flatten(params):
    """All parameters in one vector: per layer w (o, c, ky, kx) then bias."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def unflatten(vec, channels=CHANNELS):
    out, k = [], 0
    for l in range(len(channels) - 1):
        ci, co = channels[l], channels[l + 1]
        nw = co * ci * 9
        out.append((np.asarray(vec[k:k + nw], dtype=np.float64).reshape(co, ci, 3, 3),
                    np.asarray(vec[k + nw:k + nw + co], dtype=np.float64)))
        k += nw + co
    return out


def _shift(x, dy, dx):
    """s[..., i, j] = x[..., i + dy, j + dx], zero outside the grid."""
    H, W = x.shape[-2:]
    s = np.zeros_like(x)
    i0, i1 = max(0, -dy), min(H, H - dy)
    j0, j1 = max(0, -dx), min(W, W - dx)
    if i0 < i1 and j0 < j1:
        s[..., i0:i1, j0:j1] = x[..., i0 + dy:i1 + dy, j0 + dx:j1 + dx]
    return s


def conv_forward(x, w, bias, dil):
    """The dilated 3x3 convolution above, summed tap by tap."""
    B, C, H, W = x.shape
    y = np.broadcast_to(bias[None, :, None, None], (B, w.shape[0], H, W)).copy()
    for ky in range(3):
        for kx in range(3):
            xs = _shift(x, dil * (ky - 1), dil * (kx - 1))
            y += np.einsum("oc,bchw->bohw", w[:, :, ky, kx], xs)
    return y


def conv_backward(x, w, dil, dy):
    """Gradients of sum(dy * conv_forward(x, w, bias, dil)) with respect to
    x, w and bias:
      dw[o, c, ky, kx] = sum dy[b, o, i, j] x[b, c, i + d (ky-1), j + d (kx-1)]
      dx[b, c, i, j]   = sum_{o, ky, kx} w[o, c, ky, kx] dy[b, o, i - d (ky-1), j - d (kx-1)]
      dbias[o]         = sum dy[b, o, i, j]."""
    dw = np.zeros_like(w)
    dx = np.zeros_like(x)
    for ky in range(3):
        for kx in range(3):
            oy, ox = dil * (ky - 1), dil * (kx - 1)
            dw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", dy, _shift(x, oy, ox))
            dx += np.einsum("oc,bohw->bchw", w[:, :, ky, kx], _shift(dy, -oy, -ox))
    return dx, dw, dy.sum(axis=(0, 2, 3))


def forward(params, x, dilations=DILATIONS):
    """Returns (output, activations): activations[l] is the input of layer l
    (after the previous ReLU)."""
    acts = [x]
    h = x
    L = len(params)
    for l, ((w, b), d) in enumerate(zip(params, dilations)):
        h = conv_forward(h, w, b, d)
        if l < L - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return h, acts


def mse(out, target):
    """Loss and its gradient with respect to out."""
    diff = out - target
    return float(np.mean(diff * diff)), 2.0 * diff / diff.size


def energy(out, target, g):
    """Energy-norm loss (1 / N) sum_p e_p (A e)_p, e = out - target, A the
    5-point variable-coefficient operator of each sample (cell coefficients
    exp(g), faces the harmonic mean of the two cells, a boundary face the
    cell's own coefficient), and its gradient 2 A e / N.  out, target
    (B, 1, H, W); g (B, H, W)."""
    e = (out - target)[:, 0]
    c = np.exp(g)
    ae = np.zeros_like(e)
    B, H, W = e.shape
    for di, dj in ((-1, 0), (0, -1), (0, 1), (1, 0)):
        cn = _shift(c, di, dj)
        en = _shift(e, di, dj)
        inside = _shift(np.ones_like(c), di, dj) > 0
        f = np.where(inside, 2.0 * c * cn / np.where(inside, c + cn, 1.0), c)
        ae += f * e - np.where(inside, f * en, 0.0)
    n = e.size
    return float(np.sum(e * ae) / n), (2.0 * ae / n)[:, None]


def backward(params, acts, dout, dilations=DILATIONS):
    """Gradients of the loss for every (w, bias), given dL/d(output)."""
    grads = [None] * len(params)
    g = dout
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        dx, dw, db = conv_backward(acts[l], w, dilations[l], g)
        grads[l] = (dw, db)
        if l > 0:
            g = dx * (acts[l] > 0.0)  # ReLU of layer l - 1
    return grads


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma and Ba, 2015) on flat vectors, step t >= 1; returns the
    new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64:
    keep the top 16 bits of the float32 pattern after adding 0x7FFF plus the
    lowest kept bit (IEEE round-to-nearest-even on the 16 dropped bits)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def infer_bf16(params, x, dilations=DILATIONS):
    """The inference the BF16 kernel computes: weights, biases, the input
    and every hidden activation rounded to BF16; products and sums exact
    (float64 here, FP32 accumulation in the kernel); the output kept in
    full precision."""
    h = bf16(x)
    L = len(params)
    for l, ((w, b), d) in enumerate(zip(params, dilations)):
        h = conv_forward(h, bf16(w), bf16(b), d)
        if l < L - 1:
            h = bf16(np.maximum(h, 0.0))
    return h


def features(g, b):
    """Network input of one problem: (2, H, W) = [g, b / rms(b)] and rms(b)."""
    H, W = g.shape
    s = float(np.sqrt(np.mean(b * b)))
    return np.stack([g, b.reshape(H, W) / (s if s > 0 else 1.0)]), s
