"""FP64 CPU oracle of the learned proposal network (TEST INFRASTRUCTURE ONLY).

The network is this project's extension, not the paper's: a 4-level
convolutional encoder-decoder that reads the half-resolution state of the
checkerboard update and proposes one plane per pixel, which the unchanged
matching cost of Eq. (8) then scores as one more candidate.  This module
writes its forward pass, loss and backward pass out plainly (3x3
convolutions as sums over the nine taps, 2x2 average pooling, nearest
upsampling, ReLU, additive skips, an L1 loss) so the CUDA kernels' outputs
and gradients can be checked.  Where the kernels store BF16 (weights, stored
activations, the output gradients the weight and data gradients read) the
oracle can round the same values to BF16 (``bf16=True``) so the comparison
isolates the arithmetic.

Layout: activations (H, W, C); conv weights (9, Cout, Cin) with tap
t = 3 * (dy + 1) + (dx + 1); bias (Cout,).
"""
from __future__ import annotations

import numpy as np

# (name, Cin, Cout, relu): e1..e4 encoder, d3..d1 decoder, out head
LAYERS = [("e1", 16, 32, True), ("e2", 32, 64, True), ("e3", 64, 96, True), ("e4", 96, 128, True),
          ("d3", 128, 96, True), ("d2", 96, 64, True), ("d1", 64, 32, True), ("out", 32, 16, False)]
OUT_USED = 4


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.asarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, w, b):
    """y[p, co] = b[co] + sum_t sum_ci w[t, co, ci] x[p + off(t), ci], zero padding."""
    H, W, _ = x.shape
    xp = np.zeros((H + 2, W + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    y = np.broadcast_to(b, (H, W, w.shape[1])).astype(np.float64).copy()
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        y += xp[1 + dy:1 + dy + H, 1 + dx:1 + dx + W] @ w[t].T
    return y


def conv3x3_dgrad(dy, w):
    """dx[q, ci] = sum_t sum_co dy[q - off(t), co] w[t, co, ci]."""
    H, W, _ = dy.shape
    dp = np.zeros((H + 2, W + 2, dy.shape[2]))
    dp[1:-1, 1:-1] = dy
    dx = np.zeros((H, W, w.shape[2]))
    for t in range(9):
        oy, ox = t // 3 - 1, t % 3 - 1
        dx += dp[1 - oy:1 - oy + H, 1 - ox:1 - ox + W] @ w[t]
    return dx


def conv3x3_wgrad(x, dy):
    """dw[t, co, ci] = sum_p dy[p, co] x[p + off(t), ci]; db[co] = sum_p dy[p, co]."""
    H, W, _ = x.shape
    xp = np.zeros((H + 2, W + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    dw = np.zeros((9, dy.shape[2], x.shape[2]))
    for t in range(9):
        oy, ox = t // 3 - 1, t % 3 - 1
        xs = xp[1 + oy:1 + oy + H, 1 + ox:1 + ox + W].reshape(-1, x.shape[2])
        dw[t] = dy.reshape(-1, dy.shape[2]).T @ xs
    return dw, dy.reshape(-1, dy.shape[2]).sum(0)


def pool2(x):
    H, W, C = x.shape
    return x.reshape(H // 2, 2, W // 2, 2, C).mean(axis=(1, 3))


def pool2_bwd(d):
    return np.repeat(np.repeat(d, 2, axis=0), 2, axis=1) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=0), 2, axis=1)


def up2_bwd(d):
    H, W, C = d.shape
    return d.reshape(H // 2, 2, W // 2, 2, C).sum(axis=(1, 3))


def forward(params, x0, bf16=False):
    """Returns (out, cache).  params: {name: (w, b)}."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    P = {k: (rnd(w), np.asarray(b, np.float64)) for k, (w, b) in params.items()}
    c = {}
    x = rnd(x0)
    c["in_e1"] = x
    c["e1"] = rnd(np.maximum(conv3x3(x, *P["e1"]), 0))
    c["in_e2"] = rnd(pool2(c["e1"]))
    c["e2"] = rnd(np.maximum(conv3x3(c["in_e2"], *P["e2"]), 0))
    c["in_e3"] = rnd(pool2(c["e2"]))
    c["e3"] = rnd(np.maximum(conv3x3(c["in_e3"], *P["e3"]), 0))
    c["in_e4"] = rnd(pool2(c["e3"]))
    c["e4"] = rnd(np.maximum(conv3x3(c["in_e4"], *P["e4"]), 0))
    c["in_d3"] = up2(c["e4"])
    c["r3"] = rnd(np.maximum(conv3x3(c["in_d3"], *P["d3"]), 0))
    c["d3"] = rnd(c["r3"] + c["e3"])
    c["in_d2"] = up2(c["d3"])
    c["r2"] = rnd(np.maximum(conv3x3(c["in_d2"], *P["d2"]), 0))
    c["d2"] = rnd(c["r2"] + c["e2"])
    c["in_d1"] = up2(c["d2"])
    c["r1"] = rnd(np.maximum(conv3x3(c["in_d1"], *P["d1"]), 0))
    c["d1"] = rnd(c["r1"] + c["e1"])
    c["in_out"] = c["d1"]
    out = conv3x3(c["d1"], *P["out"])
    c["P"] = P
    return out, c


def l1_loss(out, target, mask):
    """mean over masked pixels of sum_{c < 4} |out - target|, and d loss / d out."""
    n = max(1, int(mask.sum()))
    diff = out[..., :OUT_USED] - target[..., :OUT_USED]
    loss = float(np.abs(diff)[mask].sum() / n)
    g = np.zeros_like(out)
    g[..., :OUT_USED] = np.sign(diff) * mask[..., None] / n
    return loss, g


def backward(cache, dout, bf16=False):
    """Gradients {name: (dw, db)} for d loss / d out = dout."""
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    P = cache["P"]
    g = {}

    def conv_bwd(name, x_in, dy, need_dx=True):
        # weight and data gradients take dy as stored for the tensor cores
        # (BF16 when bf16), the bias gradient the unrounded dy
        g[name] = (conv3x3_wgrad(x_in, rnd(dy))[0], conv3x3_wgrad(x_in, dy)[1])
        return conv3x3_dgrad(rnd(dy), P[name][0]) if need_dx else None

    dd1 = conv_bwd("out", cache["in_out"], dout)
    dr1 = dd1 * (cache["r1"] > 0)
    de1 = dd1.copy()
    dd2 = up2_bwd(conv_bwd("d1", cache["in_d1"], dr1))
    dr2 = dd2 * (cache["r2"] > 0)
    de2 = dd2.copy()
    dd3 = up2_bwd(conv_bwd("d2", cache["in_d2"], dr2))
    dr3 = dd3 * (cache["r3"] > 0)
    de3 = dd3.copy()
    de4 = up2_bwd(conv_bwd("d3", cache["in_d3"], dr3))
    dc4 = de4 * (cache["e4"] > 0)
    de3 = de3 + pool2_bwd(conv_bwd("e4", cache["in_e4"], dc4))
    dc3 = de3 * (cache["e3"] > 0)
    de2 = de2 + pool2_bwd(conv_bwd("e3", cache["in_e3"], dc3))
    dc2 = de2 * (cache["e2"] > 0)
    de1 = de1 + pool2_bwd(conv_bwd("e2", cache["in_e2"], dc2))
    dc1 = de1 * (cache["e1"] > 0)
    conv_bwd("e1", cache["in_e1"], dc1, need_dx=False)
    return g


def init_params(seed=0):
    """He-normal weights, zero bias (float64)."""
    rng = np.random.default_rng(seed)
    return {name: (rng.normal(0, np.sqrt(2.0 / (9 * cin)), (9, cout, cin)), np.zeros(cout))
            for name, cin, cout, _ in LAYERS}
