"""FP64 reference of the warm-start network (test infrastructure; not part of the paper's method):
the 3x3x3 convolution and its gradients, a small plain CNN, and the 3-level U-Net (max-pools,
stride-2 transposed convolutions, skip concatenation) built from them.

Activations are [nz, ny, nx, C]; a 3x3x3 convolution with zero padding 1 computes
    out[v, co] = b[co] + sum_{tap, ci} x[v + off(tap), ci] w[co, tap, ci],
tap = 9 (dz+1) + 3 (dy+1) + (dx+1).  With bf16=True the convolution's input and weights are first
rounded to the nearest bfloat16 (the operands the tensor cores see) and the sum is exact in FP64.
"""
from __future__ import annotations

import numpy as np

from .philox import round_to_bf16


def _r(a, bf16):
    return round_to_bf16(np.asarray(a, np.float32)).astype(np.float64) if bf16 else np.asarray(a, np.float64)


def taps():
    return [(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1) for t in range(27)]


def conv3d(x, w, b, bf16=False):
    x = _r(x, bf16)
    w = _r(w, bf16)
    nz, ny, nx, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((nz, ny, nx, w.shape[0])) + (0 if b is None else np.asarray(b, np.float64))
    for t, (dz, dy, dx) in enumerate(taps()):
        sl = xp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        out += sl @ w[:, t, :].T
    return out


def conv3d_bwd(x, w, gout, bf16=False):
    """(gx, gw, gb) of conv3d.  With bf16=True both products see BF16 operands, as the tensor-core
    kernels do: gx the rounded weights and gout (the data-gradient convolution), gw the rounded
    input and gout (the weight-gradient implicit GEMM); gb sums the unrounded gout."""
    nz, ny, nx, cin = x.shape
    wr = _r(w, bf16)
    gr = _r(gout, bf16)
    gxp = np.zeros((nz + 2, ny + 2, nx + 2, cin))
    xp = np.pad(_r(x, bf16), ((1, 1), (1, 1), (1, 1), (0, 0)))
    gw = np.zeros_like(np.asarray(w, np.float64))
    g64 = np.asarray(gout, np.float64)
    for t, (dz, dy, dx) in enumerate(taps()):
        sl = xp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        gw[:, t, :] = np.einsum("zyxo,zyxc->oc", gr, sl)
        gxp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx] += gr @ wr[:, t, :]
    return gxp[1:-1, 1:-1, 1:-1], gw, g64.sum(axis=(0, 1, 2))


def forward(params, f, bf16=False):
    """params = [w1, b1, w2, b2, w3, b3, w4, b4]; f [nz, ny, nx, 4] -> (out [.., 2], activations)."""
    acts = [np.asarray(f, np.float64)]
    cur = acts[0]
    for li in range(3):
        cur = np.maximum(conv3d(cur, params[2 * li], params[2 * li + 1], bf16), 0.0)
        acts.append(cur)
    out = cur @ np.asarray(params[6], np.float64).T + np.asarray(params[7], np.float64)
    return out, acts


def backward(params, acts, gout, bf16=False):
    grads = [None] * 8
    g = np.asarray(gout, np.float64)
    grads[6] = np.einsum("zyxo,zyxc->oc", g, acts[3])
    grads[7] = g.sum(axis=(0, 1, 2))
    gcur = g @ np.asarray(params[6], np.float64)
    for li in range(2, -1, -1):
        gcur = gcur * (acts[li + 1] > 0)
        gx, gw, gb = conv3d_bwd(acts[li], params[2 * li], gcur, bf16)
        grads[2 * li], grads[2 * li + 1] = gw, gb
        gcur = gx
    return grads


def mse(out, tgt):
    d = np.asarray(out, np.float64) - np.asarray(tgt, np.float64)
    n = d.size
    return float((d * d).sum() / n), 2.0 * d / n


# ---------------------------------------------------------------------------------------------
# 3-level U-Net (widths c1/c2/c3, two 2x2x2 max-pools, two 2x2x2 stride-2 transposed
# convolutions, skip concatenation [up-path channels, encoder channels], two 3x3x3 convolutions
# with ReLU per level, a 1x1x1 output layer to 2 channels).  Parameter list order:
#   e1a, e1b, e2a, e2b, b1, b2 (3x3x3 w [cout, 27, cin], b), u2 (transposed w [cout, 8, cin], b),
#   d2a, d2b (3x3x3), u1 (transposed), d1a, d1b (3x3x3), out (w [2, c1], b)   -> 26 arrays.

def sub8():
    """child offsets (dz, dy, dx) of a 2x2x2 block, child index a = 4 dz + 2 dy + dx."""
    return [(a // 4, (a // 2) % 2, a % 2) for a in range(8)]


def maxpool2(x, idx=None):
    """2x2x2 max-pool; the argmax index per output is the first maximal child in the order of
    sub8().  With idx given, the children idx are taken instead (a decision made elsewhere)."""
    x = np.asarray(x, np.float64)
    nz, ny, nx, c = x.shape
    kids = np.stack([x[dz::2, dy::2, dx::2] for dz, dy, dx in sub8()])   # [8, nz/2, ny/2, nx/2, c]
    if idx is None:
        idx = np.argmax(kids, axis=0)          # first maximum on ties
    out = np.take_along_axis(kids, idx[None], axis=0)[0]
    return out, idx


def maxpool2_bwd(g, idx, shape):
    gin = np.zeros(shape)
    g = np.asarray(g, np.float64)
    for a, (dz, dy, dx) in enumerate(sub8()):
        gin[dz::2, dy::2, dx::2] = np.where(idx == a, g, 0.0)
    return gin


def upconv2(x, w, b):
    """Transposed convolution, kernel 2, stride 2: out[2v + sub(a), co] = b[co] + sum_ci x[v, ci] w[co, a, ci]."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    nz, ny, nx, _ = x.shape
    out = np.zeros((2 * nz, 2 * ny, 2 * nx, w.shape[0])) + np.asarray(b, np.float64)
    for a, (dz, dy, dx) in enumerate(sub8()):
        out[dz::2, dy::2, dx::2] += x @ w[:, a, :].T
    return out


def upconv2_bwd(x, w, gout):
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    g = np.asarray(gout, np.float64)
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for a, (dz, dy, dx) in enumerate(sub8()):
        ga = g[dz::2, dy::2, dx::2]
        gx += ga @ w[:, a, :]
        gw[:, a, :] = np.einsum("zyxo,zyxc->oc", ga, x)
    return gx, gw, g.sum(axis=(0, 1, 2))


def unet_forward(params, f, bf16=False, pool_idx=None):
    """params: the 26 arrays above; f [nz, ny, nx, 4] (sizes divisible by 4) -> (out [.., 2], cache).
    pool_idx: optional (idx1, idx2) argmax decisions of the two pools."""
    P = [np.asarray(p, np.float64) for p in params]
    relu = lambda v: np.maximum(v, 0.0)
    c = {"f": np.asarray(f, np.float64)}
    c["e1a"] = relu(conv3d(c["f"], P[0], P[1], bf16))
    c["e1"] = relu(conv3d(c["e1a"], P[2], P[3], bf16))
    c["p1"], c["i1"] = maxpool2(c["e1"], None if pool_idx is None else pool_idx[0])
    c["e2a"] = relu(conv3d(c["p1"], P[4], P[5], bf16))
    c["e2"] = relu(conv3d(c["e2a"], P[6], P[7], bf16))
    c["p2"], c["i2"] = maxpool2(c["e2"], None if pool_idx is None else pool_idx[1])
    c["b1"] = relu(conv3d(c["p2"], P[8], P[9], bf16))
    c["b2"] = relu(conv3d(c["b1"], P[10], P[11], bf16))
    c["cat2"] = np.concatenate([upconv2(c["b2"], P[12], P[13]), c["e2"]], axis=-1)
    c["d2a"] = relu(conv3d(c["cat2"], P[14], P[15], bf16))
    c["d2"] = relu(conv3d(c["d2a"], P[16], P[17], bf16))
    c["cat1"] = np.concatenate([upconv2(c["d2"], P[18], P[19]), c["e1"]], axis=-1)
    c["d1a"] = relu(conv3d(c["cat1"], P[20], P[21], bf16))
    c["d1"] = relu(conv3d(c["d1a"], P[22], P[23], bf16))
    out = c["d1"] @ P[24].T + P[25]
    return out, c


def unet_backward(params, c, gout, bf16=False):
    P = [np.asarray(p, np.float64) for p in params]
    G = [None] * 26
    g = np.asarray(gout, np.float64)
    G[24] = np.einsum("zyxo,zyxc->oc", g, c["d1"])
    G[25] = g.sum(axis=(0, 1, 2))
    g = g @ P[24]

    def conv_back(g, act_out, act_in, wi):
        g = g * (act_out > 0)
        gx, G[wi], G[wi + 1] = conv3d_bwd(act_in, P[wi], g, bf16)
        return gx

    g = conv_back(g, c["d1"], c["d1a"], 22)
    gcat1 = conv_back(g, c["d1a"], c["cat1"], 20)
    c1 = P[18].shape[0]
    g, G[18], G[19] = upconv2_bwd(c["d2"], P[18], gcat1[..., :c1])
    g_e1_skip = gcat1[..., c1:]
    g = conv_back(g, c["d2"], c["d2a"], 16)
    gcat2 = conv_back(g, c["d2a"], c["cat2"], 14)
    c2 = P[12].shape[0]
    g, G[12], G[13] = upconv2_bwd(c["b2"], P[12], gcat2[..., :c2])
    g_e2_skip = gcat2[..., c2:]
    g = conv_back(g, c["b2"], c["b1"], 10)
    g = conv_back(g, c["b1"], c["p2"], 8)
    g = maxpool2_bwd(g, c["i2"], c["e2"].shape) + g_e2_skip
    g = conv_back(g, c["e2"], c["e2a"], 6)
    g = conv_back(g, c["e2a"], c["p1"], 4)
    g = maxpool2_bwd(g, c["i1"], c["e1"].shape) + g_e1_skip
    g = conv_back(g, c["e1"], c["e1a"], 2)
    conv_back(g, c["e1a"], c["f"], 0)
    return G


def unet_shapes(c1=16, c2=32, c3=64):
    """Shapes of the 26 parameters for widths c1/c2/c3 (input 4 channels, output 2)."""
    conv = lambda ci, co: [(co, 27, ci), (co,)]
    up = lambda ci, co: [(co, 8, ci), (co,)]
    return (conv(4, c1) + conv(c1, c1) + conv(c1, c2) + conv(c2, c2) + conv(c2, c3) + conv(c3, c3) +
            up(c3, c2) + conv(2 * c2, c2) + conv(c2, c2) + up(c2, c1) + conv(2 * c1, c1) + conv(c1, c1) +
            [(2, c1), (2,)])
