"""FP64 reference of the warm-start network (test infrastructure; not part of the paper's method).

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
    """(gx, gw, gb) of conv3d.  gx uses the rounded weights and gout (as the data-gradient
    convolution does); gw uses the FP32 input and gradient (computed on CUDA cores)."""
    nz, ny, nx, cin = x.shape
    wr = _r(w, bf16)
    gr = _r(gout, bf16)
    gxp = np.zeros((nz + 2, ny + 2, nx + 2, cin))
    xp = np.pad(np.asarray(x, np.float64), ((1, 1), (1, 1), (1, 1), (0, 0)))
    gw = np.zeros_like(np.asarray(w, np.float64))
    g64 = np.asarray(gout, np.float64)
    for t, (dz, dy, dx) in enumerate(taps()):
        sl = xp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        gw[:, t, :] = np.einsum("zyxo,zyxc->oc", g64, sl)
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
