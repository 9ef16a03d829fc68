"""Learned warm start for the sketched sub-problems (not part of the paper's method).

A small 3D CNN maps the sub-problem's (x^t, d) - normalised by s, the RMS of (x^t, eta d) with
eta the FISTA step - to a correction of x^t; x^t + s * net(.) starts the sub-problem's solver only
when the sub-problem objective (Eq. 9-10) is lower there than at x^t, otherwise the solver
starts from x^t as in Algorithm 1.  Network: three 3x3x3 convolutions 4 -> 16 -> 16 -> 16 with
ReLU (BF16 implicit GEMMs on the tensor cores, FP32 accumulation) and a 1x1x1 layer 16 -> 2.
Every forward, backward and optimiser step runs in the library's kernels; this module only
holds the parameters (torch tensors as storage) and sequences the calls.

Training pairs come from the method itself on seeded synthetic phantoms: at each outer
iteration the input is (x^t, d) and the target is the sub-problem solved tightly (many more
inner iterations) from x^t.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import torch

from . import (CoilSketchError, Plan, REG_L1_WAVELET, _check, _ptr, _stream, coil_pca, coil_rotate, lib,
               sense_grad, sketch_draw, sketched_maps, sketched_subproblem_solve, subproblem_objective,
               power_iteration, PREC_FP32)

CH = 16
LAYERS = [(4, CH), (CH, CH), (CH, CH)]   # 3x3x3 convolutions (cin, cout)


def _kpad(k):
    return ((k + 15) // 16) * 16


class WarmNet:
    """Parameters: w_l [cout][27][cin], b_l [cout] for the three 3x3x3 layers, w4 [2][16], b4 [2]."""

    def __init__(self, seed=0, device="cuda"):
        g = torch.Generator().manual_seed(seed)
        self.device = torch.device(device)
        self.params = []
        for cin, cout in LAYERS:
            std = math.sqrt(2.0 / (27 * cin))
            self.params.append((torch.randn((cout, 27, cin), generator=g) * std).to(self.device))
            self.params.append(torch.zeros(cout, device=self.device))
        self.params.append((torch.randn((2, CH), generator=g) * math.sqrt(1.0 / CH) * 0.1).to(self.device))
        self.params.append(torch.zeros(2, device=self.device))
        self.grads = [torch.zeros_like(p) for p in self.params]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.step_count = 0
        self._packed = None

    # ---- weights in the tensor-core layout ----
    def pack(self, stream=None):
        packed = []
        for li, (cin, cout) in enumerate(LAYERS):
            w = self.params[2 * li]
            fw = torch.empty((16, _kpad(27 * cin)), dtype=torch.int16, device=self.device)
            _check(lib().cs_nn_pack_weights(_ptr(w), cout, cin, 0, _ptr(fw), 16, fw.shape[1], _stream(stream)))
            tw = torch.empty((16, _kpad(27 * cout)), dtype=torch.int16, device=self.device)
            _check(lib().cs_nn_pack_weights(_ptr(w), cout, cin, 1, _ptr(tw), 16, tw.shape[1], _stream(stream)))
            packed.append((fw, tw))
        self._packed = packed

    def forward(self, feat, dims, stream=None, keep=False):
        """feat [V][4] -> out [V][2]; keeps the activations for backward when keep=True."""
        if self._packed is None:
            self.pack(stream)
        nz, ny, nx = dims
        V = nz * ny * nx
        acts = [feat]
        cur = feat
        for li, (cin, cout) in enumerate(LAYERS):
            fw, _ = self._packed[li]
            out = torch.empty((V, cout), dtype=torch.float32, device=self.device)
            _check(lib().cs_nn_conv3d(_ptr(cur), nz, ny, nx, cin, _ptr(fw), 16, fw.shape[1], cout,
                                      _ptr(self.params[2 * li + 1]), 1, 0, _ptr(out), cout, 0, _stream(stream)))
            acts.append(out)
            cur = out
        y = torch.empty((V, 2), dtype=torch.float32, device=self.device)
        _check(lib().cs_nn_conv1(_ptr(cur), V, CH, 2, _ptr(self.params[6]), _ptr(self.params[7]), _ptr(y),
                                 _stream(stream)))
        if keep:
            self._acts = acts
        return y

    def backward(self, gout, dims, stream=None):
        """Accumulate parameter gradients for dL/dout = gout [V][2] (after forward(keep=True))."""
        nz, ny, nx = dims
        V = nz * ny * nx
        for g in self.grads:
            g.zero_()
        acts = self._acts
        g3 = torch.empty((V, CH), dtype=torch.float32, device=self.device)
        _check(lib().cs_nn_conv1_bwd(_ptr(acts[3]), _ptr(gout), V, CH, 2, _ptr(self.params[6]), _ptr(g3),
                                     _ptr(self.grads[6]), _ptr(self.grads[7]), _stream(stream)))
        gcur = g3
        for li in range(len(LAYERS) - 1, -1, -1):
            cin, cout = LAYERS[li]
            _check(lib().cs_nn_relu_bwd(_ptr(acts[li + 1]), _ptr(gcur), V * cout, _stream(stream)))
            _check(lib().cs_nn_conv3d_wgrad(_ptr(acts[li]), _ptr(gcur), nz, ny, nx, cin, cout,
                                            _ptr(self.grads[2 * li]), _ptr(self.grads[2 * li + 1]), _stream(stream)))
            if li > 0:
                _, tw = self._packed[li]
                gin = torch.empty((V, cin), dtype=torch.float32, device=self.device)
                _check(lib().cs_nn_conv3d(_ptr(gcur), nz, ny, nx, cout, _ptr(tw), 16, tw.shape[1], cin, None, 0, 1,
                                          _ptr(gin), cin, 0, _stream(stream)))
                gcur = gin

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        self.step_count += 1
        for p, g, m, v in zip(self.params, self.grads, self.m, self.v):
            _check(lib().cs_nn_adam(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), ctypes.c_float(lr),
                                    ctypes.c_float(b1), ctypes.c_float(b2), ctypes.c_float(eps), self.step_count,
                                    _stream(stream)))
        self._packed = None

    def loss_and_grad(self, out, tgt, stream=None):
        g = torch.empty_like(out)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        _check(lib().cs_nn_mse(_ptr(out), _ptr(tgt), out.numel(), _ptr(g), _ptr(loss), _stream(stream)))
        return loss, g


def features(xt, d, eta, stream=None):
    n = xt.numel()
    ss = torch.empty(1, dtype=torch.float32, device=xt.device)
    f = torch.empty((n, 4), dtype=torch.float32, device=xt.device)
    _check(lib().cs_nn_features(_ptr(xt), _ptr(d), n, ctypes.c_float(eta), _ptr(ss), _ptr(f), _stream(stream)))
    return f, ss


def target(xt, xs, ss, stream=None):
    n = xt.numel()
    tgt = torch.empty((n, 2), dtype=torch.float32, device=xt.device)
    _check(lib().cs_nn_target(_ptr(xt), _ptr(xs), n, _ptr(ss), _ptr(tgt), _stream(stream)))
    return tgt


def apply(xt, delta, ss, stream=None):
    out = torch.empty_like(xt)
    _check(lib().cs_nn_apply(_ptr(xt), _ptr(delta), xt.numel(), _ptr(ss), _ptr(out), _stream(stream)))
    return out


@dataclass
class SketchSetup:
    plan: Plan
    y_r: torch.Tensor
    maps_r: torch.Tensor
    sketches: torch.Tensor
    eta: float
    V: int
    S: int
    lam: float
    levels: int


def setup(plan, y, maps, lam, V, S, T, seed, power_v0, levels):
    """Coil PCA + rotation, sketch draws and the FISTA step of the first sub-problem."""
    U, _ = coil_pca(y)
    y_r = coil_rotate(U, y)
    maps_r = coil_rotate(U, maps)
    C = maps.shape[0]
    sk = sketch_draw(seed, 0, T, C, V, S)
    ms0 = sketched_maps(sk[0].contiguous(), maps_r, V)
    L = power_iteration(plan, power_v0, maps_r[:V], ms0, 20)
    return SketchSetup(plan, y_r, maps_r, sk, 1.0 / L, V, S, lam, levels)


def run(su: SketchSetup, T, K, net: Optional[WarmNet] = None, x0=None, record_pairs=0, tight_K=40, callback=None):
    """Algorithm 1 with FISTA sub-problems, optionally warm-started by `net`; with record_pairs
    the training pairs (features, target) of every outer iteration are returned as well."""
    p = su.plan
    dims = p.img
    x = torch.zeros(dims, dtype=torch.complex64, device=su.y_r.device) if x0 is None else x0.clone()
    C = su.maps_r.shape[0]
    pairs, accepted = [], []
    for t in range(T):
        d = sense_grad(p, x, su.maps_r, su.y_r)
        ms = sketched_maps(su.sketches[t].contiguous(), su.maps_r, su.V)
        mv = su.maps_r[:su.V]
        xt = x.clone()
        if record_pairs:
            f, ss = features(xt, d, su.eta)
            xs = xt.clone()
            sketched_subproblem_solve(p, d, xt, xs, mv, ms, su.lam, REG_L1_WAVELET, tight_K, su.eta, su.levels)
            pairs.append((f, target(xt, xs, ss)))
        start = xt.clone()
        if net is not None:
            f, ss = features(xt, d, su.eta)
            xh = apply(xt, net.forward(f, dims), ss)
            f_hat = subproblem_objective(p, xh, xt, d, mv, ms, su.lam, REG_L1_WAVELET, su.levels)
            f_t = subproblem_objective(p, xt, xt, d, mv, ms, su.lam, REG_L1_WAVELET, su.levels)
            ok = f_hat < f_t
            accepted.append(bool(ok))
            if ok:
                start = xh
        sketched_subproblem_solve(p, d, xt, start, mv, ms, su.lam, REG_L1_WAVELET, K, su.eta, su.levels)
        x = start
        if callback is not None:
            callback(t, x)
    return x, pairs, accepted


def train(net: WarmNet, pairs, dims, steps=200, lr=1e-3, seed=0):
    """Adam on random pairs, one volume per step; returns the loss history."""
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(steps):
        f, tgt = pairs[int(rng.integers(len(pairs)))]
        out = net.forward(f, dims, keep=True)
        loss, g = net.loss_and_grad(out, tgt)
        net.backward(g, dims)
        net.adam(lr=lr)
        hist.append(float(loss.item()))
    _check(lib().cs_nn_status(_stream()))
    return hist
