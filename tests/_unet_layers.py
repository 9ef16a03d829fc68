"""The warm-start U-Net sequenced layer by layer from Python over the library's layer kernels
(test infrastructure): it keeps every activation and, on request, every activation gradient, so
that tests can check each layer against the FP64 reference on the GPU's own inputs.  The product
path is the library's own network object (ws_net_*), which runs the same kernel sequence."""
from __future__ import annotations

import ctypes
import math

import torch

from paper_2305_06482_gb300 import _check, _ptr, _stream, lib
from paper_2305_06482_gb300.warmstart import WIDTHS


def _kpad(k):
    return ((k + 15) // 16) * 16


def _npad(n):
    for v in (16, 32, 64):
        if n <= v:
            return v
    raise ValueError(f"{n} channels exceed the tensor-core tile (64)")


def unet_layers(c1, c2, c3):
    """(parameter index, kind, cin, cout) of the U-Net's layers; kinds 'conv' (3x3x3), 'up'
    (2x2x2 stride-2 transposed), 'out' (1x1x1).  Parameters come in (w, b) pairs."""
    return [(0, "conv", 4, c1), (2, "conv", c1, c1), (4, "conv", c1, c2), (6, "conv", c2, c2),
            (8, "conv", c2, c3), (10, "conv", c3, c3), (12, "up", c3, c2), (14, "conv", 2 * c2, c2),
            (16, "conv", c2, c2), (18, "up", c2, c1), (20, "conv", 2 * c1, c1), (22, "conv", c1, c1),
            (24, "out", c1, 2)]


class LayeredUNet:
    """The warm-start U-Net: 3 levels of c1/c2/c3 channels (two 3x3x3 convolutions with ReLU per
    level, 2x2x2 max-pools down, 2x2x2 stride-2 transposed convolutions up, skip concatenation
    [up-path, encoder]) and a 1x1x1 output layer to 2 channels; ~0.34 M weights at 16/32/64.
    Parameters: for each layer of unet_layers, w ([cout][27][cin], [cout][8][cin] or [2][c1])
    and b [cout].  Volume sizes must be divisible by 4."""

    def __init__(self, seed=0, device="cuda", widths=WIDTHS):
        g = torch.Generator().manual_seed(seed)
        self.device = torch.device(device)
        self.widths = tuple(widths)
        self.layers = unet_layers(*self.widths)
        self.params = []
        for _, kind, cin, cout in self.layers:
            if kind == "conv":
                w = torch.randn((cout, 27, cin), generator=g) * math.sqrt(2.0 / (27 * cin))
            elif kind == "up":
                w = torch.randn((cout, 8, cin), generator=g) * math.sqrt(1.0 / cin)
            else:
                w = torch.randn((cout, cin), generator=g) * math.sqrt(1.0 / cin) * 0.1
            self.params.append(w.to(self.device))
            self.params.append(torch.zeros(cout, device=self.device))
        self.grads = [torch.zeros_like(p) for p in self.params]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.step_count = 0
        self._packed = None

    # ---- weights of the 3x3x3 layers in the tensor-core layout (forward and transposed) ----
    def pack(self, stream=None):
        packed = {}
        for pi, kind, cin, cout in self.layers:
            if kind != "conv":
                continue
            w = self.params[pi]
            fw = torch.empty((_npad(cout), _kpad(27 * cin)), dtype=torch.int16, device=self.device)
            _check(lib().cs_nn_pack_weights(_ptr(w), cout, cin, 0, _ptr(fw), fw.shape[0], fw.shape[1], _stream(stream)))
            tw = None
            if pi > 0:
                tw = torch.empty((_npad(cin), _kpad(27 * cout)), dtype=torch.int16, device=self.device)
                _check(lib().cs_nn_pack_weights(_ptr(w), cout, cin, 1, _ptr(tw), tw.shape[0], tw.shape[1],
                                                _stream(stream)))
            packed[pi] = (fw, tw)
        self._packed = packed

    def _conv(self, x, dims, pi, cin, cout, stream, out=None, ldo=None, coff=0):
        nz, ny, nx = dims
        fw, _ = self._packed[pi]
        if out is None:
            out = torch.empty((nz * ny * nx, cout), dtype=torch.float32, device=self.device)
            ldo = cout
        _check(lib().cs_nn_conv3d(_ptr(x), nz, ny, nx, cin, _ptr(fw), fw.shape[0], fw.shape[1], cout,
                                  _ptr(self.params[pi + 1]), 1, 0, _ptr(out), ldo, coff, _stream(stream)))
        return out

    def _dgrad(self, g, dims, pi, cin, cout, stream):
        nz, ny, nx = dims
        _, tw = self._packed[pi]
        gin = torch.empty((nz * ny * nx, cin), dtype=torch.float32, device=self.device)
        _check(lib().cs_nn_conv3d(_ptr(g), nz, ny, nx, cout, _ptr(tw), tw.shape[0], tw.shape[1], cin, None, 0, 1,
                                  _ptr(gin), cin, 0, _stream(stream)))
        return gin

    def _pool(self, x, dims, C, stream):
        nz, ny, nx = (d // 2 for d in dims)
        out = torch.empty((nz * ny * nx, C), dtype=torch.float32, device=self.device)
        idx = torch.empty((nz * ny * nx, C), dtype=torch.uint8, device=self.device)
        _check(lib().cs_nn_maxpool2(_ptr(x), nz, ny, nx, C, _ptr(out), _ptr(idx), _stream(stream)))
        return out, idx

    def _up(self, x, cdims, pi, cin, cout, out, ldo, stream):
        nz, ny, nx = cdims
        _check(lib().cs_nn_upconv2(_ptr(x), nz, ny, nx, cin, _ptr(self.params[pi]), _ptr(self.params[pi + 1]), cout,
                                   _ptr(out), ldo, 0, _stream(stream)))

    def _slice(self, src, lds, soff, n, dst, ldd, doff, nvox, acc, stream):
        _check(lib().cs_nn_slice(_ptr(src), lds, soff, n, _ptr(dst), ldd, doff, nvox, int(acc), _stream(stream)))

    def forward(self, feat, dims, stream=None, keep=False):
        """feat [V][4] -> out [V][2]; keeps the activations for backward when keep=True."""
        if self._packed is None:
            self.pack(stream)
        c1, c2, c3 = self.widths
        d1 = tuple(dims)
        d2 = tuple(v // 2 for v in d1)
        d3 = tuple(v // 2 for v in d2)
        if any(v % 4 for v in d1):
            raise ValueError(f"U-Net volume sizes must be divisible by 4, got {d1}")
        V1, V2 = d1[0] * d1[1] * d1[2], d2[0] * d2[1] * d2[2]
        a = {"f": feat}
        a["e1a"] = self._conv(feat, d1, 0, 4, c1, stream)
        a["e1"] = self._conv(a["e1a"], d1, 2, c1, c1, stream)
        a["p1"], a["i1"] = self._pool(a["e1"], d1, c1, stream)
        a["e2a"] = self._conv(a["p1"], d2, 4, c1, c2, stream)
        a["e2"] = self._conv(a["e2a"], d2, 6, c2, c2, stream)
        a["p2"], a["i2"] = self._pool(a["e2"], d2, c2, stream)
        a["b1"] = self._conv(a["p2"], d3, 8, c2, c3, stream)
        a["b2"] = self._conv(a["b1"], d3, 10, c3, c3, stream)
        a["cat2"] = torch.empty((V2, 2 * c2), dtype=torch.float32, device=self.device)
        self._up(a["b2"], d3, 12, c3, c2, a["cat2"], 2 * c2, stream)
        self._slice(a["e2"], c2, 0, c2, a["cat2"], 2 * c2, c2, V2, False, stream)
        a["d2a"] = self._conv(a["cat2"], d2, 14, 2 * c2, c2, stream)
        a["d2"] = self._conv(a["d2a"], d2, 16, c2, c2, stream)
        a["cat1"] = torch.empty((V1, 2 * c1), dtype=torch.float32, device=self.device)
        self._up(a["d2"], d2, 18, c2, c1, a["cat1"], 2 * c1, stream)
        self._slice(a["e1"], c1, 0, c1, a["cat1"], 2 * c1, c1, V1, False, stream)
        a["d1a"] = self._conv(a["cat1"], d1, 20, 2 * c1, c1, stream)
        a["d1"] = self._conv(a["d1a"], d1, 22, c1, c1, stream)
        y = torch.empty((V1, 2), dtype=torch.float32, device=self.device)
        _check(lib().cs_nn_conv1(_ptr(a["d1"]), V1, c1, 2, _ptr(self.params[24]), _ptr(self.params[25]), _ptr(y),
                                 _stream(stream)))
        if keep:
            self._acts = a
        return y

    def backward(self, gout, dims, stream=None, keep=False):
        """Parameter gradients for dL/dout = gout [V][2] (after forward(keep=True)).  With keep,
        copies of the activation gradients are kept per layer: _gup[pi] (w.r.t. the layer's
        output), _gz[pi] (after the ReLU mask), _gx[pi] (w.r.t. its input), _gx['e2'/'e1'] (w.r.t.
        the pooled encoder outputs, routed plus skip)."""
        c1, c2, c3 = self.widths
        d1 = tuple(dims)
        d2 = tuple(v // 2 for v in d1)
        d3 = tuple(v // 2 for v in d2)
        V1, V2, V3 = d1[0] * d1[1] * d1[2], d2[0] * d2[1] * d2[2], d3[0] * d3[1] * d3[2]
        a, G = self._acts, self.grads
        for g in G:
            g.zero_()
        L = lib()
        st = _stream(stream)

        self._gup, self._gz, self._gx = {}, {}, {}

        def conv_back(g, act_out, act_in, dims, pi, cin, cout, need_gin=True):
            n = dims[0] * dims[1] * dims[2]
            if keep:
                self._gup[pi] = g.clone()
            _check(L.cs_nn_relu_bwd(_ptr(act_out), _ptr(g), n * cout, st))
            if keep:
                self._gz[pi] = g.clone()
            _check(L.cs_nn_conv3d_wgrad(_ptr(act_in), _ptr(g), dims[0], dims[1], dims[2], cin, cout, _ptr(G[pi]),
                                        _ptr(G[pi + 1]), st))
            if not need_gin:
                return None
            gin = self._dgrad(g, dims, pi, cin, cout, stream)
            if keep:
                self._gx[pi] = gin.clone()
            return gin

        def up_back(x, cdims, pi, cin, cout, gcat, ldg):
            n = cdims[0] * cdims[1] * cdims[2]
            gin = torch.empty((n, cin), dtype=torch.float32, device=self.device)
            _check(L.cs_nn_upconv2_bwd(_ptr(x), _ptr(gcat), ldg, 0, cdims[0], cdims[1], cdims[2], cin,
                                       _ptr(self.params[pi]), cout, _ptr(gin), _ptr(G[pi]), _ptr(G[pi + 1]), st))
            if keep:
                self._gx[pi] = gin.clone()
            return gin

        g = torch.empty((V1, c1), dtype=torch.float32, device=self.device)
        _check(L.cs_nn_conv1_bwd(_ptr(a["d1"]), _ptr(gout), V1, c1, 2, _ptr(self.params[24]), _ptr(g), _ptr(G[24]),
                                 _ptr(G[25]), st))
        if keep:
            self._gx[24] = g.clone()
        g = conv_back(g, a["d1"], a["d1a"], d1, 22, c1, c1)
        gcat1 = conv_back(g, a["d1a"], a["cat1"], d1, 20, 2 * c1, c1)
        g = up_back(a["d2"], d2, 18, c2, c1, gcat1, 2 * c1)
        g = conv_back(g, a["d2"], a["d2a"], d2, 16, c2, c2)
        gcat2 = conv_back(g, a["d2a"], a["cat2"], d2, 14, 2 * c2, c2)
        g = up_back(a["b2"], d3, 12, c3, c2, gcat2, 2 * c2)
        g = conv_back(g, a["b2"], a["b1"], d3, 10, c3, c3)
        g = conv_back(g, a["b1"], a["p2"], d3, 8, c2, c3)
        ge2 = torch.empty((V2, c2), dtype=torch.float32, device=self.device)
        _check(L.cs_nn_maxpool2_bwd(_ptr(g), _ptr(a["i2"]), d3[0], d3[1], d3[2], c2, _ptr(ge2), st))
        self._slice(gcat2, 2 * c2, c2, c2, ge2, c2, 0, V2, True, stream)
        if keep:
            self._gx["e2"] = ge2.clone()
        g = conv_back(ge2, a["e2"], a["e2a"], d2, 6, c2, c2)
        g = conv_back(g, a["e2a"], a["p1"], d2, 4, c1, c2)
        ge1 = torch.empty((V1, c1), dtype=torch.float32, device=self.device)
        _check(L.cs_nn_maxpool2_bwd(_ptr(g), _ptr(a["i1"]), d2[0], d2[1], d2[2], c1, _ptr(ge1), st))
        self._slice(gcat1, 2 * c1, c1, c1, ge1, c1, 0, V1, True, stream)
        if keep:
            self._gx["e1"] = ge1.clone()
        g = conv_back(ge1, a["e1"], a["e1a"], d1, 2, c1, c1)
        conv_back(g, a["e1a"], a["f"], d1, 0, 4, c1, need_gin=False)

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
