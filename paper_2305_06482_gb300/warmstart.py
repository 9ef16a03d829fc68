"""Learned warm start for the sketched sub-problems (not part of the paper's method).

A 3D U-Net maps the sub-problem's (x^t, d) - normalised by s, the RMS of (x^t, eta d) with eta
the FISTA step - to a correction of x^t; x^t + s * net(.) starts the sub-problem's solver only
when the sub-problem objective (Eq. 9-10) is lower there than at x^t, otherwise the solver
starts from x^t as in Algorithm 1.  Network: 3 levels of 16/32/64 channels, two 3x3x3
convolutions with ReLU per level (BF16 implicit GEMMs on the tensor cores, FP32 accumulation),
2x2x2 max-pools, 2x2x2 stride-2 transposed convolutions and skip concatenation, and a 1x1x1
layer to 2 channels.
The network is a library object (ws_net_*): parameters, Adam state and activation buffers live
on the device, and inference and training steps run as the library's kernel sequences; this
module wraps the handle and drives Algorithm 1 around it.

Training pairs come from the method itself on seeded synthetic phantoms: at each outer
iteration the input is (x^t, d) and the target is the sub-problem solved tightly (many more
inner iterations) from x^t.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import (Plan, REG_L1_WAVELET, _check, _ptr, _stream, coil_pca, coil_rotate, lib, power_iteration,
               sense_grad, sketch_draw, sketched_maps, sketched_subproblem_solve, subproblem_objective)

WIDTHS = (16, 32, 64)     # channels of the three U-Net levels


class UNet:
    """The warm-start U-Net, a library object (ws_net_*): 3 levels of c1/c2/c3 channels (two
    3x3x3 convolutions with ReLU per level, 2x2x2 max-pools down, 2x2x2 stride-2 transposed
    convolutions up, skip concatenation [up-path, encoder]) and a 1x1x1 output layer to 2
    channels; ~0.34 M weights at 16/32/64.  Parameters, Adam state and buffers live on the
    device inside the library; volume sizes must be multiples of 4."""

    def __init__(self, seed=0, widths=WIDTHS):
        self.widths = tuple(widths)
        h = ctypes.c_void_p()
        _check(lib().ws_net_create(*self.widths, ctypes.c_uint64(seed), ctypes.byref(h)))
        self._h = h
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ws_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _dims(x):
        if x.dim() != 3 or x.dtype != torch.complex64 or not x.is_cuda:
            raise ValueError("expected a complex64 [nz, ny, nx] CUDA tensor")
        return (ctypes.c_int * 3)(*x.shape)

    def infer(self, xt, d, eta, out=None, stream=None):
        """x^t + s net([x^t / s, eta d / s]) for one volume."""
        out = torch.empty_like(xt) if out is None else out
        _check(lib().ws_net_infer(self._h, _ptr(xt), _ptr(d), self._dims(xt), ctypes.c_float(eta), _ptr(out),
                                  _stream(stream)))
        return out

    def train_step(self, xt, d, x_target, eta, lr, stream=None):
        """One Adam step towards (x_target - x^t) / s; returns the loss before the step (device)."""
        _check(lib().ws_net_train_step(self._h, _ptr(xt), _ptr(d), _ptr(x_target), self._dims(xt),
                                       ctypes.c_float(eta), ctypes.c_float(lr), _ptr(self._loss), _stream(stream)))
        return self._loss

    def param(self, index, which=0):
        """A copy of parameter `index` (which: 0 parameters, 1 gradients, 2/3 Adam moments)."""
        n = ctypes.c_int64()
        _check(lib().ws_net_param(self._h, which, index, None, None, ctypes.byref(n), _stream(None)))
        out = torch.empty(n.value, dtype=torch.float32, device="cuda")
        _check(lib().ws_net_param(self._h, which, index, None, _ptr(out), None, _stream(None)))
        return out

    def set_param(self, index, value, which=0):
        _check(lib().ws_net_param(self._h, which, index, _ptr(value.contiguous()), None, None, _stream(None)))

    def save(self, path):
        _check(lib().ws_net_save(self._h, str(path).encode()))

    def load(self, path):
        _check(lib().ws_net_load(self._h, str(path).encode()))


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


def run(su: SketchSetup, T, K, net: Optional[UNet] = None, x0=None, record_pairs=0, tight_K=40, callback=None):
    """Algorithm 1 with FISTA sub-problems, optionally warm-started by `net`; with record_pairs
    the training pairs (x^t, d, tightly solved sub-problem, eta) of every outer iteration are
    returned as well."""
    p = su.plan
    dims = p.img
    x = torch.zeros(dims, dtype=torch.complex64, device=su.y_r.device) if x0 is None else x0.clone()
    pairs, accepted = [], []
    for t in range(T):
        d = sense_grad(p, x, su.maps_r, su.y_r)
        ms = sketched_maps(su.sketches[t].contiguous(), su.maps_r, su.V)
        mv = su.maps_r[:su.V]
        xt = x.clone()
        if record_pairs:
            xs = xt.clone()
            sketched_subproblem_solve(p, d, xt, xs, mv, ms, su.lam, REG_L1_WAVELET, tight_K, su.eta, su.levels)
            pairs.append((xt.clone(), d.clone(), xs, su.eta))
        start = xt.clone()
        if net is not None:
            xh = net.infer(xt, d, su.eta)
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


def crop3d(x, origin, box, out=None, stream=None):
    """The box [origin, origin + box) of a complex64 [nz, ny, nx] CUDA volume (library kernel)."""
    out = torch.empty(tuple(box), dtype=x.dtype, device=x.device) if out is None else out
    i3 = ctypes.c_int * 3
    _check(lib().cs_crop3d(_ptr(x), i3(*x.shape), i3(*origin), i3(*box), _ptr(out), _stream(stream)))
    return out


def make_crops(pairs, n, crop, seed=0):
    """n training pairs stored as random boxes of size crop = (cz, cy, cx) of the given volume pairs
    (x^t, d, x_target, eta): pair and box origin drawn from a seeded generator, every box copied to
    its own device buffers."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        xt, d, xs, eta = pairs[int(rng.integers(len(pairs)))]
        o = [int(rng.integers(0, m - c + 1)) for m, c in zip(xt.shape, crop)]
        out.append(tuple(crop3d(a, o, crop) for a in (xt, d, xs)) + (eta,))
    return out


def train(net: UNet, pairs, steps=200, lr=1e-3, seed=0, crop=None):
    """Adam on random pairs (x^t, d, x_target, eta), one volume per step; with crop = (cz, cy, cx)
    (multiples of 4) each step uses a random box of that size from the pair's volumes.  Returns
    the loss history."""
    rng = np.random.default_rng(seed)
    hist = []
    bufs = None
    for _ in range(steps):
        xt, d, xs, eta = pairs[int(rng.integers(len(pairs)))]
        if crop is not None:
            o = [int(rng.integers(0, n - c + 1)) for n, c in zip(xt.shape, crop)]
            if bufs is None:
                bufs = [torch.empty(tuple(crop), dtype=torch.complex64, device=xt.device) for _ in range(3)]
            xt, d, xs = (crop3d(a, o, crop, out=b) for a, b in zip((xt, d, xs), bufs))
        hist.append(float(net.train_step(xt, d, xs, eta, lr).item()))
    _check(lib().cs_nn_status(_stream()))
    return hist
