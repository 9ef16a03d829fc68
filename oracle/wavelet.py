"""Periodised orthonormal Daubechies wavelet transform for the l1-wavelet regulariser
g(x) = lambda ||Psi x||_1 with Psi unitary (Sec. 2.1; Daubechies 4 in Sec. 3.3).

Reading: "Daubechies 4" is db4 in the PyWavelets sense (4 vanishing moments, 8 taps).  The
filter is derived here from Daubechies' construction: |m0(xi)|^2 = cos^8(xi/2) P(sin^2(xi/2))
with P(y) = sum_{k<4} binom(3+k, k) y^k, factorised by keeping the roots inside the unit
circle (minimum phase).  Periodic extension makes every level an orthogonal map, so Psi is
unitary.  Conventions (fixed, shared with the GPU by specification, not by code):

  a[k] = sum_m h[m] x[(2k+m) mod n],  d[k] = sum_m g[m] x[(2k+m) mod n],  g[m] = (-1)^m h[7-m],
  coefficients stored as [a | d] along the axis; separable over all axes (x, then y, then z);
  ``levels`` levels applied to the low-pass corner block; complex data -> real filters on the
  real and imaginary parts; soft threshold soft(z, tau) = z max(0, 1 - tau/|z|) on every
  coefficient (approximation included).
"""
from __future__ import annotations

from math import comb

import numpy as np


def db_filter(N=4):
    """Daubechies scaling filter h (length 2N, sum sqrt(2)), minimum phase."""
    # P(y) coefficients, y = sin^2(xi/2) = (2 - z - 1/z)/4
    P = [comb(N - 1 + k, k) for k in range(N)]
    yroots = np.roots(P[::-1]) if N > 1 else np.array([])
    zroots = []
    for yr in yroots:
        # (2 - z - 1/z)/4 = yr  <=>  z^2 - (2 - 4 yr) z + 1 = 0
        zs = np.roots([1.0, -(2.0 - 4.0 * yr), 1.0])
        zroots.append(zs[np.argmin(np.abs(zs))])
    q = np.real(np.poly(zroots)) if zroots else np.array([1.0])
    h = np.array([1.0])
    for _ in range(N):
        h = np.convolve(h, [1.0, 1.0])
    h = np.convolve(h, q)
    h = h * np.sqrt(2.0) / h.sum()
    # orient so that the energy sits at the start (the usual reconstruction-lowpass layout)
    if np.abs(h[: len(h) // 2]).sum() < np.abs(h[len(h) // 2:]).sum():
        h = h[::-1]
    return h


H = db_filter(4)
G = np.array([(-1) ** m * H[len(H) - 1 - m] for m in range(len(H))])


def dwt1(x, axis):
    """One analysis level along ``axis`` (length n even): returns [a | d] along that axis."""
    x = np.moveaxis(np.asarray(x), axis, -1)
    n = x.shape[-1]
    k = np.arange(n // 2)
    a = np.zeros(x.shape[:-1] + (n // 2,), dtype=np.result_type(x, np.float64))
    d = np.zeros_like(a)
    for m in range(len(H)):
        xm = x[..., (2 * k + m) % n]
        a = a + H[m] * xm
        d = d + G[m] * xm
    return np.moveaxis(np.concatenate([a, d], axis=-1), -1, axis)


def idwt1(c, axis):
    """Inverse (= transpose) of dwt1."""
    c = np.moveaxis(np.asarray(c), axis, -1)
    n = c.shape[-1]
    a, d = c[..., : n // 2], c[..., n // 2:]
    x = np.zeros(c.shape, dtype=np.result_type(c, np.float64))
    k = np.arange(n // 2)
    for m in range(len(H)):
        idx = (2 * k + m) % n
        x[..., idx] += H[m] * a + G[m] * d
    return np.moveaxis(x, -1, axis)


def wavedec(x, levels=4):
    """Multi-level separable periodised DWT (Mallat corner layout), same shape as x."""
    c = np.array(x, dtype=np.complex128, copy=True)
    nd = c.ndim
    for lev in range(levels):
        sl = tuple(slice(0, s >> lev) for s in c.shape)
        blk = c[sl]
        for ax in range(nd - 1, -1, -1):   # x (last axis) first
            blk = dwt1(blk, ax)
        c[sl] = blk
    return c


def waverec(c, levels=4):
    """Inverse of wavedec."""
    x = np.array(c, dtype=np.complex128, copy=True)
    nd = x.ndim
    for lev in range(levels - 1, -1, -1):
        sl = tuple(slice(0, s >> lev) for s in x.shape)
        blk = x[sl]
        for ax in range(nd):               # reverse order of wavedec
            blk = idwt1(blk, ax)
        x[sl] = blk
    return x


def soft_threshold(z, tau):
    """soft(z, tau) = z * max(0, 1 - tau/|z|), 0 where z = 0."""
    z = np.asarray(z)
    mag = np.abs(z)
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.where(mag > 0, np.maximum(0.0, 1.0 - tau / np.where(mag > 0, mag, 1.0)), 0.0)
    return z * scale


def prox_l1_wavelet(v, tau, levels=4):
    """prox of tau ||Psi x||_1 for unitary Psi: Psi^H soft(Psi v, tau)."""
    return waverec(soft_threshold(wavedec(v, levels), tau), levels)
