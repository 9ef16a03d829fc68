"""Cartesian multicoil SENSE operator, restated from Sec. 2.1 of the paper.

Forward model (Eq. 1): k_c[i] = D^-1/2 sum_d c_c[d] x[d] exp(-i 2 pi <f_i, r_d>), with r_d the
centred integer coordinates of voxel d and f_i the sampled frequency in cycles/pixel.  The
paper prints the exponent as f_i d / N; we read it as the inner product of the frequency and
the centred voxel position (the standard unitary DFT on the image grid).  In Cartesian imaging
F~ = U F~_u (Sec. 2.1): a centred orthonormal FFT followed by the undersampling U, which keeps
the sampled grid entries in ascending row-major order.  A = F C with C the stacked diag(c_c).
"""
from __future__ import annotations

import numpy as np

from . import fftlib


def centred_fft(u, axes):
    """Centred orthonormal DFT: fftshift(fftn(ifftshift(u), norm='ortho'))."""
    return np.fft.fftshift(fftlib.fftn(np.fft.ifftshift(u, axes=axes), axes=axes, norm="ortho"), axes=axes)


def centred_ifft(k, axes):
    """Adjoint (= inverse) of centred_fft."""
    return np.fft.fftshift(fftlib.ifftn(np.fft.ifftshift(k, axes=axes), axes=axes, norm="ortho"), axes=axes)


def mask_indices(mask):
    """Sampling operator U as the ascending row-major list of sampled flat indices (int64)."""
    return np.flatnonzero(np.asarray(mask).ravel())


def cartesian_fwd(x, maps, idx):
    """A x for A = U F C: y[c, i] = (F(c_c * x)).flat[idx[i]].  maps [C, *shape]; returns [C, N]."""
    nd = x.ndim
    axes = tuple(range(1, nd + 1))
    k = centred_fft(maps * x[None], axes)
    return k.reshape(maps.shape[0], -1)[:, idx]


def cartesian_adj(y, maps, idx):
    """A^H y = sum_c conj(c_c) * F^H(U^H y_c)."""
    C = maps.shape[0]
    shape = maps.shape[1:]
    axes = tuple(range(1, len(shape) + 1))
    full = np.zeros((C, int(np.prod(shape))), dtype=np.complex128)
    full[:, idx] = y
    z = centred_ifft(full.reshape((C,) + shape), axes)
    return np.sum(np.conj(maps) * z, axis=0)


def sampled_frequencies(shape, idx):
    """Frequencies f_i (cycles/pixel, [N, nd]) of the sampled Cartesian grid entries."""
    coords = np.unravel_index(idx, shape)
    return np.stack([(coords[a] - shape[a] // 2) / shape[a] for a in range(len(shape))], axis=-1)


def dense_sense_matrix(maps, freqs, dcf=None):
    """Brute-force A (C*N x D) built entry by entry from Eq. 1 (tiny inputs only).

    Row (c, i), column d: sqrt(w_i) * c_c[d] * exp(-i 2 pi <f_i, r_d>) / sqrt(D).
    """
    C = maps.shape[0]
    shape = maps.shape[1:]
    D = int(np.prod(shape))
    r = np.stack(np.meshgrid(*[np.arange(n) - n // 2 for n in shape], indexing="ij"), -1).reshape(D, -1)
    E = np.exp(-2j * np.pi * (np.asarray(freqs, dtype=np.float64) @ r.T.astype(np.float64))) / np.sqrt(D)
    if dcf is not None:
        E = E * np.sqrt(np.asarray(dcf, dtype=np.float64))[:, None]
    blocks = [E * maps[c].reshape(1, D) for c in range(C)]
    return np.concatenate(blocks, axis=0)
