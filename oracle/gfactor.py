"""Inverse g-factor (Pruessmann et al. 1999; the paper's Sec. 3.2 noise analysis): the noise
amplification of an undersampled reconstruction relative to the fully sampled one, g =
std_R / (std_full sqrt(R)) per pixel, estimated by the Monte Carlo pseudo-replica method
(Robson et al. 2008: reconstruct many copies of the data with independent noise and take the
per-pixel standard deviation), and - for unregularised SENSE with regular Cartesian
undersampling - in closed form.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def noise_std(recons):
    """Per-pixel standard deviation over the first axis (trials): sqrt(mean_k |x_k - mean|^2)."""
    x = np.asarray(recons, dtype=np.complex128)
    mu = x.mean(axis=0)
    return np.sqrt(np.mean(np.abs(x - mu) ** 2, axis=0))


def inverse_gfactor_mc(recons_R, recons_full, R):
    """1/g = std_full sqrt(R) / std_R from two stacks of reconstructions of noisy replicas."""
    return noise_std(recons_full) * np.sqrt(R) / noise_std(recons_R)


def inverse_gfactor_sense(maps, R, offset=0):
    """Closed form for SENSE with every R-th row sampled (rows = first image axis) and white
    noise: the pixels y, y + ny/R, ... fold onto each other; with the encoding matrix
    E = maps[:, fold, x] (C x R), g_i = sqrt([(E^H E)^-1]_ii [E^H E]_ii)."""
    maps = np.asarray(maps, dtype=np.complex128)
    C, ny, nx = maps.shape
    assert ny % R == 0
    step = ny // R
    inv_g = np.zeros((ny, nx))
    for y0 in range(step):
        fold = [y0 + j * step for j in range(R)]
        for x in range(nx):
            E = maps[:, fold, x]
            H = E.conj().T @ E
            Hi = np.linalg.inv(H)
            g = np.sqrt(np.real(np.diag(Hi) * np.diag(H)))
            inv_g[fold, x] = 1.0 / g
    return inv_g
