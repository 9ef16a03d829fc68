"""l1 total variation (Sec. 2.1, regulariser g(x) = lambda ||T x||_1 with T first-order finite
differences under periodic boundary extension) and the pieces the PDHG solver of Chambolle and
Pock (2011, cited for l1-TV in Sec. 2.1) needs.

Reading: T stacks the forward difference along every image axis, (T x)_a[r] = x[r + e_a] - x[r]
(indices modulo the image size), and ||.||_1 sums the complex moduli of all its entries
(anisotropic TV).  The prox of sigma g* (g* the conjugate of lambda ||.||_1) is then the
entry-wise projection onto the complex disc of radius lambda.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def tv_fwd(x):
    """T x: array [ndim, *x.shape], forward differences with periodic wrap along every axis."""
    x = np.asarray(x, dtype=np.complex128)
    return np.stack([np.roll(x, -1, axis=a) - x for a in range(x.ndim)])


def tv_adj(z):
    """T^H z = sum_a (z_a[r - e_a] - z_a[r]) (minus the periodic backward divergence)."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.zeros(z.shape[1:], dtype=np.complex128)
    for a in range(z.shape[0]):
        out += np.roll(z[a], 1, axis=a) - z[a]
    return out


def tv_norm_sq(ndim):
    """||T||^2 = 4 ndim: T^H T is the periodic negative Laplacian, whose largest eigenvalue is
    sum_a 4 sin^2(pi k_a / n_a) at k_a = n_a / 2 (even sizes)."""
    return 4.0 * ndim


def tv_value(x, lam):
    """lambda ||T x||_1 (sum of the complex moduli of all differences)."""
    return float(lam * np.sum(np.abs(tv_fwd(x))))


def project_disc(z, lam):
    """Entry-wise projection onto {|z_i| <= lam}: z_i / max(1, |z_i| / lam)."""
    z = np.asarray(z, dtype=np.complex128)
    return z / np.maximum(1.0, np.abs(z) / lam)
