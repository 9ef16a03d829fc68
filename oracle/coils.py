"""Coil compression (PCA) and the structured coil sketch (Sec. 2.3, Sec. 3.1, Algorithm 1).

* Coil compression: SVD-based compression of the k-space data (Sec. 3.1; Algorithm 1 keeps
  the first C^_0 high-energy virtual coils).  We form R = Y Y^H over all acquired samples,
  take its eigenvectors sorted by descending eigenvalue (the left singular vectors of Y),
  fix each eigenvector's phase so that its largest-magnitude entry is real positive, and
  rotate maps and data with U^H: c' = U^H c, y' = U^H y.
* Structured sketch (Sec. 2.3): S^t = S~^t (x) I_N, S~^t = [[I_V, 0], [0, S~_S^t]] with
  S~_S^t in R^{S x (C-V)} i.i.d.; C^ = V + S.
* Sketch/operator commutation (Eq. 7-8): A_S^t = S^t W^1/2 F C = W^^1/2 F^ C_S^t, with sketched
  maps c^[d] = S~^t c[d] for every voxel d.
"""
from __future__ import annotations

import numpy as np


def coil_covariance(y):
    """R[a, b] = sum_i y_a[i] conj(y_b[i]) for y [C, N] (complex128 [C, C])."""
    y = np.asarray(y, dtype=np.complex128)
    return y @ y.conj().T


def coil_pca(y):
    """Eigenvectors U (columns, descending eigenvalue, phase-fixed) and eigenvalues of Y Y^H."""
    R = coil_covariance(y)
    evals, evecs = np.linalg.eigh(R)
    order = np.argsort(evals)[::-1]
    evals = evals[order]
    U = evecs[:, order]
    for k in range(U.shape[1]):
        j = int(np.argmax(np.abs(U[:, k])))
        ph = U[j, k] / np.abs(U[j, k])
        U[:, k] = U[:, k] / ph
    return U, evals


def rotate(U, a):
    """a' = U^H a along the coil axis (axis 0); works for maps [C, ...] and data [C, N]."""
    a = np.asarray(a, dtype=np.complex128)
    C = a.shape[0]
    return (U.conj().T @ a.reshape(C, -1)).reshape(a.shape)


def full_sketch(S_low, C, V):
    """S~ = blockdiag(I_V, S~_S) of shape (V+S, C) from the random block S~_S (S x (C-V))."""
    S_low = np.asarray(S_low, dtype=np.float64).reshape(-1, C - V) if C > V else np.zeros((0, 0))
    S = S_low.shape[0] if C > V else 0
    M = np.zeros((V + S, C))
    M[:V, :V] = np.eye(V)
    if S:
        M[V:, V:] = S_low
    return M


def sketched_maps(S_low, maps_rot, V):
    """c^ = S~ c' per voxel: rows 0..V-1 are c'_0..c'_{V-1}, rows V.. are S~_S c'_{V..C-1}."""
    C = maps_rot.shape[0]
    M = full_sketch(S_low, C, V)
    return (M.astype(np.complex128) @ maps_rot.reshape(C, -1)).reshape((M.shape[0],) + maps_rot.shape[1:])


def sketch_data(S_low, y, V):
    """(S~ (x) I_N) y for k-space y [C, N]: the sketch applied in the coil dimension."""
    C = y.shape[0]
    M = full_sketch(S_low, C, V)
    return M.astype(np.complex128) @ y
