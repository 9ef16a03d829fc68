"""Pins for coil PCA and the structured sketch (Sec. 2.3, Eq. 7-8; Sec. 3.1 coil compression)."""
import numpy as np

import synthdata
from oracle import coils, fourier, nufft


def test_pca_spectral_identities():
    y = synthdata.random_complex((6, 500), 1) * np.arange(1, 7)[:, None]
    U, ev = coils.coil_pca(y)
    R = y @ y.conj().T
    assert abs(ev.sum() - np.linalg.norm(y) ** 2) <= 1e-10 * ev.sum()          # trace
    assert np.allclose(U.conj().T @ U, np.eye(6), atol=1e-12)                  # unitary
    assert np.all(np.diff(ev) <= 0)                                            # descending
    assert np.allclose(R @ U, U * ev[None, :], atol=1e-9 * ev[0])              # eigenpairs
    j = np.argmax(np.abs(U), axis=0)
    piv = U[j, np.arange(6)]
    assert np.allclose(piv.imag, 0, atol=1e-15) and np.all(piv.real > 0)      # phase convention
    # rotated data energies equal the eigenvalues
    yr = coils.rotate(U, y)
    assert np.allclose(np.sum(np.abs(yr) ** 2, axis=1), ev, rtol=1e-10)


def test_rotation_leaves_objective_invariant():
    shape = (12, 12)
    maps = synthdata.coil_maps(shape, 5)
    idx = fourier.mask_indices(np.random.default_rng(2).random(shape) < 0.4)
    x = synthdata.random_complex(shape, 3)
    y = fourier.cartesian_fwd(synthdata.random_complex(shape, 4), maps, idx)
    U, _ = coils.coil_pca(y)
    r1 = np.linalg.norm(fourier.cartesian_fwd(x, maps, idx) - y)
    r2 = np.linalg.norm(fourier.cartesian_fwd(x, coils.rotate(U, maps), idx) - coils.rotate(U, y))
    assert abs(r1 - r2) <= 1e-12 * r1


def test_sketch_commutes_with_operator_cartesian_and_nufft():
    """Eq. 7: (S~ (x) I_N) W^1/2 F C x = W^1/2 F C_S x with c^ = S~ c per voxel (Eq. 8)."""
    rng = np.random.default_rng(5)
    C, V, S = 6, 2, 3
    S_low = rng.standard_normal((S, C - V))
    shape = (10, 12)
    maps = synthdata.random_complex((C,) + shape, 6)
    x = synthdata.random_complex(shape, 7)
    idx = fourier.mask_indices(rng.random(shape) < 0.5)
    lhs = coils.sketch_data(S_low, fourier.cartesian_fwd(x, maps, idx), V)
    rhs = fourier.cartesian_fwd(x, coils.sketched_maps(S_low, maps, V), idx)
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()
    img, grid = (8, 8, 8), (10, 10, 10)
    traj = rng.uniform(-0.5, 0.5, (300, 3)).astype(np.float32)
    dcf = rng.uniform(0.2, 1, 300).astype(np.float32)
    m3 = synthdata.random_complex((C,) + img, 8)
    x3 = synthdata.random_complex(img, 9)
    plan = nufft.Plan(traj, img, grid)
    lhs = coils.sketch_data(S_low, nufft.sense_fwd(plan, x3, m3, dcf), V)
    rhs = nufft.sense_fwd(plan, x3, coils.sketched_maps(S_low, m3, V), dcf)
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()


def test_virtual_coil_block_form_and_identity_case():
    C, V = 5, 2
    S_low = np.arange(6, dtype=float).reshape(2, 3)
    M = coils.full_sketch(S_low, C, V)
    assert M.shape == (4, 5)
    assert np.array_equal(M[:2, :2], np.eye(2)) and not M[:2, 2:].any() and not M[2:, :2].any()
    maps = synthdata.random_complex((C, 4, 4), 1)
    # V = C: S~ = I, the sketched maps are the rotated maps exactly
    full = coils.sketched_maps(np.zeros((0, 0)), maps, C)
    assert np.array_equal(full, maps)
