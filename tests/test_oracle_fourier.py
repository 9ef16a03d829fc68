"""Pins for the Cartesian SENSE oracle (Sec. 2.1, Eq. 1-2): brute-force dense A built from
Eq. 1, adjointness, Parseval, A^H A = I for full sampling with RSS-normalised maps."""
import numpy as np

import synthdata
from oracle import fourier


def _tiny(seed=0, shape=(8, 8), C=3, frac=0.5):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    maps = rng.standard_normal((C,) + shape) + 1j * rng.standard_normal((C,) + shape)
    mask = rng.random(shape) < frac
    return x, maps, fourier.mask_indices(mask), mask


def test_matches_dense_matrix_from_eq1():
    for shape in [(8, 8), (6, 10), (4, 6, 8)]:
        x, maps, idx, _ = _tiny(1, shape)
        A = fourier.dense_sense_matrix(maps, fourier.sampled_frequencies(shape, idx))
        y_dense = A @ x.ravel()
        y = fourier.cartesian_fwd(x, maps, idx).ravel()
        assert np.abs(y - y_dense).max() <= 1e-12 * np.abs(y_dense).max()
        # adjoint equals the dense conjugate transpose
        yy = np.random.default_rng(2).standard_normal(y.shape) * (1 + 1j)
        xa = fourier.cartesian_adj(yy.reshape(maps.shape[0], -1), maps, idx).ravel()
        assert np.abs(xa - A.conj().T @ yy).max() <= 1e-12 * np.abs(xa).max()


def test_adjointness():
    x, maps, idx, _ = _tiny(3, (16, 12), C=4)
    y = np.random.default_rng(4).standard_normal((4, idx.size)) + 0j
    lhs = np.vdot(fourier.cartesian_fwd(x, maps, idx), y)
    rhs = np.vdot(x, fourier.cartesian_adj(y, maps, idx))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_parseval_and_centring():
    rng = np.random.default_rng(5)
    u = rng.standard_normal((12, 16)) + 1j * rng.standard_normal((12, 16))
    k = fourier.centred_fft(u, (0, 1))
    assert abs(np.linalg.norm(k) - np.linalg.norm(u)) <= 1e-12 * np.linalg.norm(u)
    # a delta at the image centre (r = 0) has the constant transform 1/sqrt(D)
    d = np.zeros((12, 16), complex)
    d[6, 8] = 1
    assert np.allclose(fourier.centred_fft(d, (0, 1)), 1 / np.sqrt(12 * 16), atol=1e-15)
    # a delta at r = (0, 1) has phase exp(-i 2 pi f_x) at frequency f_x = (p - n/2)/n
    d = np.zeros((12, 16), complex)
    d[6, 9] = 1
    f = (np.arange(16) - 8) / 16
    assert np.allclose(fourier.centred_fft(d, (0, 1))[3], np.exp(-2j * np.pi * f) / np.sqrt(192), atol=1e-15)


def test_full_sampling_rss_maps_gives_identity_normal_operator():
    shape = (16, 16)
    maps = synthdata.coil_maps(shape, 6)
    idx = np.arange(256)
    x = synthdata.random_complex(shape, 7)
    z = fourier.cartesian_adj(fourier.cartesian_fwd(x, maps, idx), maps, idx)
    assert np.abs(z - x).max() <= 1e-12
