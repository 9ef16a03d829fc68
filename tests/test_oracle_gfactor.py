"""Pins of the inverse g-factor (the paper's Sec. 3.2 noise analysis, Pruessmann et al. 1999):
the closed form for regular SENSE undersampling against the exact noise covariance of the
dense least-squares reconstruction, and the Monte Carlo pseudo-replica estimate against both."""
import numpy as np
import pytest

import synthdata
from oracle import fourier, gfactor


def _dense_case(shape=(12, 10), C=4, R=2):
    maps = synthdata.coil_maps(shape, C)
    mask = synthdata.regular_mask(shape, R)
    idx = fourier.mask_indices(mask)
    A = fourier.dense_sense_matrix(maps, fourier.sampled_frequencies(shape, idx))
    A_full = fourier.dense_sense_matrix(maps, fourier.sampled_frequencies(shape, np.arange(np.prod(shape))))
    return maps, A, A_full


@pytest.mark.parametrize("R", [2, 3])
def test_closed_form_matches_exact_noise_covariance(R):
    maps, A, A_full = _dense_case(shape=(12, 10), R=R)
    # white noise of unit variance per sample: recon covariance (A^H A)^-1
    cov_R = np.linalg.inv(A.conj().T @ A)
    cov_1 = np.linalg.inv(A_full.conj().T @ A_full)
    inv_g = np.sqrt(np.real(np.diag(cov_1)) * R / np.real(np.diag(cov_R))).reshape(12, 10)
    assert np.allclose(inv_g, gfactor.inverse_gfactor_sense(maps, R), atol=1e-9)
    assert inv_g.max() <= 1 + 1e-9          # g >= 1: undersampling never lowers the noise below sqrt(R)


def test_no_undersampling_gives_unit_inverse_gfactor():
    maps = synthdata.coil_maps((8, 6), 3)
    assert np.allclose(gfactor.inverse_gfactor_sense(maps, 1), 1.0)


def test_monte_carlo_estimate_converges_to_closed_form():
    R, shape = 2, (12, 10)
    maps, A, A_full = _dense_case(shape=shape, R=R)
    rng = np.random.default_rng(7)
    trials = 3000
    pinv_R = np.linalg.pinv(A)
    pinv_1 = np.linalg.pinv(A_full)
    nR = (rng.standard_normal((trials, A.shape[0])) + 1j * rng.standard_normal((trials, A.shape[0]))) / np.sqrt(2)
    n1 = (rng.standard_normal((trials, A_full.shape[0])) + 1j * rng.standard_normal((trials, A_full.shape[0]))) / np.sqrt(2)
    xR = (nR @ pinv_R.T).reshape((trials,) + shape)
    x1 = (n1 @ pinv_1.T).reshape((trials,) + shape)
    est = gfactor.inverse_gfactor_mc(xR, x1, R)
    ref = gfactor.inverse_gfactor_sense(maps, R)
    assert np.median(np.abs(est / ref - 1)) < 0.03
    assert np.abs(est / ref - 1).max() < 0.12
    # noise_std is the per-pixel standard deviation over trials
    z = rng.standard_normal((5, 3)) + 1j * rng.standard_normal((5, 3))
    assert np.allclose(gfactor.noise_std(z), np.std(z, axis=0))
