"""Pins for the periodised db4 transform: the Daubechies filter identities (normalisation,
double-shift orthonormality, four vanishing moments), Psi unitary (explicit matrix), vanishing
detail coefficients on cubic polynomials, and the soft-threshold prox as an exact minimiser."""
import numpy as np

from oracle import wavelet


def test_db4_filter_identities():
    h, g = wavelet.H, wavelet.G
    assert h.size == 8
    assert abs(h.sum() - np.sqrt(2)) < 1e-14
    for m in range(4):
        assert abs(np.dot(h[: 8 - 2 * m], h[2 * m:]) - (1.0 if m == 0 else 0.0)) < 1e-14
        assert abs(np.dot(h[: 8 - 2 * m], g[2 * m:])) < 1e-14 and abs(np.dot(g[: 8 - 2 * m], h[2 * m:])) < 1e-14
    k = np.arange(8)
    for p in range(4):
        assert abs(np.sum(g * k ** p)) < 1e-11 * max(1, 8 ** p)     # 4 vanishing moments
    assert abs(np.sum(g * k ** 4)) > 1e-3                          # and not 5


def test_transform_is_unitary_explicit_matrix():
    shape = (16, 16)
    n = 256
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1
        M[:, j] = wavelet.wavedec(e.reshape(shape), 2).real.ravel()
    assert np.allclose(M.T @ M, np.eye(n), atol=1e-13)
    x = np.random.default_rng(1).standard_normal((32, 48, 16)) * (1 + 0.5j)
    c = wavelet.wavedec(x, 4 - 1)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    assert np.abs(wavelet.waverec(c, 3) - x).max() < 1e-12


def test_details_vanish_on_cubics_away_from_the_wrap():
    n = 64
    t = np.arange(n, dtype=float)
    x = 0.3 - 0.2 * t + 0.01 * t ** 2 - 0.0004 * t ** 3
    c = wavelet.dwt1(x.astype(complex), 0)
    d = c[n // 2:]
    assert np.abs(d[: n // 2 - 4]).max() < 1e-9       # windows that do not wrap around


def test_prox_is_the_exact_minimiser():
    rng = np.random.default_rng(3)
    v = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    tau = 0.7
    x = wavelet.prox_l1_wavelet(v, tau, 2)
    obj = lambda z: 0.5 * np.linalg.norm(z - v) ** 2 + tau * np.abs(wavelet.wavedec(z, 2)).sum()
    f0 = obj(x)
    for _ in range(50):
        assert obj(x + 1e-3 * (rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape))) >= f0 - 1e-12
    # soft threshold closed form
    z = np.array([3 + 4j, 0.1j, 0, -2])
    assert np.allclose(wavelet.soft_threshold(z, 1.0), [(3 + 4j) * 0.8, 0, 0, -1])
