"""Operator use of the oracle's solvers against the counts printed in Table 2 (Sec. 4, 3D cones
l1-Wavelets; fixture tests/golden/table2_fft_counts.txt): the full-coil FISTA baseline,
aggressive coil compression and AccProxSGD each apply the forward and the adjoint operator once
per iteration on every coil they use, so coil FFTs = 2 x coils x iterations and one wavelet
prox per iteration.  The counts are reproduced by running each oracle solver for the printed
number of iterations on a small 2D Cartesian problem with the printed coil numbers and counting
the coil FFTs and prox evaluations it performs."""
import os

import numpy as np
import pytest

from oracle import fourier, solvers, wavelet


def _table2():
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_fft_counts.txt")
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, coils, ffts, wav = line.split()
        out[name] = (int(coils), int(ffts), int(wav))
    return out


@pytest.fixture
def counters(monkeypatch):
    n = {"fft": 0, "prox": 0}
    f0, i0, p0 = fourier.centred_fft, fourier.centred_ifft, wavelet.prox_l1_wavelet

    def fft(u, axes):
        n["fft"] += u.shape[0] if len(axes) < u.ndim else 1     # one FFT per coil
        return f0(u, axes)

    def ifft(k, axes):
        n["fft"] += k.shape[0] if len(axes) < k.ndim else 1
        return i0(k, axes)

    def prox(v, tau, levels=4):
        n["prox"] += 1
        return p0(v, tau, levels)

    monkeypatch.setattr(fourier, "centred_fft", fft)
    monkeypatch.setattr(fourier, "centred_ifft", ifft)
    monkeypatch.setattr(wavelet, "prox_l1_wavelet", prox)
    return n


def _problem(C, n=16, seed=0):
    rng = np.random.default_rng(seed)
    maps = rng.standard_normal((C, n, n)) + 1j * rng.standard_normal((C, n, n))
    maps /= np.sqrt((np.abs(maps) ** 2).sum(axis=0, keepdims=True))
    mask = rng.random((n, n)) < 0.5
    idx = fourier.mask_indices(mask)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y = fourier.cartesian_fwd(x, maps, idx)

    def ops(m):
        return (lambda v: fourier.cartesian_fwd(v, m, idx)), (lambda k: fourier.cartesian_adj(k, m, idx))

    return maps, y, ops


def test_table2_rows_are_one_forward_and_adjoint_per_iteration():
    t = _table2()
    for name in ("baseline", "coil_compression", "acc_prox_sgd"):
        coils, ffts, wav = t[name]
        assert ffts == 2 * coils * wav, name
    assert t["baseline"][0] == 20 and t["coil_compression"][0] == 4


def test_baseline_fista_counts(counters):
    coils, ffts, wav = _table2()["baseline"]
    maps, y, ops = _problem(coils)
    fwd, adj = ops(maps)
    counters["fft"] = counters["prox"] = 0
    solvers.plain_fista(fwd, adj, y, 1e-3, 0.5, np.zeros((16, 16), complex), wav, levels=2)
    assert (counters["fft"], counters["prox"]) == (ffts, wav)


def test_coil_compression_counts(counters):
    coils, ffts, wav = _table2()["coil_compression"]
    maps, y, ops = _problem(20)
    counters["fft"] = counters["prox"] = 0
    solvers.coil_compressed(ops, maps, y, coils,
                            lambda f, a, yk: solvers.plain_fista(f, a, yk, 1e-3, 0.5, np.zeros((16, 16), complex),
                                                                 wav, levels=2))
    assert (counters["fft"], counters["prox"]) == (ffts, wav)


def test_acc_prox_sgd_counts(counters):
    coils, ffts, wav = _table2()["acc_prox_sgd"]
    maps, y, ops = _problem(20)
    rng = np.random.default_rng(1)
    batches = np.stack([rng.choice(20, coils, replace=False) for _ in range(wav)])
    counters["fft"] = counters["prox"] = 0
    solvers.acc_prox_sgd(ops, maps, y, 1e-3, batches, 0.1, 0.99, 0.1, np.zeros((16, 16), complex), wav, levels=2)
    assert (counters["fft"], counters["prox"]) == (ffts, wav)
