"""GPU parity of coil PCA (FP64 Jacobi on the device), coil rotation, sketch draws (Philox bit
patterns, Sec. 3.2 distributions) and the FP32 sketched-maps contraction (Eq. 8)."""
import numpy as np
import pytest
import torch

import synthdata
from oracle import coils, philox

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from tests._gpu import ensure_built
    ensure_built()


@pytest.mark.parametrize("C,N", [(8, 4096), (5, 1000), (32, 20000), (40, 7777)])
def test_coil_pca(C, N):
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h
    y = synthdata.random_complex((C, N), C) * np.geomspace(3, 0.05, C)[:, None]
    U, eig = cs.coil_pca(t(y))
    Ug, eg = h(U), eig.cpu().numpy()
    Ur, er = coils.coil_pca(y.astype(np.complex64).astype(np.complex128))
    assert np.allclose(eg, er, rtol=1e-5)      # FP32 blocked accumulation of R, FP64 eig
    assert abs(eg.sum() - np.linalg.norm(y) ** 2) <= 1e-5 * eg.sum()
    # distinct eigenvalues: eigenvectors agree after the shared phase convention
    assert np.abs(Ug - Ur).max() < 1e-3
    assert np.allclose(Ug.conj().T @ Ug, np.eye(C), atol=1e-5)
    # the FP64 block sums are added in a fixed order: a second call is bit-identical
    U2, eig2 = cs.coil_pca(t(y))
    assert torch.equal(U2, U) and torch.equal(eig2, eig)


def test_coil_rotate():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    C = 12
    y = synthdata.random_complex((C, 3000), 1)
    U, _ = coils.coil_pca(y)
    m = synthdata.random_complex((C, 20, 36), 2)
    out = cs.coil_rotate(t(U), t(m))
    assert nrmse(h(out), coils.rotate(U, m)) < 1e-6
    out5 = cs.coil_rotate(t(U), t(m), c_out=5)
    assert nrmse(h(out5), coils.rotate(U, m)[:5]) < 1e-6


@pytest.mark.parametrize("dist,norm", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_sketch_draw_matches_oracle_bits(dist, norm):
    import paper_2305_06482_gb300 as cs
    got = cs.sketch_draw(0x123456789, 3, 4, 40, 5, 5, dist=dist, norm=norm).cpu().numpy()
    want = philox.sketch_draw(0x123456789, 3, 4, 40, 5, 5, dist=dist, norm=norm)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_sketched_maps_fp32():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    C, V, S = 32, 4, 4
    m = synthdata.random_complex((C, 24, 40), 3)
    Sk = philox.sketch_draw(7, 0, 1, C, V, S)[0]
    out = cs.sketched_maps(t(Sk), t(m), V)
    ref = coils.sketched_maps(Sk.astype(np.float64), m.astype(np.complex64).astype(np.complex128), V)[V:]
    assert nrmse(h(out), ref) < 1e-6


@pytest.mark.parametrize("C,V,S,D", [(32, 4, 4, 4096 + 37), (40, 5, 5, 20000), (12, 2, 16, 1000), (20, 4, 3, 64 * 300)])
def test_sketched_maps_bf16_split_tensor_cores(C, V, S, D):
    """BF16 x (hi + lo) split on the tensor cores vs the FP64 product: the split keeps about 16
    mantissa bits of each map entry, so the relative error is of order 2^-17."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    m = synthdata.random_complex((C, D), 3)
    Sk = philox.sketch_draw(7, 0, 1, C, V, S)[0]
    out = cs.sketched_maps(t(Sk), t(m), V, precision=cs.PREC_BF16_SPLIT)
    cs.device_status()
    ref = coils.sketched_maps(Sk.astype(np.float64), m.astype(np.complex64).astype(np.complex128), V)[V:]
    err = nrmse(h(out), ref)
    assert err < 2e-5, err
    fp32 = cs.sketched_maps(t(Sk), t(m), V, precision=cs.PREC_FP32)
    assert nrmse(h(fp32), ref) < 1e-6
