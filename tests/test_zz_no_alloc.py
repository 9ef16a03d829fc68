"""coil_pca_noalloc, the allocation-free variant of coil_pca for callers that cannot allocate
device memory while they run: its results must match coil_pca's on the same data, on two calls
in a row (the shared static scratch is cleared by each call), and sizes above its 64-coil limit
must be refused on the host.  Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from tests._gpu import ensure_built
    ensure_built()


@pytest.mark.parametrize("C,N", [(8, 4096), (40, 7777), (64, 3000)])
def test_noalloc_matches_coil_pca_twice(C, N):
    import torch
    import paper_2305_06482_gb300 as cs
    import synthdata
    from tests._gpu import t
    y = t(synthdata.random_complex((C, N), C) * np.geomspace(3, 0.05, C)[:, None])
    U_ref, e_ref = cs.coil_pca(y)
    torch.cuda.synchronize()
    for _ in range(2):
        U, e = cs.coil_pca_noalloc(y)
        torch.cuda.synchronize()
        assert np.allclose(e.cpu().numpy(), e_ref.cpu().numpy(), rtol=1e-9, atol=0)
        assert np.abs(U.cpu().numpy() - U_ref.cpu().numpy()).max() < 1e-5
    # a different input next: the scratch must not carry the previous call's covariance
    y2 = t(synthdata.random_complex((C, N), C + 100))
    U2_ref, e2_ref = cs.coil_pca(y2)
    U2, e2 = cs.coil_pca_noalloc(y2)
    torch.cuda.synchronize()
    assert np.allclose(e2.cpu().numpy(), e2_ref.cpu().numpy(), rtol=1e-9, atol=0)


def test_noalloc_rejects_too_many_coils():
    import paper_2305_06482_gb300 as cs
    import synthdata
    from tests._gpu import t
    y = t(synthdata.random_complex((65, 64), 1))
    with pytest.raises(cs.CoilSketchError) as e:
        cs.coil_pca_noalloc(y)
    assert e.value.code == 2
