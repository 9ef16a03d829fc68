"""GPU inverse g-factor by pseudo-replicas (the paper's Sec. 3.2): the batched replica solve
(one captured graph) against the FP64 oracle run on the same noise, for the plain SENSE solver
and for coil sketching, and the plain solver's map against the closed form."""
import numpy as np
import pytest
import torch

import synthdata
from oracle import fourier, gfactor, philox, solvers

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from tests._gpu import ensure_built
    ensure_built()


def _case(shape=(48, 40), C=6, R=3, replicas=12):
    mask = synthdata.regular_mask(shape, R)
    idx = fourier.mask_indices(mask)
    full = np.arange(int(np.prod(shape)))
    maps = synthdata.coil_maps(shape, C)
    x = synthdata.phantom(shape, seed=1)
    sigma = 1e-2
    nR = np.stack([synthdata.complex_noise((C, len(idx)), sigma, seed=100 + k) for k in range(replicas)])
    n1 = np.stack([synthdata.complex_noise((C, len(full)), sigma, seed=500 + k) for k in range(replicas)])
    return shape, C, R, idx, full, maps, x, nR, n1


def test_replica_gfactor_matches_oracle_plain_and_sketched():
    import paper_2305_06482_gb300 as cs
    from paper_2305_06482_gb300 import gfactor as gf
    from tests._gpu import t, h, nrmse
    shape, C, R, idx, full, maps, x, nR, n1 = _case()
    lam, K = 1e-4, 40
    yR = fourier.cartesian_fwd(x, maps, idx)
    y1 = fourier.cartesian_fwd(x, maps, full)
    plain = cs.SolveParams(K=K, sketch=False, do_pca=False, use_graph=True)
    ysR, ys1 = gf.replicas(t(yR), t(nR)), gf.replicas(t(y1), t(n1))
    xR, _ = gf.replica_reconstructions(shape, t(maps), t(idx, np.int32), ysR, lam, plain)
    x1, _ = gf.replica_reconstructions(shape, t(maps), t(full, np.int32), ys1, lam, plain)
    ops = lambda ix: (lambda v: fourier.cartesian_fwd(v, maps, ix), lambda r: fourier.cartesian_adj(r, maps, ix))
    fR, aR = ops(idx)
    f1, a1 = ops(full)
    z = np.zeros(shape, complex)
    refR = np.stack([solvers.plain_cg(fR, aR, yR + n, lam, z, K) for n in nR])
    ref1 = np.stack([solvers.plain_cg(f1, a1, y1 + n, lam, z, K) for n in n1])
    assert nrmse(h(xR), refR) < 1e-4 and nrmse(h(x1), ref1) < 1e-4
    ig = gf.inverse_gfactor(xR, x1, R)
    ig_ref = gfactor.inverse_gfactor_mc(refR, ref1, R)
    assert nrmse(h(ig), ig_ref) < 1e-3
    # few replicas, but the map already follows the closed form of unregularised SENSE
    assert np.median(np.abs(h(ig).real / gfactor.inverse_gfactor_sense(maps, R) - 1)) < 0.3
    # coil sketching (l2, C^ = 4 of 6), same sketch for every replica
    V, S, T, Ks = 3, 1, 4, 10
    sk = philox.sketch_draw(3, 0, T, C, V, S)
    sketched = cs.SolveParams(T=T, K=Ks, V=V, S=S, seed=3, use_graph=True)   # batched solves draw S~ themselves
    xs, _ = gf.replica_reconstructions(shape, t(maps), t(idx, np.int32), ysR, lam, sketched)
    opsm = lambda m: (lambda v: fourier.cartesian_fwd(v, m, idx), lambda r: fourier.cartesian_adj(r, m, idx))
    refs = np.stack([solvers.coil_sketching(opsm, maps, yR + n, lam, "l2", sk.astype(np.float64), V=V, K=Ks)[0]
                     for n in nR])
    assert nrmse(h(xs), refs) < 1e-4
    assert nrmse(h(gf.inverse_gfactor(xs, x1, R)), gfactor.inverse_gfactor_mc(refs, ref1, R)) < 1e-3
