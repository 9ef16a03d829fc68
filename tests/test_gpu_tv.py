"""GPU parity of l1-TV reconstruction (Sec. 2.1: g(x) = lambda ||T x||_1, solved by PDHG whose
data step runs CG): the two element-wise PDHG steps against the oracle's T, T^H and dual
projection, then Algorithm 1 and the plain solver with PDHG against the FP64 oracle run with
the same inputs and sketches (final-image NRMSE <= 1e-4), and graph replay against eager."""
import numpy as np
import pytest
import torch

import synthdata
from oracle import fourier, nufft, philox, solvers, tv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from tests._gpu import ensure_built
    ensure_built()


@pytest.mark.parametrize("shape", [(37, 50), (9, 12, 17), (1, 7, 3)])
def test_pdhg_steps_match_oracle(shape):
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    nd = len(shape)
    x = synthdata.random_complex(shape, 1)
    xp = synthdata.random_complex(shape, 2)
    z = 0.5 * synthdata.random_complex((nd,) + shape, 3)
    sigma, lam = 0.4, 0.7
    zg = t(z)
    cs.tv_dual_update(t(x), zg, sigma, lam, x_prev=t(xp))
    ref = tv.project_disc(z + sigma * tv.tv_fwd(2 * x - xp), lam)
    assert nrmse(h(zg), ref) < 1e-6
    assert np.abs(h(zg)).max() <= lam * (1 + 1e-6)
    zg2 = t(np.zeros((nd,) + shape, dtype=np.complex64))
    cs.tv_dual_update(t(x), zg2, 1.0, 1e30)              # no projection, x_prev None: z = T x
    assert nrmse(h(zg2), tv.tv_fwd(x)) < 1e-6
    b0 = synthdata.random_complex(shape, 4)
    xo = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    xg = t(x)
    rhs = cs.tv_rhs(xg, t(z), 1.7, b0=t(b0), x_prev_out=xo)
    assert nrmse(h(rhs), b0 + 1.7 * x - tv.tv_adj(z)) < 1e-6
    assert torch.equal(xo, xg)
    rhs0 = cs.tv_rhs(xg, t(z), 0.0)
    assert nrmse(h(rhs0), -tv.tv_adj(z)) < 1e-6


def _cart_problem(shape=(64, 64), C=8, seed=1):
    mask = synthdata.poisson_disc_mask(shape, R=3.0, centre=16, seed=2)
    idx = fourier.mask_indices(mask)
    maps = synthdata.coil_maps(shape, C)
    y = fourier.cartesian_fwd(synthdata.phantom(shape, seed=seed), maps, idx)
    y = y + synthdata.complex_noise(y.shape, 1e-3 * np.abs(y).max(), seed=3)
    ops = lambda m: (lambda v: fourier.cartesian_fwd(v, m, idx), lambda k: fourier.cartesian_adj(k, m, idx))
    return idx, maps, y, ops


def test_coil_sketching_tv_cartesian():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    shape = (64, 64)
    idx, maps, y, ops = _cart_problem(shape)
    C, V, S, T, K, M, lam = 8, 5, 3, 3, 6, 4, 2e-3
    sk = philox.sketch_draw(7, 0, T, C, V, S)
    x_ref, its = solvers.coil_sketching(ops, maps, y, lam, "l1tv", sk.astype(np.float64), V=V, K=K, cg_iters=M)
    plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=t(idx, np.int32))
    iters = torch.empty((T,) + shape, dtype=torch.complex64, device="cuda")
    x, _ = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_TV,
                          cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk), cg_iters=M, iterates=iters))
    assert nrmse(h(x), x_ref) < 1e-4
    for k in range(T):
        assert nrmse(h(iters[k]), its[k]) < 1e-4


def test_plain_tv_cartesian():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    shape = (64, 64)
    idx, maps, y, ops = _cart_problem(shape)
    fwd, adj = ops(maps)
    lam, K, M = 2e-3, 12, 4
    tau, sigma = solvers.pdhg_steps(2)
    x_ref, _ = solvers.plain_pdhg(fwd, adj, y, lam, np.zeros(shape, complex), np.zeros((2,) + shape, complex),
                                  tau, sigma, K, M)
    plan = cs.Plan(cs.CARTESIAN, shape, 8, mask_idx=t(idx, np.int32))
    x, _ = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_TV,
                          cs.SolveParams(K=K, sketch=False, do_pca=False, cg_iters=M))
    assert nrmse(h(x), x_ref) < 1e-4


def test_coil_sketching_tv_nufft():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    img, grid, C, V, S, T, K, M, lam = (24, 24, 24), (30, 30, 30), 6, 3, 2, 2, 4, 3, 5e-3
    traj = synthdata.cones_trajectory(300, 96)
    dcf = synthdata.cones_dcf(traj, img, 300, 96)
    maps = synthdata.coil_maps(img, C)
    op = nufft.Plan(traj, img, grid)
    y = nufft.sense_fwd(op, synthdata.phantom(img, seed=1), maps, dcf)
    sk = philox.sketch_draw(8, 0, T, C, V, S, dist=1)   # Rademacher, as in the paper's l1-TV experiment
    opsf = lambda m: (lambda v: nufft.sense_fwd(op, v, m, dcf), lambda k: nufft.sense_adj(op, k, m, dcf))
    x_ref, _ = solvers.coil_sketching(opsf, maps, y, lam, "l1tv", sk.astype(np.float64), V=V, K=K, cg_iters=M)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=t(traj), dcf=t(dcf), grid=grid)
    x, _ = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_TV,
                          cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk), cg_iters=M))
    assert nrmse(h(x), x_ref) < 1e-4


@pytest.mark.parametrize("sketch", [True, False])
def test_tv_graph_replay_matches_eager(sketch):
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    shape = (64, 64)
    idx, maps, y, _ = _cart_problem(shape)
    plan = cs.Plan(cs.CARTESIAN, shape, 8, mask_idx=t(idx, np.int32))
    p = dict(T=3, K=5, V=4, S=2, cg_iters=3, sketch=sketch, do_pca=sketch)
    x0, _ = cs.recon_solve(plan, t(y), t(maps), 2e-3, cs.REG_L1_TV, cs.SolveParams(use_graph=False, **p))
    x1, st1 = cs.recon_solve(plan, t(y), t(maps), 2e-3, cs.REG_L1_TV, cs.SolveParams(use_graph=True, **p))
    x2, st2 = cs.recon_solve(plan, t(y), t(maps), 2e-3, cs.REG_L1_TV, cs.SolveParams(use_graph=True, **p))
    assert st1["graph_used"] and st2["graph_used"]
    assert nrmse(h(x1), h(x0)) < 1e-6 and nrmse(h(x2), h(x0)) < 1e-6
