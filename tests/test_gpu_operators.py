"""GPU parity of the SENSE operators (Sec. 2.1, Eq. 1-5) against the FP64 oracle: Cartesian
(2D, several tiles and ragged line blocks) and the Kaiser-Bessel gridding NUFFT (3D), forward,
adjoint, gradient and sketched normal operator; bit-exact binning; adjointness."""
import numpy as np
import pytest
import torch

import synthdata
from oracle import binning, coils, fourier, nufft

pytestmark = pytest.mark.gpu

TOL = 1e-5   # NRMSE per FP32 operator application


@pytest.fixture(scope="module", autouse=True)
def _built():
    from tests._gpu import ensure_built
    ensure_built()


def _cart_case(shape, C, seed, R=4.0):
    mask = synthdata.poisson_disc_mask(shape, R=R, centre=min(24, shape[0] // 4), seed=seed)
    idx = fourier.mask_indices(mask)
    maps = synthdata.coil_maps(shape, C)
    x = synthdata.phantom(shape, seed=seed)
    return idx, maps, x


@pytest.mark.parametrize("shape,C", [((128, 128), 8), ((96, 80), 3), ((160, 120), 5), ((48, 352), 2)])
def test_cartesian_fwd_adj(shape, C):
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    idx, maps, x = _cart_case(shape, C, 3)
    plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=t(idx, np.int32))
    y = cs.sense_fwd(plan, t(x), t(maps))
    y_ref = fourier.cartesian_fwd(x, maps, idx)
    assert nrmse(h(y), y_ref) < TOL
    yy = synthdata.random_complex((C, idx.size), 5)
    xa = cs.sense_adj(plan, t(yy), t(maps))
    xa_ref = fourier.cartesian_adj(yy, maps, idx)
    assert nrmse(h(xa), xa_ref) < TOL
    # accumulate mode adds
    xa2 = cs.sense_adj(plan, t(yy), t(maps), x=xa.clone(), accumulate=True)
    assert nrmse(h(xa2), 2 * xa_ref) < TOL
    # adjointness of the GPU pair
    xg, yg = h(cs.sense_fwd(plan, t(x), t(maps))), yy
    lhs = np.vdot(xg, yg)
    rhs = np.vdot(x, h(cs.sense_adj(plan, t(yy), t(maps))))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_cartesian_grad_and_sketched_normal():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    shape, C, V, S, lam = (128, 128), 8, 2, 2, 1e-3
    idx, maps, x = _cart_case(shape, C, 7)
    y = fourier.cartesian_fwd(synthdata.phantom(shape, seed=8), maps, idx)
    plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=t(idx, np.int32))
    d = cs.sense_grad(plan, t(x), t(maps), t(y))
    d_ref = fourier.cartesian_adj(fourier.cartesian_fwd(x, maps, idx) - y, maps, idx)
    assert nrmse(h(d), d_ref) < TOL
    rng = np.random.default_rng(1)
    S_low = rng.standard_normal((S, C - V))
    msk = coils.sketched_maps(S_low, maps, V)
    z = cs.sketched_normal_apply(plan, t(x), t(msk[:V]), t(msk[V:]), lam)
    z_ref = fourier.cartesian_adj(fourier.cartesian_fwd(x, msk, idx), msk, idx) + lam * x
    assert nrmse(h(z), z_ref) < TOL


def _nufft_case(img, grid, C, n_int, n_read, seed=0):
    traj = synthdata.cones_trajectory(n_int, n_read)
    dcf = synthdata.cones_dcf(traj, img, n_int, n_read)
    maps = synthdata.coil_maps(img, C)
    x = synthdata.phantom(img, seed=seed + 1)
    return traj, dcf, maps, x


@pytest.mark.parametrize("img,grid,C,n_int,tile", [
    ((32, 32, 32), (40, 40, 40), 4, 300, (16, 16, 16)),
    ((16, 24, 32), (20, 30, 40), 3, 200, (8, 8, 16)),
    ((32, 48, 48), (40, 60, 60), 2, 400, (16, 16, 16)),
])
def test_nufft_fwd_adj(img, grid, C, n_int, tile):
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    traj, dcf, maps, x = _nufft_case(img, grid, C, n_int, 128)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=t(traj), dcf=t(dcf), grid=grid, tile=tile)
    op = nufft.Plan(traj, img, grid)
    y = cs.sense_fwd(plan, t(x), t(maps))
    y_ref = nufft.sense_fwd(op, x, maps, dcf)
    assert nrmse(h(y), y_ref) < TOL
    yy = synthdata.random_complex((C, traj.shape[0]), 5)
    xa = cs.sense_adj(plan, t(yy), t(maps))
    xa_ref = nufft.sense_adj(op, yy, maps, dcf)
    assert nrmse(h(xa), xa_ref) < TOL
    lhs = np.vdot(h(y), yy)
    rhs = np.vdot(x, h(xa))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("img,grid,C,spokes", [((240, 240), (300, 300), 5, 96), ((64, 48), (80, 60), 3, 40)])
def test_nufft_2d_fwd_adj(img, grid, C, spokes):
    """2D radial plans: one lane per coil in the gridding kernels; a 300-point grid axis takes
    two 150-row tensor-copy boxes in the strided pass and the 240-row crop one box."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    traj = synthdata.radial_trajectory(spokes, 256)
    dcf = synthdata.radial_dcf(traj, img, spokes, 256)
    maps = synthdata.coil_maps(img, C)
    x = synthdata.phantom(img, seed=4)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=t(traj), dcf=t(dcf), grid=grid)
    op = nufft.Plan(traj, img, grid)
    y = cs.sense_fwd(plan, t(x), t(maps))
    assert nrmse(h(y), nufft.sense_fwd(op, x, maps, dcf)) < TOL
    yy = synthdata.random_complex((C, traj.shape[0]), 6)
    xa = cs.sense_adj(plan, t(yy), t(maps))
    assert nrmse(h(xa), nufft.sense_adj(op, yy, maps, dcf)) < TOL


@pytest.mark.parametrize("C", [7, 33])
def test_nufft_coil_chunks(C):
    """Coil counts that split the gridding into several chunks (33: three chunks of 11 coils)
    and an odd count for the coil-combining pass's chunk choice."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    img, grid = (16, 16, 16), (20, 20, 20)
    traj, dcf, maps, x = _nufft_case(img, grid, C, 60, 64)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=t(traj), dcf=t(dcf), grid=grid)
    op = nufft.Plan(traj, img, grid)
    y = cs.sense_fwd(plan, t(x), t(maps))
    assert nrmse(h(y), nufft.sense_fwd(op, x, maps, dcf)) < TOL
    yy = synthdata.random_complex((C, traj.shape[0]), 7)
    xa = cs.sense_adj(plan, t(yy), t(maps))
    assert nrmse(h(xa), nufft.sense_adj(op, yy, maps, dcf)) < TOL


def test_gridding_parameters_and_autotune():
    """Every gridding configuration the autotuner tries (coils per warp 8 / 16 / 32 for the
    interpolation, 8 / 16 for the spreading, 32 / 64 / 128 samples per warp) against the FP64
    oracle, with 20 coils (chunks of 7, 10 and 20), then the autotuner itself."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    img, grid, C = (16, 16, 16), (20, 20, 20), 20
    traj, dcf, maps, x = _nufft_case(img, grid, C, 80, 64, seed=2)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=t(traj), dcf=t(dcf), grid=grid)
    op = nufft.Plan(traj, img, grid)
    y_ref = nufft.sense_fwd(op, x, maps, dcf)
    yy = synthdata.random_complex((C, traj.shape[0]), 8)
    xa_ref = nufft.sense_adj(op, yy, maps, dcf)
    for ic in (8, 16, 32):
        for sc in (8, 16):
            for k in (32, 64, 128):
                plan.set_gridding(ic, k, sc, k)
                assert nrmse(h(cs.sense_fwd(plan, t(x), t(maps))), y_ref) < TOL, (ic, sc, k)
                assert nrmse(h(cs.sense_adj(plan, t(yy), t(maps))), xa_ref) < TOL, (ic, sc, k)
    # the deterministic (owner-computes) spreading with work items of 64 / 256 / 4096 sample
    # visits: small items split every tile's list into many partial slots added afterwards
    for sc in (8, 16):
        for q in (64, 256, 4096):
            plan.set_gridding(16, 64, sc, 64)
            plan.set_deterministic(True, q)
            assert nrmse(h(cs.sense_adj(plan, t(yy), t(maps))), xa_ref) < TOL, (sc, q)
    plan.set_deterministic(False)
    with pytest.raises(cs.CoilSketchError):
        plan.set_gridding(0, 64, 16, 64)
    with pytest.raises(cs.CoilSketchError):
        plan.set_gridding(16, 64, 32, 64)          # spreading takes at most 16 coils per warp
    with pytest.raises(cs.CoilSketchError):
        plan.set_deterministic(True, 32)           # work items hold at least 64 sample visits
    choice, ms = plan.autotune(C, reps=2)
    assert choice[0] in (8, 16, 32) and choice[2] in (8, 16) and choice[1] in (32, 64, 128) and choice[3] in (32, 64, 128)
    assert all(v > 0 for v in ms) and ms[0] <= ms[2] and ms[1] <= ms[3]
    assert nrmse(h(cs.sense_fwd(plan, t(x), t(maps))), y_ref) < TOL
    assert nrmse(h(cs.sense_adj(plan, t(yy), t(maps))), xa_ref) < TOL


def test_nufft_binning_bit_exact():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t
    img, grid, tile = (32, 32, 32), (40, 40, 40), (16, 8, 16)
    traj = synthdata.cones_trajectory(300, 128)
    # add samples exactly on the edge f = +-0.5 and on grid points
    traj = np.concatenate([traj, np.array([[0.5, -0.5, 0.0], [0.25, 0.125, -0.5], [0, 0, 0]], np.float32)])
    dcf = np.ones(traj.shape[0], np.float32)
    plan = cs.Plan(cs.NONCARTESIAN, img, 1, traj=t(traj), dcf=t(dcf), grid=grid, tile=tile)
    perm, off, j0, nt = plan.binning()
    g = binning.grid_coords(traj, grid)
    j0_ref = binning.kernel_box_start(g)
    perm_ref, off_ref, ntr = binning.sample_order(j0_ref, grid, tile)
    assert tuple(nt) == tuple(int(v) for v in ntr)
    assert np.array_equal(j0.cpu().numpy(), j0_ref)
    assert np.array_equal(perm.cpu().numpy(), perm_ref)
    assert np.array_equal(off.cpu().numpy(), off_ref)


def test_nufft_grad_and_sketched_normal():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    img, grid, C, V, S, lam = (32, 32, 32), (40, 40, 40), 6, 2, 2, 1e-3
    traj, dcf, maps, x = _nufft_case(img, grid, C, 300, 128)
    op = nufft.Plan(traj, img, grid)
    y = nufft.sense_fwd(op, synthdata.phantom(img, seed=9), maps, dcf)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=t(traj), dcf=t(dcf), grid=grid)
    d = cs.sense_grad(plan, t(x), t(maps), t(y))
    d_ref = nufft.sense_adj(op, nufft.sense_fwd(op, x, maps, dcf) - y, maps, dcf)
    assert nrmse(h(d), d_ref) < TOL
    S_low = np.random.default_rng(2).standard_normal((S, C - V))
    msk = coils.sketched_maps(S_low, maps, V)
    z = cs.sketched_normal_apply(plan, t(x), t(msk[:V]), t(msk[V:]), lam)
    z_ref = nufft.sense_adj(op, nufft.sense_fwd(op, x, msk, dcf), msk, dcf) + lam * x
    assert nrmse(h(z), z_ref) < TOL


def test_two_coils_per_lane_gridding_paths():
    """Chunks of 10 .. 16 coils at even offsets run the two-coils-per-lane gridding kernels: forward
    (user-order output), adjoint (user-order input), gradient (residual into the sorted scratch)
    and sketched normal operator (sorted output and input) with 12 and 14 coils against the FP64
    oracle; 13 coils (odd chunk) and 24 coils (chunks of 12) beside them."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    img, grid = (24, 32, 32), (30, 40, 40)
    for C in (12, 13, 14, 24):
        traj, dcf, maps, x = _nufft_case(img, grid, C, 300, 128, seed=C)
        op = nufft.Plan(traj, img, grid)
        plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=t(traj), dcf=t(dcf), grid=grid)
        yy = synthdata.random_complex((C, traj.shape[0]), C + 1)
        assert nrmse(h(cs.sense_fwd(plan, t(x), t(maps))), nufft.sense_fwd(op, x, maps, dcf)) < TOL, C
        assert nrmse(h(cs.sense_adj(plan, t(yy), t(maps))), nufft.sense_adj(op, yy, maps, dcf)) < TOL, C
        d_ref = nufft.sense_adj(op, nufft.sense_fwd(op, x, maps, dcf) - yy, maps, dcf)
        assert nrmse(h(cs.sense_grad(plan, t(x), t(maps), t(yy))), d_ref) < TOL, C
        V = C // 2
        z_ref = nufft.sense_adj(op, nufft.sense_fwd(op, x, maps, dcf), maps, dcf) + 1e-3 * x
        assert nrmse(h(cs.sketched_normal_apply(plan, t(x), t(maps[:V]), t(maps[V:]), 1e-3)), z_ref) < TOL, C


def test_plan_rejects_bad_arguments():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t
    with pytest.raises(cs.CoilSketchError):
        cs.Plan(cs.CARTESIAN, (64, 64), 2, mask_idx=t(np.array([5, 3, 9]), np.int32))       # not ascending
    with pytest.raises(cs.CoilSketchError):
        cs.Plan(cs.CARTESIAN, (64, 62 + 1), 2, mask_idx=t(np.array([1, 2]), np.int32))     # odd size
    with pytest.raises(cs.CoilSketchError):
        cs.Plan(cs.CARTESIAN, (26, 26), 2, mask_idx=t(np.array([1, 2]), np.int32))          # prime 13


@pytest.mark.parametrize("img,grid,tile,item", [((32, 32, 32), (40, 40, 40), (8, 8, 8), 4096),
                                                ((32, 48, 48), (40, 60, 60), (8, 8, 8), 128),
                                                ((16, 16, 32), (20, 18, 40), (8, 8, 16), 300),
                                                ((16, 16, 32), (18, 20, 40), (16, 8, 8), 512)])
def test_deterministic_spreading_is_bit_reproducible(img, grid, tile, item):
    """In the deterministic mode the owner-computes spreading adds every grid point's contributions
    in one fixed order (no atomics): two runs of the adjoint, of the gradient and of the sketched
    normal operator give bit-identical images; with small work items (many partial slots added in
    slot order) too.  The 18-point axis has a last tile of 10 (its 2-point remainder folds into
    it); a z size of 2 mod 4 (the third case's 20 is 0 mod 4, the 18 of the second axis is 2 mod 4)
    exercises the lane mapping choice."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    C = 6
    traj, dcf, maps, x = _nufft_case(img, grid, C, 400, 128, seed=3)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=t(traj), dcf=t(dcf), grid=grid, tile=tile)
    plan.set_deterministic(True, item)
    op = nufft.Plan(traj, img, grid)
    yy = synthdata.random_complex((C, traj.shape[0]), 11)
    a1 = h(cs.sense_adj(plan, t(yy), t(maps)))
    a2 = h(cs.sense_adj(plan, t(yy), t(maps)))
    assert np.array_equal(a1.view(np.uint64), a2.view(np.uint64))
    assert nrmse(a1, nufft.sense_adj(op, yy, maps, dcf)) < TOL
    d1 = h(cs.sense_grad(plan, t(x), t(maps), t(yy)))
    d2 = h(cs.sense_grad(plan, t(x), t(maps), t(yy)))
    assert np.array_equal(d1.view(np.uint64), d2.view(np.uint64))
    z1 = h(cs.sketched_normal_apply(plan, t(x), t(maps[:2]), t(maps[2:5]), 1e-3))
    z2 = h(cs.sketched_normal_apply(plan, t(x), t(maps[:2]), t(maps[2:5]), 1e-3))
    assert np.array_equal(z1.view(np.uint64), z2.view(np.uint64))


def test_retile_matches_a_fresh_plan_and_the_oracle():
    """cs_plan_set_tile re-bins a plan exactly as a plan created with those tiles (same order, bit
    for bit, against the CPU restatement of the sort); the operators stay within the FP64 oracle's
    tolerance for every tile; the tile autotuner returns one of its candidates and leaves the plan
    binned with it; deterministic spreading stays bit-reproducible after a re-binning; a solve with
    a captured graph, re-run after the tiles change, is captured again and agrees with the first."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    img, grid, C = (32, 32, 32), (40, 40, 40), 5
    traj, dcf, maps, x = _nufft_case(img, grid, C, 300, 128, seed=4)
    op = nufft.Plan(traj, img, grid)
    yy = synthdata.random_complex((C, traj.shape[0]), 12)
    adj_ref = nufft.sense_adj(op, yy, maps, dcf)
    fwd_ref = nufft.sense_fwd(op, x, maps, dcf)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=t(traj), dcf=t(dcf), grid=grid)
    j0_ref = binning.kernel_box_start(binning.grid_coords(traj, grid))
    for tile in ((8, 8, 8), (16, 8, 32), (40, 40, 40), (4, 12, 20), (16, 16, 16)):
        plan.set_tile(tile)
        perm, off, j0, nt = plan.binning()
        perm_ref, off_ref, ntr = binning.sample_order(j0_ref, grid, tile)
        assert tuple(nt) == tuple(int(v) for v in ntr), tile
        assert np.array_equal(perm.cpu().numpy(), perm_ref), tile
        assert np.array_equal(off.cpu().numpy(), off_ref), tile
        assert np.array_equal(j0.cpu().numpy(), j0_ref), tile
        assert nrmse(h(cs.sense_adj(plan, t(yy), t(maps))), adj_ref) < TOL, tile
        assert nrmse(h(cs.sense_fwd(plan, t(x), t(maps))), fwd_ref) < TOL, tile
    best, ms = plan.autotune_tile(C, candidates=(8, 16, 32), reps=2)
    assert best in (8, 16, 32) and len(ms) == 3 and all(v > 0 for v in ms)
    assert ms[(8, 16, 32).index(best)] == min(ms)
    perm, off, _, nt = plan.binning()
    perm_ref, off_ref, ntr = binning.sample_order(j0_ref, grid, (best,) * 3)
    assert np.array_equal(perm.cpu().numpy(), perm_ref) and np.array_equal(off.cpu().numpy(), off_ref)
    plan.set_deterministic(True, 256)
    plan.set_tile((8, 16, 8))
    a1 = h(cs.sense_adj(plan, t(yy), t(maps)))
    a2 = h(cs.sense_adj(plan, t(yy), t(maps)))
    assert np.array_equal(a1.view(np.uint64), a2.view(np.uint64))
    assert nrmse(a1, adj_ref) < TOL
    plan.set_deterministic(False)
    y = t(nufft.sense_fwd(op, synthdata.phantom(img, seed=8), maps, dcf))
    res = []
    for tile in ((16, 16, 16), (8, 8, 8)):
        plan.set_tile(tile)
        xs, st = cs.recon_solve(plan, y, t(maps), 1e-3, cs.REG_L2,
                                cs.SolveParams(T=2, K=3, V=2, S=2, seed=3, use_graph=True))
        res.append(h(xs))
    assert nrmse(res[1], res[0]) < 1e-4
    with pytest.raises(cs.CoilSketchError):
        plan.set_tile((2, 8, 8))                    # narrower than the kernel
    with pytest.raises(cs.CoilSketchError):
        plan.autotune_tile(C, candidates=(3,))
