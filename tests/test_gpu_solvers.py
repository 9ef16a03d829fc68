"""GPU parity of the solvers: db4 wavelet transform and soft threshold, CG / FISTA sub-problems
inside Algorithm 1, and the plain full-coil solvers, against the FP64 oracle run with the same
inputs and the same sketch matrices (final-image NRMSE <= 1e-4)."""
import numpy as np
import pytest
import torch

import synthdata
from oracle import fourier, nufft, philox, solvers, wavelet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from tests._gpu import ensure_built
    ensure_built()


@pytest.mark.parametrize("shape,levels", [((64, 96), 3), ((128, 128), 4), ((32, 64, 48), 2), ((16, 32, 64), 1)])
def test_wavelet_matches_oracle(shape, levels):
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    x = synthdata.random_complex(shape, 4)
    c = cs.wavelet_fwd(t(x), levels)
    assert nrmse(h(c), wavelet.wavedec(x, levels)) < 1e-6
    xr = cs.wavelet_inv(c, levels)
    assert nrmse(h(xr), x) < 1e-6
    z = synthdata.random_complex(shape, 5)
    zz = cs.soft_threshold_(t(z), 0.8)
    assert nrmse(h(zz), wavelet.soft_threshold(z.astype(np.complex64), 0.8)) < 1e-6


def _cart_problem(shape=(128, 128), C=8, R=4.0, seed=1):
    mask = synthdata.poisson_disc_mask(shape, R=R, centre=24, seed=2)
    idx = fourier.mask_indices(mask)
    maps = synthdata.coil_maps(shape, C)
    x_true = synthdata.phantom(shape, seed=seed)
    y = fourier.cartesian_fwd(x_true, maps, idx)
    y = y + synthdata.complex_noise(y.shape, 1e-3 * np.abs(y).max(), seed=3)
    ops = lambda m: (lambda v: fourier.cartesian_fwd(v, m, idx), lambda k: fourier.cartesian_adj(k, m, idx))
    return idx, maps, y, ops


def test_coil_sketching_cg_cartesian():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    idx, maps, y, ops = _cart_problem()
    C, V, S, T, K, lam = 8, 4, 2, 4, 10, 1e-2
    sk = philox.sketch_draw(4, 0, T, C, V, S)
    x_ref, its = solvers.coil_sketching(ops, maps, y, lam, "l2", sk.astype(np.float64), V=V, K=K)
    plan = cs.Plan(cs.CARTESIAN, (128, 128), C, mask_idx=t(idx, np.int32))
    iters = torch.empty((T, 128, 128), dtype=torch.complex64, device="cuda")
    x, st = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L2,
                           cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk), iterates=iters))
    assert nrmse(h(x), x_ref) < 1e-4
    for k in range(T):
        assert nrmse(h(iters[k]), its[k]) < 1e-4


def test_plain_cg_and_fista_cartesian():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    idx, maps, y, ops = _cart_problem(shape=(64, 64))
    fwd, adj = ops(maps)
    plan = cs.Plan(cs.CARTESIAN, (64, 64), 8, mask_idx=t(idx, np.int32))
    x_ref = solvers.plain_cg(fwd, adj, y, 1e-3, np.zeros((64, 64), complex), 15)
    x, _ = cs.recon_solve(plan, t(y), t(maps), 1e-3, cs.REG_L2, cs.SolveParams(K=15, sketch=False, do_pca=False))
    assert nrmse(h(x), x_ref) < 1e-4
    v0 = synthdata.random_complex((64, 64), 5)
    L = solvers.power_iteration(lambda v: adj(fwd(v)), v0, 20)
    x_ref = solvers.plain_fista(fwd, adj, y, 5e-3, 1 / L, np.zeros((64, 64), complex), 20, levels=3)
    x, st = cs.recon_solve(plan, t(y), t(maps), 5e-3, cs.REG_L1_WAVELET,
                           cs.SolveParams(K=20, sketch=False, do_pca=False, power_v0=t(v0)), wavelet_levels=3)
    assert abs(st["L"] - L) < 1e-5 * L
    assert nrmse(h(x), x_ref) < 1e-4


def test_coil_sketching_cg_bf16_split_maps():
    """Algorithm 1 with the sketched maps contracted on the tensor cores (BF16 split) stays
    within the final-image tolerance of the FP64 oracle."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    idx, maps, y, ops = _cart_problem()
    C, V, S, T, K, lam = 8, 4, 2, 4, 10, 1e-2
    sk = philox.sketch_draw(4, 0, T, C, V, S)
    x_ref, _ = solvers.coil_sketching(ops, maps, y, lam, "l2", sk.astype(np.float64), V=V, K=K)
    plan = cs.Plan(cs.CARTESIAN, (128, 128), C, mask_idx=t(idx, np.int32))
    x, _ = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L2,
                          cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk), precision=cs.PREC_BF16_SPLIT))
    assert nrmse(h(x), x_ref) < 1e-4


def test_coil_sketching_fista_cartesian():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    shape = (128, 128)
    idx, maps, y, ops = _cart_problem(shape, C=8)
    C, V, S, T, K, lam = 8, 3, 3, 3, 8, 5e-3
    sk = philox.sketch_draw(11, 0, T, C, V, S)
    v0 = synthdata.random_complex(shape, 5)
    x_ref, _ = solvers.coil_sketching(ops, maps, y, lam, "l1wav", sk.astype(np.float64), V=V, K=K, power_v0=v0)
    plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=t(idx, np.int32))
    x, _ = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_WAVELET,
                          cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk), power_v0=t(v0)))
    assert nrmse(h(x), x_ref) < 1e-4


@pytest.mark.parametrize("use_graph", [False, True])
def test_coil_sketching_fista_with_the_step_re_estimated_every_outer_iteration(use_graph):
    """step_per_outer = 4: every outer iteration continues the power iteration on its own sketched
    operator and uses 1/L_t; the trace's step field matches the oracle's L_t, and every iterate
    and the final image match the oracle run with the same option."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    shape = (128, 128)
    idx, maps, y, ops = _cart_problem(shape, C=8)
    C, V, S, T, K, lam = 8, 3, 3, 4, 8, 5e-3
    sk = philox.sketch_draw(12, 0, T, C, V, S)
    v0 = synthdata.random_complex(shape, 6)
    L_ref = []
    x_ref, its = solvers.coil_sketching(ops, maps, y, lam, "l1wav", sk.astype(np.float64), V=V, K=K, power_v0=v0,
                                        step_per_outer=4, L_out=L_ref)
    assert np.ptp(L_ref) > 1e-3 * max(L_ref)          # the blocks' operators do differ
    plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=t(idx, np.int32))
    iters = torch.empty((T,) + shape, dtype=torch.complex64, device="cuda")
    x, st = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_WAVELET,
                           cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk), power_v0=t(v0), step_per_outer=4,
                                          iterates=iters, trace=True, use_graph=use_graph))
    assert np.allclose(st["trace"][:, cs.TRACE_STEP_L], L_ref, rtol=1e-5, atol=0)
    assert nrmse(h(x), x_ref) < 1e-4
    for k in range(T):
        assert nrmse(h(iters[k]), its[k]) < 1e-4
    with pytest.raises(cs.CoilSketchError):          # needs FISTA with the step from power iterations
        cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L2,
                       cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk), step_per_outer=4))


def test_coil_sketching_cg_nufft():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    img, grid, C, V, S, T, K, lam = (32, 32, 32), (40, 40, 40), 8, 4, 2, 3, 8, 1e-2
    traj = synthdata.cones_trajectory(400, 128)
    dcf = synthdata.cones_dcf(traj, img, 400, 128)
    maps = synthdata.coil_maps(img, C)
    op = nufft.Plan(traj, img, grid)
    y = nufft.sense_fwd(op, synthdata.phantom(img, seed=1), maps, dcf)
    sk = philox.sketch_draw(4, 0, T, C, V, S)
    opsf = lambda m: (lambda v: nufft.sense_fwd(op, v, m, dcf), lambda k: nufft.sense_adj(op, k, m, dcf))
    x_ref, _ = solvers.coil_sketching(opsf, maps, y, lam, "l2", sk.astype(np.float64), V=V, K=K)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=t(traj), dcf=t(dcf), grid=grid)
    x, _ = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L2, cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk)))
    assert nrmse(h(x), x_ref) < 1e-4


def test_nonfinite_input_is_reported():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t
    idx, maps, y, _ = _cart_problem(shape=(64, 64))
    y = y.copy()
    y[0, 3] = np.nan
    plan = cs.Plan(cs.CARTESIAN, (64, 64), 8, mask_idx=t(idx, np.int32))
    with pytest.raises(cs.CoilSketchError) as e:
        cs.recon_solve(plan, t(y), t(maps), 1e-3, cs.REG_L2, cs.SolveParams(K=3, sketch=False, do_pca=False))
    assert e.value.code == 5


@pytest.mark.parametrize("reg,sketch", [("l2", True), ("l1", True), ("l2", False), ("l1", False)])
def test_graph_replay_matches_eager(reg, sketch):
    """use_graph captures one outer iteration (or one plain iteration), caches it in the plan and
    replays it; results equal the eagerly launched solve and a second call reuses the graph."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    idx, maps, y, _ = _cart_problem(shape=(64, 64))
    C, V, S, T, K = 8, 4, 2, 3, 6
    v0 = t(synthdata.random_complex((64, 64), 5))
    regc = cs.REG_L2 if reg == "l2" else cs.REG_L1_WAVELET
    plan = cs.Plan(cs.CARTESIAN, (64, 64), C, mask_idx=t(idx, np.int32))
    yt, mt = t(y), t(maps)
    sk = t(philox.sketch_draw(4, 0, T, C, V, S))
    iters_e = torch.zeros((max(T, K), 64, 64), dtype=torch.complex64, device="cuda")
    iters_g = torch.zeros_like(iters_e)
    kw = dict(T=T, K=K, V=V, S=S, sketch=sketch, sketches=sk, power_v0=v0, do_pca=sketch)
    x_e, st_e = cs.recon_solve(plan, yt, mt, 5e-3, regc, cs.SolveParams(iterates=iters_e, **kw), wavelet_levels=3)
    x_g, st_g = cs.recon_solve(plan, yt, mt, 5e-3, regc, cs.SolveParams(iterates=iters_g, use_graph=True, **kw),
                               wavelet_levels=3)
    assert st_e["graph_used"] == 0 and st_g["graph_used"] == 1
    assert nrmse(h(x_g), h(x_e)) < 1e-6
    assert nrmse(h(iters_g), h(iters_e)) < 1e-6
    # the cached graph is replayed on an identical call
    x_g2, st_g2 = cs.recon_solve(plan, yt, mt, 5e-3, regc, cs.SolveParams(iterates=iters_g, use_graph=True, **kw),
                                 wavelet_levels=3)
    assert st_g2["graph_used"] == 1 and nrmse(h(x_g2), h(x_e)) < 1e-6
    # a different lambda is a different graph
    x_l, _ = cs.recon_solve(plan, yt, mt, 1e-2, regc, cs.SolveParams(use_graph=True, **kw), wavelet_levels=3)
    x_le, _ = cs.recon_solve(plan, yt, mt, 1e-2, regc, cs.SolveParams(**kw), wavelet_levels=3)
    assert nrmse(h(x_l), h(x_le)) < 1e-6


@pytest.mark.parametrize("reg", ["l1", "l2"])
def test_batched_slices_match_individual_solves(reg):
    """recon_solve_batched (eager fork/join and one captured graph for all slices) gives the same
    images as solving every slice on its own."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    regc = cs.REG_L2 if reg == "l2" else cs.REG_L1_WAVELET
    C = 8
    items, refs = [], []
    for k, n in enumerate([64, 96, 80, 128]):
        shape = (n, n)
        mask = synthdata.line_mask(shape, R=4.0, centre_lines=12, seed=20 + k)
        idx = fourier.mask_indices(mask)
        maps = synthdata.coil_maps(shape, C)
        y = fourier.cartesian_fwd(synthdata.phantom(shape, seed=30 + k), maps, idx)
        plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=t(idx, np.int32))
        v0 = t(synthdata.random_complex(shape, 40 + k))
        items.append(dict(plan=plan, y=t(y), maps=t(maps), power_v0=v0))
    params = dict(T=3, K=5, V=3, S=3, seed=9)
    for it in items:
        x, _ = cs.recon_solve(it["plan"], it["y"], it["maps"], 5e-3, regc,
                              cs.SolveParams(power_v0=it["power_v0"], **params), wavelet_levels=2)
        refs.append(h(x))
    for g in (False, True, True):
        xs, sts = cs.recon_solve_batched(items, 5e-3, regc, cs.SolveParams(use_graph=g, **params), wavelet_levels=2)
        for x, r, s in zip(xs, refs, sts):
            assert nrmse(h(x), r) < 1e-6
            assert s["graph_used"] == int(g)


@pytest.mark.parametrize("reg", ["l2", "l1wav", "l1tv"])
def test_coil_sketching_with_classical_sketch_initialisation(reg):
    """Algorithm 1 with its classical-sketch initialisation (sketch block T) against the oracle,
    for the CG, FISTA (step from the initialisation's model) and PDHG sub-problem solvers."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    shape = (64, 64)
    idx, maps, y, ops = _cart_problem(shape, C=8)
    C, V, S, T, K, M = 8, 4, 2, 3, 6, 4
    lam = {"l2": 1e-2, "l1wav": 5e-3, "l1tv": 2e-3}[reg]
    code = {"l2": cs.REG_L2, "l1wav": cs.REG_L1_WAVELET, "l1tv": cs.REG_L1_TV}[reg]
    sk = philox.sketch_draw(9, 0, T + 1, C, V, S)
    v0 = synthdata.random_complex(shape, 5)
    x_ref, its = solvers.coil_sketching(ops, maps, y, lam, reg, sk[:T].astype(np.float64), V=V, K=K, power_v0=v0,
                                        levels=3, cg_iters=M, init_sketch=sk[T].astype(np.float64))
    plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=t(idx, np.int32))
    iters = torch.empty((T,) + shape, dtype=torch.complex64, device="cuda")
    x, _ = cs.recon_solve(plan, t(y), t(maps), lam, code,
                          cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk), power_v0=t(v0), cg_iters=M, init=True,
                                         iterates=iters), wavelet_levels=3)
    assert nrmse(h(x), x_ref) < 1e-4
    for k in range(T):
        assert nrmse(h(iters[k]), its[k]) < 1e-4


def test_aggressive_coil_compression_matches_oracle():
    """Plain FISTA on the first C^ virtual coils after coil PCA (the comparator of Sec. 3.3)."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    shape = (64, 64)
    idx, maps, y, ops = _cart_problem(shape, C=8)
    keep, K, lam = 4, 15, 1e-2
    v0 = synthdata.random_complex(shape, 5)

    def solve(f, a, yk):
        L = solvers.power_iteration(lambda v: a(f(v)), v0, 20)
        return solvers.plain_fista(f, a, yk, lam, 1 / L, np.zeros(shape, complex), K, levels=3)

    x_ref = solvers.coil_compressed(ops, maps, y, keep, solve)
    plan = cs.Plan(cs.CARTESIAN, shape, 8, mask_idx=t(idx, np.int32))
    x, _ = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_WAVELET,
                          cs.SolveParams(K=K, sketch=False, do_pca=True, keep=keep, power_v0=t(v0)), wavelet_levels=3)
    assert nrmse(h(x), x_ref) < 1e-4


@pytest.mark.parametrize("use_graph", [False, True])
def test_acc_prox_sgd_matches_oracle(use_graph):
    """AccProxSGD with given coil batches against the oracle (coil PCA off: batches index the
    caller's coils)."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    shape = (64, 64)
    idx, maps, y, ops = _cart_problem(shape, C=8)
    B, K, lam, beta, floor = 3, 14, 5e-3, 0.95, 0.2
    rng = np.random.default_rng(9)
    batches = np.stack([rng.permutation(8)[:B] for _ in range(K)]).astype(np.int32)
    v0 = synthdata.random_complex(shape, 5)
    fwd, adj = ops(maps)
    L = solvers.power_iteration(lambda v: adj(fwd(v)), v0, 20)
    x_ref = solvers.acc_prox_sgd(ops, maps, y, lam, batches, 1 / L, beta, floor, np.zeros(shape, complex), K, levels=3)
    plan = cs.Plan(cs.CARTESIAN, shape, 8, mask_idx=t(idx, np.int32))
    prm = cs.SolveParams(K=K, sketch=False, do_pca=False, sgd_batch=B, sgd_coils=t(batches, np.int32), sgd_beta=beta,
                         sgd_min=floor, power_v0=t(v0), use_graph=use_graph)
    x, st = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_WAVELET, prm, wavelet_levels=3)
    assert abs(st["L"] - L) < 1e-5 * L
    assert nrmse(h(x), x_ref) < 1e-4
    bad = batches.copy()
    bad[3, 1] = 8
    with pytest.raises(cs.CoilSketchError):
        cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_WAVELET,
                       cs.SolveParams(K=K, sketch=False, do_pca=False, sgd_batch=B, sgd_coils=t(bad, np.int32),
                                      power_v0=t(v0)), wavelet_levels=3)


def test_trace_records_match_the_oracle():
    """The per-outer trace of Algorithm 1 (FISTA, graph and eager) against the FP64 oracle on the
    same inputs: ||d^t||^2 of the true gradient at every x^t, the objective 1/2 ||A x^t - y||^2 +
    lambda ||Psi x^t||_1, the distance of every iterate to a reference, no warm start (-1), and an
    increasing device clock; the plain solver's trace records its iterate distances."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    shape, levels = (64, 64), 3
    idx, maps, y, ops = _cart_problem(shape, C=8)
    C, V, S, T, K, lam = 8, 3, 3, 4, 6, 5e-3
    sk = philox.sketch_draw(11, 0, T, C, V, S)
    v0 = synthdata.random_complex(shape, 5)
    x_ref, its = solvers.coil_sketching(ops, maps, y, lam, "l1wav", sk.astype(np.float64), V=V, K=K, power_v0=v0,
                                        levels=levels)
    fwd, adj = ops(maps)
    starts = [np.zeros(shape, complex)] + its[:-1]
    g2 = [np.linalg.norm(adj(fwd(u) - y)) ** 2 for u in starts]
    obj = [0.5 * np.linalg.norm(fwd(u) - y) ** 2 + lam * np.abs(wavelet.wavedec(u, levels)).sum() for u in starts]
    ref = synthdata.random_complex(shape, 9)
    dist = [np.linalg.norm(u - ref) ** 2 / np.linalg.norm(ref) ** 2 for u in its]
    plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=t(idx, np.int32))
    for graph in (False, True):
        x, st = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_WAVELET,
                               cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk), power_v0=t(v0), use_graph=graph,
                                              x_ref=t(ref), trace=True, trace_objective=True), wavelet_levels=levels)
        tr = st["trace"]
        assert nrmse(h(x), x_ref) < 1e-4
        assert tr.shape == (T, cs.TRACE_FIELDS)
        assert np.allclose(tr[:, cs.TRACE_GRAD2], g2, rtol=1e-4)
        assert np.allclose(tr[:, cs.TRACE_OBJECTIVE], obj, rtol=1e-5)
        assert np.all(tr[:, cs.TRACE_ACCEPT] == -1)
        assert np.allclose(tr[:, cs.TRACE_DIST2], dist, rtol=1e-4)
        assert np.all(np.diff(tr[:, cs.TRACE_TIME_NS]) > 0)
        assert np.all(tr[:, cs.TRACE_STEP_L] == st["L"])       # the first sub-problem's step, reused
    # without the objective flag the field stays NaN; without x_ref the distance is -1
    _, st = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_WAVELET,
                           cs.SolveParams(T=T, K=K, V=V, S=S, sketches=t(sk), power_v0=t(v0), trace=True),
                           wavelet_levels=levels)
    assert np.isnan(st["trace"][:, cs.TRACE_OBJECTIVE]).all() and np.all(st["trace"][:, cs.TRACE_DIST2] == -1)
    # plain FISTA: one record per iteration, distances of the stored iterates
    Kp = 7
    iters = torch.empty((Kp,) + shape, dtype=torch.complex64, device="cuda")
    _, st = cs.recon_solve(plan, t(y), t(maps), lam, cs.REG_L1_WAVELET,
                           cs.SolveParams(K=Kp, sketch=False, do_pca=False, power_v0=t(v0), iterates=iters,
                                          x_ref=t(ref), trace=True), wavelet_levels=levels)
    hi = h(iters)
    want = [np.linalg.norm(hi[k] - ref) ** 2 / np.linalg.norm(ref) ** 2 for k in range(Kp)]
    assert np.allclose(st["trace"][:, cs.TRACE_DIST2], want, rtol=1e-5)
    assert np.all(st["trace"][:, cs.TRACE_GRAD2] > 0)


def test_batched_slices_of_the_2d_workload_match_the_oracle():
    """The batched 2D workload's slice shapes against the FP64 oracle: one recon_solve_batched call
    (one captured graph) with 288^2, 352^2 and 384^2 slices, 16 coils, line masks R = 6 with 24
    centre lines, l1-db4 lambda 5e-3 by FISTA, m = 6 = 3 PCA + 3 Gaussian; every slice's final
    image within 1e-4 of oracle.solvers.coil_sketching on the same inputs and sketch blocks."""
    import paper_2305_06482_gb300 as cs
    from tests._gpu import t, h, nrmse
    C, V, S, T, K, lam, seed = 16, 3, 3, 4, 8, 5e-3, 9
    sk = philox.sketch_draw(seed, 0, T, C, V, S).astype(np.float64)
    items, refs = [], []
    for k, n in enumerate((288, 352, 384)):
        shape = (n, n)
        mask = synthdata.line_mask(shape, R=6.0, centre_lines=24, seed=60 + k)
        idx = fourier.mask_indices(mask)
        maps = synthdata.coil_maps(shape, C)
        y = fourier.cartesian_fwd(synthdata.phantom(shape, seed=70 + k), maps, idx)
        y = y + synthdata.complex_noise(y.shape, 1e-3 * np.abs(y).max(), seed=75 + k)
        v0 = synthdata.random_complex(shape, 80 + k)
        ops = lambda m, idx=idx: (lambda v: fourier.cartesian_fwd(v, m, idx), lambda r: fourier.cartesian_adj(r, m, idx))
        x_ref, _ = solvers.coil_sketching(ops, maps, y, lam, "l1wav", sk, V=V, K=K, power_v0=v0, levels=4)
        refs.append(x_ref)
        plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=t(idx, np.int32))
        items.append(dict(plan=plan, y=t(y), maps=t(maps), power_v0=t(v0)))
    xs, sts = cs.recon_solve_batched(items, lam, cs.REG_L1_WAVELET,
                                     cs.SolveParams(T=T, K=K, V=V, S=S, seed=seed, use_graph=True), wavelet_levels=4)
    for x, r, st in zip(xs, refs, sts):
        assert nrmse(h(x), r) < 1e-4
        assert st["graph_used"] == 1
