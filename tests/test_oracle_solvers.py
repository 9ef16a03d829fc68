"""Pins for CG, FISTA, power iteration, the sketched sub-problem (Eq. 9-10) and Algorithm 1:
direct dense solves, the identity-sketch Newton step, the fixed point of every sketched step,
the CG first-residual identity, eigvalsh, and prox-gradient optimality."""
import numpy as np

import synthdata
from oracle import coils, fourier, nufft, solvers, wavelet, philox


def _cart_problem(shape=(8, 8), C=4, seed=0, frac=0.5):
    rng = np.random.default_rng(seed)
    maps = synthdata.coil_maps(shape, C)
    idx = fourier.mask_indices(rng.random(shape) < frac)
    xt = synthdata.phantom(shape, seed=1)
    y = fourier.cartesian_fwd(xt, maps, idx) + synthdata.complex_noise((C, idx.size), 1e-3, seed=3)
    return maps, idx, y


def _ops(idx):
    return lambda m: (lambda v: fourier.cartesian_fwd(v, m, idx), lambda k: fourier.cartesian_adj(k, m, idx))


def _dense(maps, idx):
    return fourier.dense_sense_matrix(maps, fourier.sampled_frequencies(maps.shape[1:], idx))


def test_cg_reaches_the_direct_normal_equation_solution():
    maps, idx, y = _cart_problem()
    lam = 1e-2
    A = _dense(maps, idx)
    xs = np.linalg.solve(A.conj().T @ A + lam * np.eye(64), A.conj().T @ y.ravel())
    fwd, adj = _ops(idx)(maps)
    x = solvers.plain_cg(fwd, adj, y, lam, np.zeros((8, 8), complex), 200)
    assert np.abs(x.ravel() - xs).max() <= 1e-10 * np.abs(xs).max()


def test_identity_sketch_gives_the_full_newton_step():
    maps, idx, y = _cart_problem(seed=4)
    lam = 1e-2
    C = maps.shape[0]
    A = _dense(maps, idx)
    xs = np.linalg.solve(A.conj().T @ A + lam * np.eye(64), A.conj().T @ y.ravel())
    x, _ = solvers.coil_sketching(_ops(idx), maps, y, lam, "l2", np.zeros((1, 0, 0)), V=C, K=300, do_pca=False)
    assert np.abs(x.ravel() - xs).max() <= 1e-10 * np.abs(xs).max()


def test_full_solution_is_a_fixed_point_of_every_sketched_step():
    maps, idx, y = _cart_problem(seed=5)
    lam = 1e-2
    A = _dense(maps, idx)
    xs = np.linalg.solve(A.conj().T @ A + lam * np.eye(64), A.conj().T @ y.ravel()).reshape(8, 8)
    fwd, adj = _ops(idx)(maps)
    d = adj(fwd(xs) - y)
    assert np.abs(d + lam * xs).max() <= 1e-10 * np.abs(xs).max()        # d = -lam x*
    rng = np.random.default_rng(6)
    for _ in range(3):
        S_low = rng.standard_normal((2, 2))
        msk = coils.sketched_maps(S_low, maps, 2)
        fs, ads = _ops(idx)(msk)
        x1 = solvers.sketched_cg(lambda v: ads(fs(v)), d, xs, lam, 20)
        assert np.abs(x1 - xs).max() <= 1e-10 * np.abs(xs).max()


def test_cg_first_residual_is_minus_full_gradient():
    maps, idx, y = _cart_problem(seed=7)
    lam = 1e-2
    fwd, adj = _ops(idx)(maps)
    xt = synthdata.random_complex((8, 8), 8)
    d = adj(fwd(xt) - y)
    msk = coils.sketched_maps(np.random.default_rng(9).standard_normal((2, 2)), maps, 2)
    fs, ads = _ops(idx)(msk)
    n = lambda v: ads(fs(v))
    r0 = (n(xt) - d) - (n(xt) + lam * xt)
    assert np.abs(r0 + d + lam * xt).max() <= 1e-12 * np.abs(d).max()


def test_power_iteration_matches_eigvalsh():
    _, idx, _ = _cart_problem(seed=10, C=3)
    maps = synthdata.random_complex((3, 8, 8), 10)        # unnormalised maps: a clear spectral gap
    A = _dense(maps, idx)
    ev = np.linalg.eigvalsh(A.conj().T @ A)
    fwd, adj = _ops(idx)(maps)
    L = solvers.power_iteration(lambda v: adj(fwd(v)), synthdata.random_complex((8, 8), 11), 200)
    assert abs(L - ev[-1]) <= 1e-6 * ev[-1]


def test_fista_converges_to_a_prox_gradient_fixed_point():
    maps, idx, y = _cart_problem(shape=(16, 16), seed=12)
    lam = 5e-3
    fwd, adj = _ops(idx)(maps)
    L = solvers.power_iteration(lambda v: adj(fwd(v)), synthdata.random_complex((16, 16), 13), 100)
    eta = 1 / L
    x = solvers.plain_fista(fwd, adj, y, lam, eta, np.zeros((16, 16), complex), 3000, levels=2)
    step = wavelet.prox_l1_wavelet(x - eta * adj(fwd(x) - y), eta * lam, 2)
    assert np.abs(step - x).max() <= 1e-8


def test_coil_sketching_converges_to_the_full_solution():
    shape = (16, 16)
    C = 8
    maps, idx, y = _cart_problem(shape=shape, C=C, seed=14, frac=0.4)
    lam = 1e-2
    A = _dense(maps, idx)
    xs = np.linalg.solve(A.conj().T @ A + lam * np.eye(256), A.conj().T @ y.ravel()).reshape(shape)
    # V = 4 high-energy virtual coils + S = 2 Gaussian combinations of the other 4: the
    # sketched Hessian is accurate enough for the geometric convergence of the iterative
    # Hessian sketch (Sec. 2.2)
    sk = philox.sketch_draw(99, 0, 20, C, 4, 2)
    errs = []
    solvers.coil_sketching(_ops(idx), maps, y, lam, "l2", sk, V=4, K=40,
                           callback=lambda t, x: errs.append(solvers.nrmse(x, xs)))
    assert errs[-1] < 1e-10 and errs[-1] < errs[0] * 1e-6, errs
    assert all(b < a for a, b in zip(errs[:8], errs[1:9]))


def test_classical_sketch_initialisation_with_identity_sketch_is_the_plain_solver():
    """Algorithm 1's initialisation solves 1/2 ||S^0 A x - S^0 y||^2 + g(x); with the identity
    sketch (V = C) that is the full problem, so with CG it must equal K plain CG iterations from
    x^0, and the outer loop then continues from that point."""
    import synthdata
    from oracle import fourier
    shape, C, K, lam = (16, 16), 4, 6, 1e-2
    mask = synthdata.poisson_disc_mask(shape, R=2.0, centre=6, seed=2)
    idx = fourier.mask_indices(mask)
    maps = synthdata.coil_maps(shape, C)
    y = fourier.cartesian_fwd(synthdata.phantom(shape, seed=1), maps, idx)
    ops = lambda m: (lambda v: fourier.cartesian_fwd(v, m, idx), lambda r: fourier.cartesian_adj(r, m, idx))
    fwd, adj = ops(maps)
    x0 = synthdata.random_complex(shape, 3) * 0.1
    x_plain = solvers.plain_cg(fwd, adj, y, lam, x0, K)
    empty = np.zeros((0, 0))
    x_init_only, its = solvers.coil_sketching(ops, maps, y, lam, "l2", np.zeros((0, 0, 0)), C, K, x0=x0,
                                              do_pca=False, init_sketch=empty)
    assert its == [] and solvers.nrmse(x_init_only, x_plain) < 1e-10
    # the initialisation uses the sketched data S^0 y: a random-block sketch changes the result
    rng = np.random.default_rng(0)
    blk = rng.standard_normal((2, C - 2))
    x_sk, _ = solvers.coil_sketching(ops, maps, y, lam, "l2", np.zeros((0, 2, C - 2)), 2, K, x0=x0,
                                     do_pca=False, init_sketch=blk)
    fs, ads = ops(coils.sketched_maps(blk, maps, 2))
    ys = coils.sketch_data(blk, y, 2)
    x_direct = solvers.cg(lambda v: ads(fs(v)) + lam * v, ads(ys), x0, K)
    assert solvers.nrmse(x_sk, x_direct) < 1e-10


def _tiny_cart(shape=(16, 16), C=4, seed=1):
    mask = synthdata.poisson_disc_mask(shape, R=2.0, centre=6, seed=2)
    idx = fourier.mask_indices(mask)
    maps = synthdata.coil_maps(shape, C)
    y = fourier.cartesian_fwd(synthdata.phantom(shape, seed=seed), maps, idx)
    ops = lambda m: (lambda v: fourier.cartesian_fwd(v, m, idx), lambda r: fourier.cartesian_adj(r, m, idx))
    return maps, y, ops


def test_acc_prox_sgd_with_full_batches_is_fista():
    maps, y, ops = _tiny_cart()
    fwd, adj = ops(maps)
    C, K, lam = 4, 12, 5e-3
    L = solvers.power_iteration(lambda v: adj(fwd(v)), synthdata.random_complex((16, 16), 5), 30)
    x0 = np.zeros((16, 16), complex)
    full = np.tile(np.arange(C), (K, 1))
    x_sgd = solvers.acc_prox_sgd(ops, maps, y, lam, full, 1 / L, 1.0, 0.1, x0, K, levels=2)
    x_fista = solvers.plain_fista(fwd, adj, y, lam, 1 / L, x0, K, levels=2)
    assert solvers.nrmse(x_sgd, x_fista) < 1e-12


def test_coil_batch_gradient_is_unbiased():
    from itertools import combinations
    maps, y, ops = _tiny_cart(C=5)
    fwd, adj = ops(maps)
    z = synthdata.random_complex((16, 16), 6)
    full = adj(fwd(z) - y)
    B = 2
    subsets = list(combinations(range(5), B))
    mean = np.zeros_like(full)
    for sb in subsets:
        f, a = ops(maps[list(sb)])
        mean += (5 / B) * a(f(z) - y[list(sb)])
    mean /= len(subsets)
    assert solvers.nrmse(mean, full) < 1e-12


def test_coil_compression_keeping_every_coil_is_the_plain_solver():
    maps, y, ops = _tiny_cart()
    fwd, adj = ops(maps)
    x0 = np.zeros((16, 16), complex)
    ref = solvers.plain_cg(fwd, adj, y, 1e-2, x0, 10)
    got = solvers.coil_compressed(ops, maps, y, 4, lambda f, a, yk: solvers.plain_cg(f, a, yk, 1e-2, x0, 10))
    assert solvers.nrmse(got, ref) < 1e-10
    fewer = solvers.coil_compressed(ops, maps, y, 2, lambda f, a, yk: solvers.plain_cg(f, a, yk, 1e-2, x0, 10))
    assert solvers.nrmse(fewer, ref) > 1e-3          # dropping virtual coils changes the solution


def test_algorithm_1_resumes_from_an_outer_iterate():
    """Algorithm 1 depends on the past only through x^t and the sketch sequence (counter-based
    on (seed, t)): stopping after t outer iterations and restarting from x^t with the remaining
    sketch blocks reproduces the uninterrupted run exactly (CG and FISTA with a given step)."""
    maps, idx, y = _cart_problem(shape=(16, 16), C=6, seed=7)
    C, V, S, T = 6, 2, 2, 5
    sk = philox.sketch_draw(11, 0, T, C, V, S)
    for reg, extra in (("l2", {}), ("l1wav", {"eta": 0.3, "levels": 2})):
        x_full, its_full = solvers.coil_sketching(_ops(idx), maps, y, 1e-2, reg, sk, V, 4, **extra)
        x_2, its_a = solvers.coil_sketching(_ops(idx), maps, y, 1e-2, reg, sk[:2], V, 4, **extra)
        x_res, its_b = solvers.coil_sketching(_ops(idx), maps, y, 1e-2, reg, sk[2:], V, 4, x0=x_2, **extra)
        assert np.array_equal(x_res, x_full), reg
        assert all(np.array_equal(a, b) for a, b in zip(its_a + its_b, its_full)), reg
        # and the sketch blocks of a resumed run are the uninterrupted run's, drawn from (seed, t)
        assert np.array_equal(philox.sketch_draw(11, 2, T - 2, C, V, S), sk[2:])


# ---------------------------------------------------------------------------------------
# Iterates worked out by hand from the published recursions, so that a wrong momentum index,
# step schedule or extrapolation (which still converges to the same fixed point) fails.

def test_fista_momentum_matches_hand_iterates():
    """Beck & Teboulle (2009) on f(x) = 1/2 (x - 1)^2 with eta = 1/2 from x_0 = 0.  Worked by
    hand: t_0 = 1, t_1 = (1 + sqrt 5)/2, t_2 = (1 + sqrt(7 + 2 sqrt 5))/2 = 2.1935270853...;
    identity prox: x_1 = 1/2 (momentum (t_0 - 1)/t_1 = 0, so z_1 = x_1), x_2 = 3/4,
    z_2 = 3/4 + (t_1 - 1)/t_2 (1/4) = 0.8204383812..., x_3 = (z_2 + 1)/2 = 0.9102191906...;
    ridge prox v / (1 + eta) (prox of eta x^2/2): x_1 = 1/3, x_2 = 4/9, x_3 = 0.4919167972..."""
    grad = lambda z: z - 1.0
    one = np.zeros(1, complex)
    hand_id = [0.5, 0.75, 0.9102191906406651]
    hand_ridge = [1 / 3, 4 / 9, 0.49191679722686373]
    for k in range(1, 4):
        got = solvers.fista(grad, lambda v: v, one, 0.5, k)
        assert abs(got[0] - hand_id[k - 1]) < 1e-15
        got = solvers.fista(grad, lambda v: v / 1.5, one, 0.5, k)
        assert abs(got[0] - hand_ridge[k - 1]) < 1e-15


def test_acc_prox_sgd_step_schedule_matches_hand_iterates():
    """AccProxSGD with a decaying step (beta = 1/2 < 1) and its floor (min_frac = 1/5) on two
    image-domain coils A_c = m_c I, m = (1, 2), data y_c = m_c (x = 1), batches of one coil
    alternating 0, 1, 0, 1, lambda = 0 (identity prox), alpha_0 = 1/10.  By hand:
    alpha_k = 1/10, 1/20, 1/40, then the floor 1/50; g_k = (C/B) m_c^2 (z_k - 1);
    x_1 = 1/5, x_2 = 13/25, x_3 = 0.6296530716..., x_4 = 0.7288876446..."""
    m = np.array([1.0, 2.0])
    maps = m[:, None, None] * np.ones((2, 4, 4))
    y = maps.copy().astype(complex)
    ops = lambda mm: (lambda v: mm * v, lambda r: np.sum(np.conj(mm) * r, axis=0))
    batches = np.array([[0], [1], [0], [1]])
    hand = [0.2, 0.52, 0.62965307163809753, 0.72888764463353636]
    for k in range(1, 5):
        x = solvers.acc_prox_sgd(ops, maps, y, 0.0, batches[:k], 0.1, 0.5, 0.2, np.zeros((4, 4), complex), k,
                                 levels=1)
        assert np.abs(x - hand[k - 1]).max() < 1e-13


def test_per_outer_step_tracks_each_sketched_operators_largest_eigenvalue():
    """With step_per_outer the FISTA step of every outer iteration is 1/L_t, L_t from power
    iterations on that iteration's own sketched normal operator continued from the previous
    eigenvector.  Image-domain coils A_c = diag(m_c) make A_S^H A_S = diag(sum_i |m~_i|^2), whose
    largest eigenvalue is the largest diagonal entry; the maps give one voxel a clear lead, so the
    power iteration converges and L_t must equal that entry of each sketch block (blocks differing
    from one another).  The first L_t is the first model's power iteration run power_iters +
    step_per_outer times; without the option the first step is reused."""
    rng = np.random.default_rng(8)
    C, V, S, T = 4, 2, 1, 3
    maps = rng.uniform(0.2, 1.0, (C, 4, 4)) * np.exp(1j * rng.uniform(0, 2 * np.pi, (C, 4, 4)))
    maps[0, 0, 0] = 3.0
    ops = lambda mm: (lambda v: mm * v, lambda r: np.sum(np.conj(mm) * r, axis=0))
    y = ops(maps)[0](synthdata.phantom((4, 4), seed=2))
    sk = rng.standard_normal((T, S, C - V))
    v0 = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    diag = [np.sum(np.abs(coils.sketched_maps(sk[t], maps, V)) ** 2, axis=0) for t in range(T)]
    for w in diag:
        top2 = np.sort(w.ravel())[-2:]
        assert top2[0] < 0.7 * top2[1] and np.argmax(w) == 0
    eig = [w.max() for w in diag]
    assert np.ptp(eig) > 1e-2 * max(eig)
    Ls = []
    solvers.coil_sketching(ops, maps, y, 1e-2, "l1wav", sk, V, 2, power_v0=v0, power_iters=20, do_pca=False,
                           levels=1, step_per_outer=200, L_out=Ls)
    assert np.allclose(Ls, eig, rtol=1e-12, atol=0)
    L1 = []
    solvers.coil_sketching(ops, maps, y, 1e-2, "l1wav", sk, V, 2, power_v0=v0, power_iters=20, do_pca=False,
                           levels=1, step_per_outer=3, L_out=L1)
    fs, ads = ops(coils.sketched_maps(sk[0], maps, V))
    assert L1[0] == solvers.power_iteration(lambda v: ads(fs(v)), v0, 23)
    L0 = []
    solvers.coil_sketching(ops, maps, y, 1e-2, "l1wav", sk, V, 2, power_v0=v0, power_iters=20, do_pca=False,
                           levels=1, L_out=L0)
    assert L0 == [L0[0]] * T and L0[0] == solvers.power_iteration(lambda v: ads(fs(v)), v0, 20)
