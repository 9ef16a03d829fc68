"""Pins of the l1-TV pieces of the oracle (Sec. 2.1: g(x) = lambda ||T x||_1, T first-order
periodic differences, solved by PDHG whose data step is an l2-regularised least-squares solve)."""
import numpy as np
import pytest

from oracle import solvers, tv, wavelet


def _dense_T(shape):
    """T built entry by entry from its definition: row (a, r) has +1 at r + e_a (mod n), -1 at r."""
    D = int(np.prod(shape))
    nd = len(shape)
    T = np.zeros((nd * D, D))
    for a in range(nd):
        for flat in range(D):
            r = list(np.unravel_index(flat, shape))
            rp = list(r)
            rp[a] = (rp[a] + 1) % shape[a]
            T[a * D + flat, np.ravel_multi_index(rp, shape)] += 1.0
            T[a * D + flat, flat] -= 1.0
    return T


@pytest.mark.parametrize("shape", [(5,), (4, 6), (3, 4, 5)])
def test_tv_matches_dense_definition(shape):
    rng = np.random.default_rng(0)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    z = rng.standard_normal((len(shape),) + shape) + 1j * rng.standard_normal((len(shape),) + shape)
    T = _dense_T(shape)
    assert np.allclose(tv.tv_fwd(x).reshape(-1), T @ x.reshape(-1), atol=1e-13)
    assert np.allclose(tv.tv_adj(z).reshape(-1), T.T @ z.reshape(-1), atol=1e-13)


@pytest.mark.parametrize("shape", [(4, 6), (4, 4, 6)])
def test_tv_norm_is_4_ndim_for_even_sizes(shape):
    T = _dense_T(shape)
    lam_max = np.linalg.eigvalsh(T.T @ T).max()
    assert abs(lam_max - tv.tv_norm_sq(len(shape))) < 1e-10
    # odd sizes stay below the bound
    T3 = _dense_T((3, 5))
    assert np.linalg.eigvalsh(T3.T @ T3).max() < tv.tv_norm_sq(2)


def test_tv_of_constants_vanishes():
    x = np.full((4, 5, 6), 2.0 - 1.5j)
    assert np.abs(tv.tv_fwd(x)).max() == 0
    z = np.stack([np.full((4, 5, 6), 0.3 + 0.1j), np.full((4, 5, 6), -1.0), np.full((4, 5, 6), 2j)])
    assert np.abs(tv.tv_adj(z)).max() < 1e-15


def test_projection_is_moreau_complement_of_soft_threshold():
    # prox of sigma g* (g = lam ||.||_1) = v - sigma prox_{g/sigma}(v/sigma) = v - soft(v, lam)
    rng = np.random.default_rng(1)
    v = 3 * (rng.standard_normal(500) + 1j * rng.standard_normal(500))
    for lam in (0.1, 1.0, 2.5):
        assert np.allclose(tv.project_disc(v, lam), v - wavelet.soft_threshold(v, lam), atol=1e-13)
    assert np.abs(tv.project_disc(v, 0.7)).max() <= 0.7 + 1e-15


def _small_problem(seed=2, shape=(6, 6), M=60):
    rng = np.random.default_rng(seed)
    D = int(np.prod(shape))
    A = (rng.standard_normal((M, D)) + 1j * rng.standard_normal((M, D))) / np.sqrt(M)
    xt = np.zeros(shape)
    xt[1:4, 2:5] = 1.0
    xt = xt + 0.3j * np.roll(xt, 1, axis=0)
    y = A @ xt.reshape(-1) + 0.05 * (rng.standard_normal(M) + 1j * rng.standard_normal(M))
    fwd = lambda v: A @ v.reshape(-1)
    adj = lambda r: (A.conj().T @ r).reshape(shape)
    return A, y, fwd, adj, shape


def _exact_prox(A, y_term, shape, tau):
    D = int(np.prod(shape))
    H = A.conj().T @ A + np.eye(D) / tau
    return lambda v, xw: np.linalg.solve(H, y_term + v.reshape(-1) / tau).reshape(shape)


def test_pdhg_reaches_the_tv_kkt_point():
    A, y, fwd, adj, shape = _small_problem()
    lam = 0.05
    tau, sigma = solvers.pdhg_steps(2)
    prox_f = _exact_prox(A, A.conj().T @ y, shape, tau)
    x, z = solvers.pdhg(prox_f, lam, np.zeros(shape), np.zeros((2,) + shape), tau, sigma, 6000)
    # stationarity A^H (A x - y) + T^H z = 0, dual feasibility |z| <= lam, and z_i = lam Tx_i/|Tx_i|
    g = adj(fwd(x) - y) + tv.tv_adj(z)
    assert np.linalg.norm(g) < 1e-7 * np.linalg.norm(adj(y))
    assert np.abs(z).max() <= lam * (1 + 1e-12)
    Tx = tv.tv_fwd(x)
    big = np.abs(Tx) > 1e-6
    assert big.sum() > 5
    assert np.allclose((np.conj(z) * Tx).real[big], lam * np.abs(Tx[big]), rtol=1e-5)
    # and it minimises the objective against random perturbations
    obj = lambda u: 0.5 * np.linalg.norm(fwd(u) - y) ** 2 + tv.tv_value(u, lam)
    rng = np.random.default_rng(3)
    for _ in range(20):
        dx = 1e-3 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
        assert obj(x) <= obj(x + dx) + 1e-12


def test_sketched_pdhg_with_identity_sketch_solves_the_full_problem():
    # with A_S = A the sub-problem at any x^t equals the full problem up to a constant
    A, y, fwd, adj, shape = _small_problem(seed=4)
    lam = 0.05
    tau, sigma = solvers.pdhg_steps(2)
    x_ref, _ = solvers.pdhg(_exact_prox(A, A.conj().T @ y, shape, tau), lam, np.zeros(shape),
                            np.zeros((2,) + shape), tau, sigma, 6000)
    rng = np.random.default_rng(5)
    xt = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    normal = lambda v: adj(fwd(v))
    d = adj(fwd(xt) - y)
    D = int(np.prod(shape))
    x, _ = solvers.sketched_pdhg(normal, d, xt, lam, np.zeros((2,) + shape), tau, sigma, 6000, D)
    assert solvers.nrmse(x, x_ref) < 1e-6


def test_tv_solution_is_a_fixed_point_of_any_sketched_pdhg_step():
    # x*, z* optimal for the full problem; for any sketched model the sub-problem at x^t = x*
    # (d = A^H (A x* - y)) is optimal at (x*, z*) and PDHG does not move
    A, y, fwd, adj, shape = _small_problem(seed=6)
    lam = 0.05
    tau, sigma = solvers.pdhg_steps(2)
    x_s, z_s = solvers.pdhg(_exact_prox(A, A.conj().T @ y, shape, tau), lam, np.zeros(shape),
                            np.zeros((2,) + shape), tau, sigma, 8000)
    rng = np.random.default_rng(7)
    B = (rng.standard_normal((20, A.shape[1])) + 1j * rng.standard_normal((20, A.shape[1]))) / 5
    normal_S = lambda v: (B.conj().T @ (B @ v.reshape(-1))).reshape(shape)
    d = adj(fwd(x_s) - y)
    D = int(np.prod(shape))
    x, z = solvers.sketched_pdhg(normal_S, d, x_s, lam, z_s, tau, sigma, 50, D)
    assert solvers.nrmse(x, x_s) < 1e-6
    assert np.linalg.norm(z - z_s) < 1e-5 * np.linalg.norm(z_s)


def test_pdhg_steps_satisfy_the_convergence_condition():
    for nd in (2, 3):
        tau, sigma = solvers.pdhg_steps(nd)
        assert tau * sigma * tv.tv_norm_sq(nd) < 1.0


def test_algorithm1_with_pdhg_approaches_the_tv_solution():
    import synthdata
    from oracle import coils, fourier
    shape, C, V, S = (16, 16), 8, 6, 2
    mask = synthdata.poisson_disc_mask(shape, R=2.0, centre=6, seed=2)
    idx = fourier.mask_indices(mask)
    maps = synthdata.coil_maps(shape, C)
    x_true = synthdata.phantom(shape, seed=1)
    y = fourier.cartesian_fwd(x_true, maps, idx)
    lam = 2e-3
    op = lambda m: (lambda v: fourier.cartesian_fwd(v, m, idx), lambda r: fourier.cartesian_adj(r, m, idx))
    fwd, adj = op(maps)
    tau, sigma = solvers.pdhg_steps(2)
    x_ref, _ = solvers.plain_pdhg(fwd, adj, y, lam, np.zeros(shape), np.zeros((2,) + shape), tau, sigma, 1500, 30)
    rng = np.random.default_rng(4)
    sk = rng.standard_normal((8, S, C - V)) / np.sqrt(S)
    x, its = solvers.coil_sketching(op, maps, y, lam, "l1tv", sk, V, 40, do_pca=True, cg_iters=5)
    e = [solvers.nrmse(xi, x_ref) for xi in its]
    assert e[-1] < 0.1 * e[0] and e[-1] < 2e-2
    assert all(b < a * 1.05 for a, b in zip(e, e[1:]))


def test_pdhg_over_relaxation_matches_hand_iterates():
    """Chambolle & Pock with theta = 1 (xbar = 2 x_{k+1} - x_k) on a periodic two-pixel signal,
    f(x) = 1/2 ||x - b||^2 with b = (1, 0) (prox_{tau f}(v) = (v + tau b)/(1 + tau)), lambda = 1/4,
    tau = sigma = 1/2, x_0 = z_0 = 0.  By hand: x_1 = (1/3, 0); xbar_1 = (2/3, 0),
    z_2 = proj((-1/3, 1/3)) = (-1/4, 1/4), T^H z = (1/2, -1/2), x_2 = (7/18, 1/6);
    xbar_2 = (4/9, 1/3), z_3 = (-1/4, 1/4), x_3 = (23/54, 5/18).  Without the over-relaxation
    (xbar = x) z_2 = (-1/6, 1/6) would stay inside the disc and x_2 would differ."""
    b = np.array([1.0, 0.0])
    tau = sigma = 0.5
    prox_f = lambda v, xw: (v + tau * b) / (1 + tau)
    hand = [(1 / 3, 0.0), (7 / 18, 1 / 6), (23 / 54, 5 / 18)]
    for k in range(1, 4):
        x, z = solvers.pdhg(prox_f, 0.25, np.zeros(2, complex), np.zeros((1, 2), complex), tau, sigma, k)
        assert np.abs(x - np.array(hand[k - 1])).max() < 1e-15
    assert np.abs(z[0] - np.array([-0.25, 0.25])).max() < 1e-15
