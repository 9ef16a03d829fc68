"""Solvers and the coil-sketching outer loop (Sec. 2.1, 2.3, Algorithm 1).

Problem (Eq. 3-4): x* = argmin_x 1/2 ||A x - y||^2 + g(x), g = lambda/2 ||x||^2 (solved by CG),
g = lambda ||Psi x||_1 (solved by FISTA) or g = lambda ||T x||_1 (l1-TV, solved by PDHG whose
data step solves an l2-regularised least-squares problem with CG, Sec. 2.1 and Sec. 4).

Sketched sub-problem at outer iteration t (Eq. 9-10, Algorithm 1):
    x^{t+1} = argmin_x 1/2 ||A_S^t (x - x^t)||^2 + Re<x, d> + g(x),  d = A^H (A x^t - y).
The paper writes the inner product for real vectors; for complex images we read it as
Re<x, d>, whose (Wirtinger, A^H-convention) gradient is d.  Hence the sub-problem gradient
is A_S^H A_S (x - x^t) + d (+ lambda x for the l2 regulariser).

Operators are passed as Python callables so the same solver serves the full-coil and the
sketched problems, the Cartesian and the non-Cartesian operator.
"""
from __future__ import annotations

import numpy as np

from . import coils, tv, wavelet


def vdot(a, b):
    """<a, b> = sum conj(a) b in complex128."""
    return np.vdot(np.asarray(a, dtype=np.complex128).ravel(), np.asarray(b, dtype=np.complex128).ravel())


def nrmse(x, ref):
    """||x - ref||_2 / ||ref||_2 (the normalised distance of Sec. 3.3)."""
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(np.asarray(ref).ravel()))


def cg(H, b, x0, iters):
    """Hestenes-Stiefel conjugate gradients on H x = b (H Hermitian positive definite)."""
    x = np.array(x0, dtype=np.complex128, copy=True)
    r = b - H(x)
    p = r.copy()
    rr = vdot(r, r).real
    for _ in range(iters):
        if rr == 0:
            break
        Hp = H(p)
        alpha = rr / vdot(p, Hp).real
        x = x + alpha * p
        r = r - alpha * Hp
        rr_new = vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def power_iteration(H, v0, iters=20):
    """Largest eigenvalue of Hermitian PSD H: v <- H v / ||H v||, L = ||H v|| at the last step."""
    return power_iteration_vec(H, v0, iters)[0]


def power_iteration_vec(H, v0, iters):
    """The power iteration of power_iteration, returning (L, v) with v the last normalised iterate."""
    v = np.asarray(v0, dtype=np.complex128)
    v = v / np.linalg.norm(v.ravel())
    L = 0.0
    for _ in range(iters):
        w = H(v)
        L = float(np.linalg.norm(w.ravel()))
        v = w / L
    return L, v


def fista(grad, prox, x0, eta, iters):
    """FISTA (Beck & Teboulle 2009) from z_0 = x_0, t_0 = 1:
    x_k = prox(z_{k-1} - eta grad(z_{k-1})), t_k = (1 + sqrt(1 + 4 t_{k-1}^2))/2,
    z_k = x_k + ((t_{k-1} - 1)/t_k)(x_k - x_{k-1})."""
    x_prev = np.array(x0, dtype=np.complex128, copy=True)
    z = x_prev.copy()
    t = 1.0
    for _ in range(iters):
        x = prox(z - eta * grad(z))
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        z = x + ((t - 1.0) / t_new) * (x - x_prev)
        x_prev = x
        t = t_new
    return x_prev


def pdhg(prox_f, lam, x0, z0, tau, sigma, iters):
    """Primal-dual hybrid gradient (Chambolle & Pock 2011, their Algorithm 1 with theta = 1) on
    min_x f(x) + lam ||T x||_1:
        z_{k+1} = proj_lam(z_k + sigma T xbar_k)
        x_{k+1} = prox_{tau f}(x_k - tau T^H z_{k+1}, warm start x_k)
        xbar_{k+1} = 2 x_{k+1} - x_k,          xbar_0 = x_0.
    Returns (x_K, z_K)."""
    x = np.array(x0, dtype=np.complex128, copy=True)
    z = np.array(z0, dtype=np.complex128, copy=True)
    xbar = x.copy()
    for _ in range(iters):
        z = tv.project_disc(z + sigma * tv.tv_fwd(xbar), lam)
        x_new = prox_f(x - tau * tv.tv_adj(z), x)
        xbar = 2.0 * x_new - x
        x = x_new
    return x, z


def pdhg_steps(ndim):
    """Default step sizes (reading; the paper gives none): tau = sigma = 0.99 / ||T||, so that
    tau sigma ||T||^2 < 1 as PDHG's convergence requires."""
    s = 0.99 / np.sqrt(tv.tv_norm_sq(ndim))
    return float(s), float(s)


# ---------------------------------------------------------------------------------------
# Sub-problem solvers (Eq. 9-10)

def sketched_cg(normal_S, d, xt, lam, iters):
    """l2 sub-problem: (A_S^H A_S + lam I) x = A_S^H A_S x^t - d, CG from x^t."""
    H = lambda v: normal_S(v) + lam * v
    b = normal_S(xt) - d
    return cg(H, b, xt, iters)


def sketched_fista(normal_S, d, xt, lam, eta, iters, levels=4):
    """l1-wavelet sub-problem by FISTA from x^t: grad = A_S^H A_S (z - x^t) + d."""
    grad = lambda z: normal_S(z - xt) + d
    prox = lambda v: wavelet.prox_l1_wavelet(v, eta * lam, levels)
    return fista(grad, prox, xt, eta, iters)


def sketched_pdhg(normal_S, d, xt, lam, z0, tau, sigma, iters, cg_iters):
    """l1-TV sub-problem by PDHG from x^t.  f(x) = 1/2 ||A_S (x - x^t)||^2 + Re<x, d>, so
    prox_{tau f}(v) solves (A_S^H A_S + I/tau) x = A_S^H A_S x^t - d + v/tau, here by
    ``cg_iters`` CG iterations started at the current primal iterate.  The dual variable z is
    passed in and returned (carried from one sub-problem to the next)."""
    b0 = normal_S(xt) - d
    H = lambda v: normal_S(v) + v / tau
    prox_f = lambda v, xw: cg(H, b0 + v / tau, xw, cg_iters)
    return pdhg(prox_f, lam, xt, z0, tau, sigma, iters)


def plain_pdhg(fwd, adj, y, lam, x0, z0, tau, sigma, iters, cg_iters):
    """Full-coil l1-TV by PDHG: prox_{tau f}(v) solves (A^H A + I/tau) x = A^H y + v/tau by CG."""
    b0 = adj(y)
    H = lambda v: adj(fwd(v)) + v / tau
    prox_f = lambda v, xw: cg(H, b0 + v / tau, xw, cg_iters)
    return pdhg(prox_f, lam, x0, z0, tau, sigma, iters)


def plain_cg(fwd, adj, y, lam, x0, iters):
    """Full-coil l2 problem: (A^H A + lam I) x = A^H y."""
    H = lambda v: adj(fwd(v)) + lam * v
    return cg(H, adj(y), x0, iters)


def plain_fista(fwd, adj, y, lam, eta, x0, iters, levels=4):
    grad = lambda z: adj(fwd(z) - y)
    prox = lambda v: wavelet.prox_l1_wavelet(v, eta * lam, levels)
    return fista(grad, prox, x0, eta, iters)


# ---------------------------------------------------------------------------------------
# Comparators of Sec. 3.3: aggressive coil compression and AccProxSGD

def coil_compressed(op_factory, maps, y, keep, solve):
    """Coil PCA, keep the first ``keep`` virtual coils, then ``solve(fwd, adj, y_keep)``."""
    U, _ = coils.coil_pca(y)
    maps_r = coils.rotate(U, maps)[:keep]
    y_r = coils.rotate(U, y)[:keep]
    fwd, adj = op_factory(maps_r)
    return solve(fwd, adj, y_r)


def acc_prox_sgd(op_factory, maps, y, lam, batches, alpha0, beta, min_frac, x0, iters, levels=4):
    """Accelerated proximal stochastic gradient over coils (Sec. 3.3; coil batches of size B):
        g_k = (C/B) sum_{c in batch k} A_c^H (A_c z_k - y_c)          (unbiased for the full gradient)
        alpha_k = max(beta^k alpha0, min_frac alpha0)                (the paper's decreasing rule)
        x_{k+1} = prox_{alpha_k lam ||Psi .||_1}(z_k - alpha_k g_k)
        z_{k+1} = x_{k+1} + ((t_k - 1)/t_{k+1}) (x_{k+1} - x_k)       (Nesterov / FISTA momentum)
    batches: int [iters, B] coil indices (given as inputs)."""
    C = maps.shape[0]
    batches = np.asarray(batches)
    B = batches.shape[1]
    x_prev = np.array(x0, dtype=np.complex128, copy=True)
    z = x_prev.copy()
    t = 1.0
    for k in range(iters):
        idx = batches[k]
        fwd, adj = op_factory(maps[idx])
        g = (C / B) * adj(fwd(z) - y[idx])
        alpha = max(beta ** k * alpha0, min_frac * alpha0)
        x = wavelet.prox_l1_wavelet(z - alpha * g, alpha * lam, levels)
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        z = x + ((t - 1.0) / t_new) * (x - x_prev)
        x_prev = x
        t = t_new
    return x_prev


# ---------------------------------------------------------------------------------------
# Algorithm 1

def coil_sketching(op_factory, maps, y, lam, reg, sketches, V, K, x0=None, eta=None,
                   power_v0=None, power_iters=20, do_pca=True, levels=4, callback=None,
                   cg_iters=5, tau=None, sigma=None, init_sketch=None, step_per_outer=0, L_out=None):
    """Algorithm 1, optionally with its classical-sketch initialisation.

    op_factory(maps) -> (fwd, adj) builds A for a set of maps (Cartesian or NUFFT).
    sketches: float [T, S, C-V] random blocks S~_S^t (given as inputs).
    reg: 'l2' (CG, K iterations), 'l1wav' (FISTA, K iterations, step eta; if eta is None it
    is 1/L with L from ``power_iters`` power iterations on the first sketched normal operator,
    started at power_v0, and reused for every sub-problem) or 'l1tv' (PDHG, K iterations with
    ``cg_iters`` CG iterations in each data step, steps tau/sigma (default ``pdhg_steps``); the
    dual variable starts at zero and is carried from one sub-problem to the next).
    init_sketch: optional random block S~_S^0 [S, C-V] of the initialisation, which solves
    argmin_x 1/2 ||S^0 A x - S^0 y||^2 + g(x) from x^0 with the sub-problem's solver and K
    iterations.  That problem is the sketched sub-problem at x^t = x^0 with the sketched
    gradient d = (S^0 A)^H (S^0 A x^0 - S^0 y) in place of the true one (its objective differs
    from the sub-problem's by a constant), so the same solver routine runs it.  The FISTA step
    1/L comes from the first model built (the initialisation's when there is one).
    step_per_outer > 0 (FISTA with eta None; not in the paper, whose Sec. 3.3 reuses the first
    step): every outer iteration re-estimates L with that many further power iterations on its
    own sketched normal operator, continuing from the previous eigenvector estimate; L_out (a
    list) receives the L of every outer iteration's step.
    Returns x^T and the list of iterates (the initialisation's result not included).
    """
    if do_pca:
        U, _ = coils.coil_pca(y)
        maps_r = coils.rotate(U, maps)
        y_r = coils.rotate(U, y)
    else:
        maps_r, y_r = maps, y
    fwd, adj = op_factory(maps_r)
    x = np.zeros(maps.shape[1:], dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    iterates = []
    if reg == "l1tv":
        t0, s0 = pdhg_steps(x.ndim)
        tau = t0 if tau is None else tau
        sigma = s0 if sigma is None else sigma
        zdual = np.zeros((x.ndim,) + x.shape, dtype=np.complex128)
    veig = None
    steps = [("init", init_sketch)] if init_sketch is not None else []
    steps += [("outer", sketches[t]) for t in range(sketches.shape[0])]
    for kind, S_t in steps:
        msk = coils.sketched_maps(S_t, maps_r, V)               # sketched model A_S^t
        fs, ads = op_factory(msk)
        normal_S = lambda v: ads(fs(v))
        if kind == "init":
            d = ads(fs(x) - coils.sketch_data(S_t, y_r, V))     # sketched gradient at x^0
        else:
            d = adj(fwd(x) - y_r)                               # true gradient
        if reg == "l2":
            x = sketched_cg(normal_S, d, x, lam, K)
        elif reg == "l1tv":
            x, zdual = sketched_pdhg(normal_S, d, x, lam, zdual, tau, sigma, K, cg_iters)
        else:
            if eta is None or (step_per_outer and veig is None):
                L, veig = power_iteration_vec(normal_S, power_v0, power_iters)
                eta = 1.0 / L
            if step_per_outer and kind == "outer":
                L, veig = power_iteration_vec(normal_S, veig, step_per_outer)
                eta = 1.0 / L
            if L_out is not None and kind == "outer":
                L_out.append(1.0 / eta)
            x = sketched_fista(normal_S, d, x, lam, eta, K, levels)
        if kind == "outer":
            iterates.append(x.copy())
            if callback is not None:
                callback(len(iterates) - 1, x)
    return x, iterates
