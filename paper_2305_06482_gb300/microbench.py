"""Micro-benchmarks of single operators on synthetic inputs (CUDA-event timing on the current
stream), for profiling individual kernels with small launch counts.

  python -m paper_2305_06482_gb300.microbench nufft  [--config cones3d_128|cones3d_large] [--warmup W] [--iters N] [--tile T] [--autotune] [--autotune-tile]
      multicoil NUFFT forward (sense_fwd) and adjoint (sense_adj), all coils (optionally after
      cs_plan_autotune_tile has chosen the binning tile among 8, 12, 16, 24, 32 and / or
      cs_plan_autotune the gridding launch parameters for all coils)
  python -m paper_2305_06482_gb300.microbench normal [--config cones3d_128|cones3d_large] [--warmup W] [--iters N] [--tile T] [--autotune-tile]
      sketched normal operator A_S^H A_S v + lambda v with V = 5 unsketched and S = 5 sketched coils
      (the inner-iteration operator of the sketched sub-problem), with the per-stage device times
  python -m paper_2305_06482_gb300.microbench tv [--config cones3d_128|cones3d_large] [--iters N]
      l1-TV by PDHG (data step: 5 CG iterations) on the cones workload, lambda 0.01: one coil-
      sketched reconstruction (m = 4 = 3 PCA + 1 Rademacher, T = 3 outer x K = 10 PDHG) and 10
      PDHG iterations of the plain full-coil solver, with the time per PDHG iteration of each
  python -m paper_2305_06482_gb300.microbench ablation [--seeds R]
      sketching-matrix design sweep on 2D radial data (256x256, 8 coils, 201 golden-angle spokes
      x 256 = R 2 against 402 Nyquist spokes, noise 1e-3 max|y|, l1-db4 lambda 2e-3): for
      C^ = 3 and 4, V = 0 .. C^, Gaussian (variance 1/S), Rademacher and the literal Gaussian
      scaling (sigma = 1/S), R seeds each, coil sketching T = 10 x K = 10 FISTA; objective and
      NRMSE to the phantom normalised by the full-coil solution's (mean and std over seeds)
  python -m paper_2305_06482_gb300.microbench gfactor [--replicas 60]
      inverse g-factor by pseudo-replicas: 256x256 Cartesian, 8 coils, every third line (R 3),
      noise 1e-2 max|y|, l2 lambda 1e-3: the full-coil CG solver (30 iterations) on fully and
      regularly undersampled data, and coil sketching (C^ 4 = 3 + 1 Rademacher, T 5 x K 10 CG)
      on the undersampled data, each as one batched solve of all replicas in one CUDA graph
  python -m paper_2305_06482_gb300.microbench compare [--config cones3d_128|cones3d_large]
      the method against the comparators of its evaluation on the cones workload (l1-db4,
      lambda 2e-3): full-coil FISTA, aggressive coil compression to 8 virtual coils (lambda
      halved, as the evaluation re-tuned it), AccProxSGD with batches of 8 coils (beta 0.99,
      floor 0.1) and coil sketching (m = 8 = 7 PCA + 1 Rademacher, K = 10); distance to x_inf
      (300 full-coil FISTA iterations) against device time, and the time to reach 5%
  python -m paper_2305_06482_gb300.microbench sketch [--voxels D] [--iters N]
      sketched maps (40 coils, V = 5, S = 5): FP32 CUDA cores vs BF16 split on the tensor cores
  python -m paper_2305_06482_gb300.microbench batched [--slices 64] [--iters N]
      64 2D Cartesian slices of uneven size (256..384 squared), 16 coils, line mask R = 6 with
      24 centre lines, l1-db4 FISTA (lambda 5e-3), sketch m = 6 (3 PCA + 3 Gaussian), T = 10, K = 10:
      one slice after another vs all slices forked and joined vs all slices in one CUDA graph
  python -m paper_2305_06482_gb300.microbench recon [--config cones3d_128|cones3d_large] [--outer T] [--K K] [--tile T]
      one coil-sketched reconstruction in the benchmark's configuration (T outer x K inner FISTA,
      m = 10, BF16-split maps), no reference solve: the kernel mix of the timed reconstruction
  python -m paper_2305_06482_gb300.microbench warmnet [--config cones3d_128|cones3d_large] [--iters N]
      the warm-start U-Net (16/32/64 channels): every 3x3x3 convolution alone on random inputs of
      its shape (BF16 implicit GEMM on the tensor cores), one whole inference on the image size of
      the workload, and one training step (forward, backward, Adam) on a 64^3 crop
  python -m paper_2305_06482_gb300.microbench warmtrain [--config cones3d_128|cones3d_large] [--phantoms P]
          [--outer T] [--K K] [--tight M] [--train-steps N] [--crops Q] [--ref-iters R] [--save PATH]
      the warm start trained on the method's own pairs: (x^t, d, sub-problem solved with M FISTA
      iterations) from T outer iterations of Algorithm 1 (K inner) on P seeded phantoms (l1-db4
      lambda 2e-3, m = 8 = 4 PCA + 4 Gaussian on cones3d_128, m = 10 = 5 + 5 on cones3d_large),
      N Adam steps on random 64^3 crops (with Q > 0: on Q stored crops drawn once), optionally
      saved; then a held-out phantom through
      recon_solve with and without the warm start (decision on the device): NRMSE to x_inf (R
      plain iterations) per outer iteration, acceptances, device time per reconstruction
  python -m paper_2305_06482_gb300.microbench cart2d [--iters N]
      128x128 Cartesian coil-sketched CG reconstruction (8 coils, m = 4, T = 5, K = 10),
      eager launches vs a replayed CUDA graph
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_2305_06482_gb300 as cs  # noqa: E402
import synthdata  # noqa: E402

CONFIGS = {
    "cones3d_128": dict(img=(128, 128, 128), grid=(160, 160, 160), nc=32, n_int=6000),
    "cones3d_large": dict(img=(160, 256, 256), grid=(200, 320, 320), nc=40, n_int=20000),
}


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


TILE_CANDIDATES = (8, 12, 16, 24, 32)


def _tiles(args):
    return tuple(int(v) for v in args.tiles.split(",")) if args.tiles else TILE_CANDIDATES


def _tile_tune(plan, C, cands=TILE_CANDIDATES):
    best, ms = plan.autotune_tile(C, cands)
    print(f"tile autotune for {C} coils (interp + spread ms per round): "
          + ", ".join(f"{t}^3 {m:.3f}" for t, m in zip(cands, ms)) + f" -> {best}^3", flush=True)


def nufft(args):
    cfg = CONFIGS[args.config]
    dev = torch.device("cuda")
    img, grid, C = cfg["img"], cfg["grid"], cfg["nc"]
    traj = synthdata.cones_trajectory(cfg["n_int"], 512)
    dcf = synthdata.cones_dcf(traj, img, cfg["n_int"], 512)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=torch.from_numpy(traj).to(dev), dcf=torch.from_numpy(dcf).to(dev),
                   grid=grid)
    x = synthdata.phantom_torch(img, seed=1, device=dev)
    maps = synthdata.coil_maps_torch(img, C, device=dev)
    y = torch.empty((C, traj.shape[0]), dtype=torch.complex64, device=dev)
    xa = torch.empty(img, dtype=torch.complex64, device=dev)
    if args.tile:
        plan.set_tile((args.tile,) * 3)
    if args.autotune_tile:
        _tile_tune(plan, C, _tiles(args))
    if args.autotune:
        choice, ms = plan.autotune(C)
        print(f"autotune for {C} coils: interp {choice[0]} coils x {choice[1]} samples per warp "
              f"({ms[2]:.3f} -> {ms[0]:.3f} ms per launch), spread {choice[2]} x {choice[3]} "
              f"({ms[3]:.3f} -> {ms[1]:.3f} ms)")
    for _ in range(args.warmup):
        cs.sense_fwd(plan, x, maps, y)
        cs.sense_adj(plan, y, maps, xa)
    torch.cuda.synchronize()
    a, b = _events()
    c, d = _events()
    a.record()
    for _ in range(args.iters):
        cs.sense_fwd(plan, x, maps, y)
    b.record()
    for _ in range(args.iters):
        cs.sense_adj(plan, y, maps, xa)
    d.record()
    torch.cuda.synchronize()
    f = a.elapsed_time(b) / args.iters
    g = b.elapsed_time(d) / args.iters
    D, G, N = int(np.prod(img)), int(np.prod(grid)), traj.shape[0]
    model = 2 * C * (8 * D + 48 * G + 8 * N) + 2 * (16 * N + 16 * D)
    print(f"{args.config}: forward {f:.3f} ms, adjoint {g:.3f} ms, fwd+adj model bytes {model / 1e9:.2f} GB "
          f"-> {model / ((f + g) * 1e-3) / 1e9:.0f} GB/s")


def normal(args):
    cfg = CONFIGS[args.config]
    dev = torch.device("cuda")
    img, grid, C = cfg["img"], cfg["grid"], cfg["nc"]
    V, S = 5, 5
    traj = synthdata.cones_trajectory(cfg["n_int"], 512)
    dcf = synthdata.cones_dcf(traj, img, cfg["n_int"], 512)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=torch.from_numpy(traj).to(dev), dcf=torch.from_numpy(dcf).to(dev),
                   grid=grid)
    v = synthdata.phantom_torch(img, seed=1, device=dev)
    maps = synthdata.coil_maps_torch(img, V + S, device=dev)
    mv, ms = maps[:V].contiguous(), maps[V:].contiguous()
    z = torch.empty(img, dtype=torch.complex64, device=dev)
    if args.tile:
        plan.set_tile((args.tile,) * 3)
    if args.autotune_tile:
        _tile_tune(plan, V + S, _tiles(args))
    for _ in range(args.warmup):
        cs.sketched_normal_apply(plan, v, mv, ms, 1e-3, z)
    torch.cuda.synchronize()
    a, b = _events()
    a.record()
    for _ in range(args.iters):
        cs.sketched_normal_apply(plan, v, mv, ms, 1e-3, z)
    b.record()
    torch.cuda.synchronize()
    ms_ = a.elapsed_time(b) / args.iters
    cs.profile(True)
    for _ in range(args.iters):
        cs.sketched_normal_apply(plan, v, mv, ms, 1e-3, z)
    torch.cuda.synchronize()
    st = {k: cs.profile_read(k) for k in ("spread", "interp", "fft_plain", "expand", "reduce")}
    cs.profile(False)
    parts = ", ".join(f"{k} {t / args.iters:.3f} ms" for k, (t, n) in st.items() if n)
    print(f"{args.config}: sketched normal apply (V={V}, S={S}): {ms_:.3f} ms; per stage: {parts}")


def tv(args):
    cfg = CONFIGS[args.config]
    dev = torch.device("cuda")
    img, grid, C = cfg["img"], cfg["grid"], cfg["nc"]
    traj = synthdata.cones_trajectory(cfg["n_int"], 512)
    dcf = synthdata.cones_dcf(traj, img, cfg["n_int"], 512)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=torch.from_numpy(traj).to(dev), dcf=torch.from_numpy(dcf).to(dev),
                   grid=grid)
    maps = synthdata.coil_maps_torch(img, C, device=dev)
    y = cs.sense_fwd(plan, synthdata.phantom_torch(img, seed=1, device=dev), maps)
    lam, T, K, M = 1e-2, 3, 10, 5
    sk = cs.SolveParams(T=T, K=K, V=3, S=1, dist=cs.RADEMACHER, cg_iters=M, seed=4)
    pl = cs.SolveParams(K=K, sketch=False, do_pca=False, cg_iters=M)
    res = {}
    for name, prm in (("sketched", sk), ("plain", pl)):
        cs.recon_solve(plan, y, maps, lam, cs.REG_L1_TV, prm)            # warm-up
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        for _ in range(args.iters):
            cs.recon_solve(plan, y, maps, lam, cs.REG_L1_TV, prm)
        b.record()
        torch.cuda.synchronize()
        res[name] = a.elapsed_time(b) / args.iters
    print(f"{args.config}: l1-TV PDHG, lambda {lam}, {M} CG iterations per data step")
    print(f"  sketched recon (m=4, T={T}, K={K}): {res['sketched']:.1f} ms = "
          f"{res['sketched'] / (T * K):.2f} ms per PDHG iteration (incl. PCA, sketches, true gradients)")
    print(f"  plain full-coil ({C} coils), {K} PDHG iterations: {res['plain']:.1f} ms = "
          f"{res['plain'] / K:.2f} ms per PDHG iteration")


def ablation(args):
    dev = torch.device("cuda")
    img, grid, C, spokes, n_read, lam, levels = (256, 256), (320, 320), 8, 201, 256, 2e-3, 4
    traj = synthdata.radial_trajectory(spokes, n_read)
    dcf = synthdata.radial_dcf(traj, img, spokes, n_read)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=torch.from_numpy(traj).to(dev), dcf=torch.from_numpy(dcf).to(dev),
                   grid=grid)
    maps = torch.from_numpy(synthdata.coil_maps(img, C).astype(np.complex64)).to(dev)
    x_true = torch.from_numpy(synthdata.phantom(img, seed=1).astype(np.complex64)).to(dev)
    y = cs.sense_fwd(plan, x_true, maps)
    noise = synthdata.complex_noise(tuple(y.shape), 1e-3 * float(y.abs().max()), seed=3)
    y = y + torch.from_numpy(noise.astype(np.complex64)).to(dev)
    v0 = torch.from_numpy(synthdata.random_complex(img, 5).astype(np.complex64)).to(dev)
    yy = 0.5 * float(torch.sum(y.real.double() ** 2 + y.imag.double() ** 2))
    d0 = cs.sense_adj(plan, y, maps)
    d0 = -d0
    zero = torch.zeros(img, dtype=torch.complex64, device=dev)

    def objective(x):   # 1/2 ||A x - y||^2 + lambda ||Psi x||_1 (sub-problem objective at x^t = 0, d = -A^H y)
        return cs.subproblem_objective(plan, x, zero, d0, maps, None, lam, cs.REG_L1_WAVELET, levels) + yy

    def err(x):
        return float(torch.linalg.vector_norm(x - x_true) / torch.linalg.vector_norm(x_true))

    t0 = time.perf_counter()
    x_base, _ = cs.recon_solve(plan, y, maps, lam, cs.REG_L1_WAVELET,
                               cs.SolveParams(K=300, sketch=False, do_pca=False, power_v0=v0), wavelet_levels=levels)
    f_base, e_base = objective(x_base), err(x_base)
    print(f"2D radial 256^2, 8 coils, {spokes} spokes: full-coil FISTA (300 it) objective {f_base:.6g}, "
          f"NRMSE to phantom {e_base:.4f}")
    designs = [("gauss", cs.GAUSSIAN, cs.NORM_UNIT_VAR), ("rademacher", cs.RADEMACHER, cs.NORM_UNIT_VAR),
               ("gauss-literal", cs.GAUSSIAN, cs.NORM_PAPER_LITERAL)]
    print("C^  V  S  distribution     f/f_full mean  std       NRMSE/NRMSE_full mean  std")
    for Ch in (3, 4):
        for V in range(0, Ch + 1):
            for name, dist, norm in designs:
                if V == Ch and name != "gauss":
                    continue                       # S = 0: no random block
                fs, es = [], []
                for seed in range(args.seeds):
                    try:
                        x, _ = cs.recon_solve(plan, y, maps, lam, cs.REG_L1_WAVELET,
                                              cs.SolveParams(T=10, K=10, V=V, S=Ch - V, dist=dist, norm=norm,
                                                             seed=1000 + seed, power_v0=v0), wavelet_levels=levels)
                        f, e = objective(x), err(x)
                    except cs.CoilSketchError:       # a diverged solve reports a non-finite reduction
                        f, e = np.inf, np.inf
                    fs.append(f / f_base if np.isfinite(f) else np.inf)
                    es.append(e / e_base if np.isfinite(e) else np.inf)
                fs, es = np.array(fs), np.array(es)
                label = "(none)" if V == Ch else name
                print(f"{Ch:2d} {V:2d} {Ch - V:2d}  {label:15s} {fs.mean():12.4g} {fs.std():9.3g}   "
                      f"{es.mean():12.4g} {es.std():9.3g}")
    print(f"sweep time {time.perf_counter() - t0:.1f} s")


def gfactor(args):
    from . import gfactor as gf
    dev = torch.device("cuda")
    shape, C, R, lam = (256, 256), 8, 3, 1e-3
    idx = np.flatnonzero(synthdata.regular_mask(shape, R).ravel()).astype(np.int32)
    full = np.arange(shape[0] * shape[1], dtype=np.int32)
    maps = torch.from_numpy(synthdata.coil_maps(shape, C).astype(np.complex64)).to(dev)
    x = torch.from_numpy(synthdata.phantom(shape, seed=1).astype(np.complex64)).to(dev)
    res = {}
    for name, ix, prm in (("full", full, cs.SolveParams(K=30, sketch=False, do_pca=False, use_graph=True)),
                          ("R3", idx, cs.SolveParams(K=30, sketch=False, do_pca=False, use_graph=True)),
                          ("R3 sketched", idx, cs.SolveParams(T=5, K=10, V=3, S=1, dist=cs.RADEMACHER, seed=4,
                                                              use_graph=True))):
        plan0 = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=torch.from_numpy(ix).to(dev))
        y = cs.sense_fwd(plan0, x, maps)
        sig = 1e-2 * float(y.abs().max())
        noise = torch.from_numpy(np.stack([synthdata.complex_noise(tuple(y.shape), sig, seed=1000 + k)
                                           for k in range(args.replicas)]).astype(np.complex64)).to(dev)
        ys = gf.replicas(y, noise)
        xs, plans = gf.replica_reconstructions(shape, maps, torch.from_numpy(ix).to(dev), ys, lam, prm)   # capture
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        xs, _ = gf.replica_reconstructions(shape, maps, torch.from_numpy(ix).to(dev), ys, lam, prm, plans=plans)
        b.record()
        torch.cuda.synchronize()
        res[name] = (xs, a.elapsed_time(b))
        print(f"{name}: {args.replicas} replicas in one batched graph: {a.elapsed_time(b):.1f} ms")
    inside = synthdata.phantom(shape, seed=1) != 0
    for name in ("R3", "R3 sketched"):
        ig = gf.inverse_gfactor(res[name][0], res["full"][0], R).cpu().numpy()
        print(f"inverse g-factor ({name}) inside the object: mean {ig[inside].mean():.3f}, "
              f"5th percentile {np.percentile(ig[inside], 5):.3f}")


def compare(args):
    cfg = CONFIGS[args.config]
    dev = torch.device("cuda")
    img, grid, C = cfg["img"], cfg["grid"], cfg["nc"]
    traj = synthdata.cones_trajectory(cfg["n_int"], 512)
    dcf = synthdata.cones_dcf(traj, img, cfg["n_int"], 512)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=torch.from_numpy(traj).to(dev), dcf=torch.from_numpy(dcf).to(dev),
                   grid=grid)
    maps = synthdata.coil_maps_torch(img, C, device=dev)
    y = cs.sense_fwd(plan, synthdata.phantom_torch(img, seed=1, device=dev), maps)
    y += 1e-3 * float(y.abs().max()) * torch.from_numpy(
        synthdata.complex_noise(tuple(y.shape), 1.0, seed=3).astype(np.complex64)).to(dev)
    v0 = synthdata.phantom_torch(img, seed=5, device=dev)
    lam, levels = 2e-3, 4
    x_inf, _ = cs.recon_solve(plan, y, maps, lam, cs.REG_L1_WAVELET,
                              cs.SolveParams(K=300, sketch=False, do_pca=False, power_v0=v0), wavelet_levels=levels)
    n_inf = float(torch.linalg.vector_norm(x_inf))

    def run(name, lam_m, prm, n_it):
        its = torch.empty((n_it,) + tuple(img), dtype=torch.complex64, device=dev)
        prm.iterates = its
        cs.recon_solve(plan, y, maps, lam_m, cs.REG_L1_WAVELET, prm, wavelet_levels=levels)   # warm-up
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        cs.recon_solve(plan, y, maps, lam_m, cs.REG_L1_WAVELET, prm, wavelet_levels=levels)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        d = [float(torch.linalg.vector_norm(its[k] - x_inf)) / n_inf for k in range(n_it)]
        hit = [k for k, e in enumerate(d) if e <= 0.05]
        t5 = f"{(hit[0] + 1) * ms / n_it:.0f} ms" if hit else "not reached"
        print(f"{name:32s} {n_it:3d} steps, {ms:7.0f} ms ({ms / n_it:6.1f} ms/step); distance to x_inf: "
              f"after 1/4 {d[n_it // 4 - 1]:.4f}, 1/2 {d[n_it // 2 - 1]:.4f}, end {d[-1]:.4f}; 5%: {t5}")

    K = 60
    rng = np.random.default_rng(11)
    batches = torch.from_numpy(np.stack([rng.permutation(C)[:8] for _ in range(K)]).astype(np.int32)).to(dev)
    print(f"{args.config}: l1-db4 lambda {lam}, {C} coils")
    run("full-coil FISTA", lam, cs.SolveParams(K=K, sketch=False, do_pca=False, power_v0=v0), K)
    run("coil compression to 8 (lam/2)", lam / 2, cs.SolveParams(K=K, sketch=False, do_pca=True, keep=8,
                                                                 power_v0=v0), K)
    run("AccProxSGD, batches of 8", lam, cs.SolveParams(K=K, sketch=False, do_pca=False, sgd_batch=8,
                                                        sgd_coils=batches, power_v0=v0), K)
    run("coil sketching m=8 (7+1 Rad.)", lam, cs.SolveParams(T=20, K=10, V=7, S=1, dist=cs.RADEMACHER, seed=4,
                                                            power_v0=v0), 20)


def sketch(args):
    dev = torch.device("cuda")
    C, V, S, D = 40, 5, 5, args.voxels
    m = torch.randn((C, D), dtype=torch.complex64, device=dev)
    sk = cs.sketch_draw(4, 0, 1, C, V, S)[0].contiguous()
    out = torch.empty((S, D), dtype=torch.complex64, device=dev)
    res = {}
    for prec, name in [(cs.PREC_FP32, "fp32"), (cs.PREC_BF16_SPLIT, "bf16_split")]:
        for _ in range(2):
            cs.sketched_maps(sk, m, V, precision=prec, out=out)
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        for _ in range(args.iters):
            cs.sketched_maps(sk, m, V, precision=prec, out=out)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.iters
        byt = (C - V) * D * 8 + S * D * 8
        res[name] = out.clone()
        print(f"sketched maps {name}: D={D}: {ms:.3f} ms, {byt / ms / 1e6:.0f} GB/s algorithmic")
    cs.device_status()
    err = float((res["bf16_split"] - res["fp32"]).norm() / res["fp32"].norm())
    print(f"bf16 split vs fp32 NRMSE {err:.2e}")


def cart2d(args):
    dev = torch.device("cuda")
    shape, C = (128, 128), 8
    mask = synthdata.poisson_disc_mask(shape, R=4.0, centre=24, seed=2)
    idx = np.flatnonzero(mask.ravel()).astype(np.int32)
    maps = torch.from_numpy(synthdata.coil_maps(shape, C).astype(np.complex64)).to(dev)
    x_true = torch.from_numpy(synthdata.phantom(shape, seed=1).astype(np.complex64)).to(dev)
    plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=torch.from_numpy(idx).to(dev))
    y = cs.sense_fwd(plan, x_true, maps)
    for g in (False, True):
        p = cs.SolveParams(T=5, K=10, V=2, S=2, use_graph=g)
        for _ in range(3):
            cs.recon_solve(plan, y, maps, 1e-3, cs.REG_L2, p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.iters):
            _, st = cs.recon_solve(plan, y, maps, 1e-3, cs.REG_L2, p)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.iters
        print(f"cart2d recon use_graph={g}: {dt * 1e3:.3f} ms wall, {st['ms_total']:.3f} ms device")


def batched(args):
    dev = torch.device("cuda")
    C = 16
    sizes = synthdata.slice_sizes(args.slices)
    items = []
    for k, n in enumerate(sizes):
        shape = (n, n)
        mask = synthdata.line_mask(shape, R=6.0, centre_lines=24, seed=200 + k)
        idx = np.flatnonzero(mask.ravel()).astype(np.int32)
        maps = synthdata.coil_maps_torch(shape, C, device=dev)
        x_true = synthdata.phantom_torch(shape, seed=300 + k, device=dev)
        plan = cs.Plan(cs.CARTESIAN, shape, C, mask_idx=torch.from_numpy(idx).to(dev))
        y = cs.sense_fwd(plan, x_true, maps)
        y += 1e-3 * y.abs().max() * torch.randn_like(y)
        items.append(dict(plan=plan, y=y, maps=maps, power_v0=synthdata.phantom_torch(shape, seed=500 + k, device=dev)))
    D_total = sum(n * n for n in sizes)
    common = dict(T=10, K=10, V=3, S=3, seed=4)

    def run_seq():
        for it in items:
            cs.recon_solve(it["plan"], it["y"], it["maps"], 5e-3, cs.REG_L1_WAVELET,
                           cs.SolveParams(power_v0=it["power_v0"], **common))

    def run_batch(g):
        cs.recon_solve_batched(items, 5e-3, cs.REG_L1_WAVELET, cs.SolveParams(use_graph=g, **common))

    for name, fn in [("one slice after another", run_seq), ("forked batch", lambda: run_batch(False)),
                     ("one CUDA graph", lambda: run_batch(True))]:
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.iters):
            fn()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.iters
        print(f"batched slices ({len(sizes)} slices, {D_total / 1e6:.2f} M pixels, 16 coils): {name}: {dt * 1e3:.1f} ms")


def _bf16_peak():
    import json
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def warmnet(args):
    import ctypes
    import paper_2305_06482_gb300.warmstart as ws
    img = CONFIGS[args.config]["img"]
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev).manual_seed(0)
    L = cs.lib()
    peak, src = _bf16_peak()
    c1, c2, c3 = ws.WIDTHS
    lv = [tuple(img), tuple(v // 2 for v in img), tuple(v // 4 for v in img)]

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        a, b = _events()
        a.record()
        for _ in range(args.iters):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.iters

    total_flops = 0.0
    print(f"warm-start U-Net on {img}: tensor-core convolutions (FLOPs 2 V 27 cin cout; peak bf16 {peak:.0f} "
          f"TFLOP/s, {src})")
    for name, level, cin, cout in (("e1a", 0, 4, c1), ("e1b", 0, c1, c1), ("e2a", 1, c1, c2), ("e2b", 1, c2, c2),
                                   ("b1", 2, c2, c3), ("b2", 2, c3, c3), ("d2a", 1, 2 * c2, c2), ("d2b", 1, c2, c2),
                                   ("d1a", 0, 2 * c1, c1), ("d1b", 0, c1, c1)):
        dims = lv[level]
        V = int(np.prod(dims))
        npad, kpad = (16 if cout <= 16 else 32 if cout <= 32 else 64), (27 * cin + 15) // 16 * 16
        w = torch.randn((cout, 27, cin), generator=gen, device=dev) * 0.1
        bias = torch.zeros(cout, device=dev)
        packed = torch.empty((npad, kpad), dtype=torch.int16, device=dev)
        cs._check(L.cs_nn_pack_weights(cs._ptr(w), cout, cin, 0, cs._ptr(packed), npad, kpad, None))
        x = torch.randn((V, cin), generator=gen, device=dev)
        out = torch.empty((V, cout), device=dev)
        ms = timed(lambda: cs._check(L.cs_nn_conv3d(cs._ptr(x), *dims, cin, cs._ptr(packed), npad, kpad, cout,
                                                    cs._ptr(bias), 1, 0, cs._ptr(out), cout, 0, None)))
        fl = 2.0 * V * 27 * cin * cout
        total_flops += fl
        print(f"  layer {name:3s} {cin:2d}->{cout:2d} on {dims}: {ms:.3f} ms, {fl / ms / 1e9:.1f} TFLOP/s "
              f"({fl / ms / 1e9 / peak:.3f} of peak)")
        gw = torch.zeros((cout, 27, cin), device=dev)
        gb = torch.zeros(cout, device=dev)
        msw = timed(lambda: cs._check(L.cs_nn_conv3d_wgrad(cs._ptr(x), cs._ptr(out), *dims, cin, cout, cs._ptr(gw),
                                                           cs._ptr(gb), None)))
        print(f"        weight gradient: {msw:.3f} ms, {fl / msw / 1e9:.1f} TFLOP/s ({fl / msw / 1e9 / peak:.3f} of peak)")
        del x, out, gw, gb
    for cdims, cin, cout in ((lv[2], c3, c2), (lv[1], c2, c1)):
        Vc = int(np.prod(cdims))
        x = torch.randn((Vc, cin), generator=gen, device=dev)
        w = torch.randn((cout, 8, cin), generator=gen, device=dev) * 0.1
        bias = torch.zeros(cout, device=dev)
        cat = torch.empty((8 * Vc, 2 * cout), device=dev)
        ms = timed(lambda: cs._check(L.cs_nn_upconv2(cs._ptr(x), *cdims, cin, cs._ptr(w), cs._ptr(bias), cout,
                                                     cs._ptr(cat), 2 * cout, 0, None)))
        byt = 4.0 * (Vc * cin + 8 * Vc * cout)
        print(f"  transposed conv {cin}->{cout} to {tuple(2 * v for v in cdims)}: {ms:.3f} ms, {byt / ms / 1e6:.0f} GB/s")
        srcs = torch.randn((8 * Vc, cout), generator=gen, device=dev)
        ms = timed(lambda: cs._check(L.cs_nn_slice(cs._ptr(srcs), cout, 0, cout, cs._ptr(cat), 2 * cout, cout, 8 * Vc,
                                                   0, None)))
        print(f"  skip copy of {cout} channels: {ms:.3f} ms, {8.0 * 8 * Vc * cout / ms / 1e6:.0f} GB/s")
        del x, cat, srcs
    for dims, C in ((lv[0], c1), (lv[1], c2)):
        V = int(np.prod(dims))
        x = torch.randn((V, C), generator=gen, device=dev)
        po = torch.empty((V // 8, C), device=dev)
        pi = torch.empty((V // 8, C), dtype=torch.uint8, device=dev)
        cd = tuple(v // 2 for v in dims)
        ms = timed(lambda: cs._check(L.cs_nn_maxpool2(cs._ptr(x), *cd, C, cs._ptr(po), cs._ptr(pi), None)))
        print(f"  max-pool of {C} channels on {dims}: {ms:.3f} ms, {4.0 * V * C * (1 + 1 / 8 + 1 / 32) / ms / 1e6:.0f} GB/s")
        del x, po, pi
    x = torch.randn((int(np.prod(lv[0])), c1), generator=gen, device=dev)
    w = torch.randn((2, c1), generator=gen, device=dev)
    bias = torch.zeros(2, device=dev)
    y = torch.empty((x.shape[0], 2), device=dev)
    ms = timed(lambda: cs._check(L.cs_nn_conv1(cs._ptr(x), x.shape[0], c1, 2, cs._ptr(w), cs._ptr(bias), cs._ptr(y),
                                               None)))
    print(f"  1x1x1 output layer {c1}->2: {ms:.3f} ms, {4.0 * x.shape[0] * (c1 + 2) / ms / 1e6:.0f} GB/s")
    del x, y
    # the library's network object: one inference on the image size, one training step on a 64^3 crop
    net = ws.UNet(seed=0)
    cplx = lambda shape: torch.complex(torch.randn(shape, generator=gen, device=dev),
                                       torch.randn(shape, generator=gen, device=dev))
    xt, d = cplx(img), cplx(img)
    xh = torch.empty_like(xt)
    ms = timed(lambda: net.infer(xt, d, 0.5, out=xh))
    print(f"  inference (whole U-Net, {total_flops / 1e12:.2f} TFLOP in the 3x3x3 layers): {ms:.2f} ms, "
          f"{total_flops / ms / 1e9:.1f} TFLOP/s")
    del xt, d, xh
    crop = (64, 64, 64)
    xc, dc, tc = cplx(crop), cplx(crop), cplx(crop)
    ms = timed(lambda: net.train_step(xc, dc, tc, 0.5, 1e-5))
    print(f"  training step on a 64^3 crop (forward, backward, Adam): {ms:.2f} ms")
    cs._check(L.cs_nn_status(None))
    net.close()


def warmtrain(args):
    """Warm-start training on pairs of the method itself, then a held-out reconstruction with and
    without the network through recon_solve (the acceptance decided on the device)."""
    import paper_2305_06482_gb300.warmstart as ws
    cfg = CONFIGS[args.config]
    dev = torch.device("cuda")
    img, grid, C = cfg["img"], cfg["grid"], cfg["nc"]
    large = args.config == "cones3d_large"
    traj = synthdata.cones_trajectory(cfg["n_int"], 512)
    dcf = synthdata.cones_dcf(traj, img, cfg["n_int"], 512)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=torch.from_numpy(traj).to(dev), dcf=torch.from_numpy(dcf).to(dev),
                   grid=grid)
    maps = synthdata.coil_maps_torch(img, C, device=dev)
    lam, levels = 2e-3, 4
    V, S = (5, 5) if large else (4, 4)
    T, K, tight = args.outer, args.K, args.tight
    t0 = time.perf_counter()
    pairs = []
    for k in range(args.phantoms):
        seed = 101 + k
        y = cs.sense_fwd(plan, synthdata.phantom_torch(img, seed=seed, device=dev), maps)
        su = ws.setup(plan, y, maps, lam, V, S, T, seed, synthdata.phantom_torch(img, seed=seed + 50, device=dev), levels)
        _, pr, _ = ws.run(su, T, K, record_pairs=1, tight_K=tight)
        pairs += pr
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    npairs = len(pairs)
    if args.crops > 0:
        # the training set stored as fixed 64^3 crops of the volume pairs
        pairs = ws.make_crops(pairs, args.crops, (64, 64, 64), seed=7)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    net = ws.UNet(seed=0)
    a, b = _events()
    a.record()
    hist = ws.train(net, pairs, steps=args.train_steps, lr=2e-3, crop=None if args.crops > 0 else (64, 64, 64))
    b.record()
    torch.cuda.synchronize()
    t_train = a.elapsed_time(b) / 1e3
    del pairs
    torch.cuda.empty_cache()
    if args.save:
        os.makedirs(os.path.dirname(os.path.abspath(args.save)), exist_ok=True)
        net.save(args.save)
    # held-out phantom: Algorithm 1 through recon_solve with and without the warm start
    seed = 199
    y = cs.sense_fwd(plan, synthdata.phantom_torch(img, seed=seed, device=dev), maps)
    v0 = synthdata.phantom_torch(img, seed=seed + 50, device=dev)
    x_inf, _ = cs.recon_solve(plan, y, maps, lam, cs.REG_L1_WAVELET,
                              cs.SolveParams(K=args.ref_iters, sketch=False, do_pca=False, power_v0=v0),
                              wavelet_levels=levels)
    res = {}
    for name, n in (("without", None), ("with", net)):
        p = cs.SolveParams(T=T, K=K, V=V, S=S, seed=seed + 4, power_v0=v0, precision=cs.PREC_BF16_SPLIT, warm=n,
                           x_ref=x_inf, trace=True)
        cs.recon_solve(plan, y, maps, lam, cs.REG_L1_WAVELET, p, wavelet_levels=levels)      # untimed
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        _, st = cs.recon_solve(plan, y, maps, lam, cs.REG_L1_WAVELET, p, wavelet_levels=levels)
        b.record()
        torch.cuda.synchronize()
        tr = st["trace"]
        res[name] = (np.sqrt(np.maximum(tr[:, cs.TRACE_DIST2], 0)), tr[:, cs.TRACE_ACCEPT], a.elapsed_time(b))
    crops = f"{args.crops} stored 64^3 crops of them" if args.crops > 0 else "random 64^3 crops"
    print(f"warm start on {args.config} ({img}, {C} coils, m = {V} + {S}): {npairs} training pairs "
          f"(x^t, d, sub-problem solved with {tight} FISTA iterations) from {args.phantoms} phantoms at K = {K} in "
          f"{t_pairs:.1f} s; {args.train_steps} Adam steps on {crops} in {t_train:.2f} s "
          f"(loss {np.mean(hist[:20]):.3e} -> {np.mean(hist[-20:]):.3e})")
    for name in ("without", "with"):
        e, acc, ms = res[name]
        extra = f", accepted {int((acc == 1).sum())}/{len(acc)}" if name == "with" else ""
        print(f"  held-out, {name} warm start: NRMSE to x_inf ({args.ref_iters} plain iterations) per outer " +
              " ".join(f"{v:.3e}" for v in e) + f"; {ms:.0f} ms per reconstruction{extra}")


def recon(args):
    """One coil-sketched reconstruction in the benchmark's configuration (l1-db4 lambda 2e-3, 4
    levels, FISTA, m = 10 = 5 PCA + 5 Gaussian, BF16-split sketched maps, noise 1e-3 max|y|) with
    --outer T outer and --K inner iterations; no reference solve.  Every outer iteration runs the
    same kernels, so a short run gives the kernel shares of the full reconstruction."""
    import math
    cfg = CONFIGS[args.config]
    dev = torch.device("cuda")
    img, grid, C = cfg["img"], cfg["grid"], cfg["nc"]
    traj = synthdata.cones_trajectory(cfg["n_int"], 512)
    dcf = synthdata.cones_dcf(traj, img, cfg["n_int"], 512)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=torch.from_numpy(traj).to(dev), dcf=torch.from_numpy(dcf).to(dev),
                   grid=grid)
    maps = synthdata.coil_maps_torch(img, C, device=dev)
    y = cs.sense_fwd(plan, synthdata.phantom_torch(img, seed=1, device=dev), maps)
    if args.tile:
        plan.set_tile((args.tile,) * 3)
    gen = torch.Generator(device=dev).manual_seed(4)
    sig = 1e-3 * y.abs().max().item()
    y += (sig / math.sqrt(2)) * torch.complex(torch.randn(y.shape, generator=gen, device=dev),
                                              torch.randn(y.shape, generator=gen, device=dev))
    v0 = synthdata.phantom_torch(img, seed=6, device=dev)
    p = cs.SolveParams(T=args.outer, K=args.K, V=5, S=5, seed=5, power_v0=v0, precision=cs.PREC_BF16_SPLIT)
    for _ in range(args.warmup):
        cs.recon_solve(plan, y, maps, 2e-3, cs.REG_L1_WAVELET, p, wavelet_levels=4)
    torch.cuda.synchronize()
    n0 = cs.launch_count()
    a, b = _events()
    a.record()
    _, st = cs.recon_solve(plan, y, maps, 2e-3, cs.REG_L1_WAVELET, p, wavelet_levels=4)
    b.record()
    torch.cuda.synchronize()
    print(f"{args.config}: coil-sketched reconstruction T = {args.outer}, K = {args.K}: {a.elapsed_time(b):.1f} ms, "
          f"{cs.launch_count() - n0} library kernel launches")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["nufft", "normal", "tv", "ablation", "gfactor", "compare", "sketch", "cart2d",
                                     "batched", "warmnet", "warmtrain", "recon"])
    ap.add_argument("--replicas", type=int, default=60)
    ap.add_argument("--seeds", type=int, default=16)
    ap.add_argument("--slices", type=int, default=64)
    ap.add_argument("--config", default="cones3d_128", choices=list(CONFIGS))
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--voxels", type=int, default=160 * 256 * 256)
    ap.add_argument("--phantoms", type=int, default=4)
    ap.add_argument("--autotune", action="store_true", help="nufft: tune the gridding launches first")
    ap.add_argument("--autotune-tile", action="store_true", help="nufft, normal: tune the binning tile first")
    ap.add_argument("--tiles", default="", help="tile candidates of --autotune-tile, comma-separated")
    ap.add_argument("--tile", type=int, default=0, help="nufft, normal: binning tile (cubic; 0 = plan default)")
    ap.add_argument("--train-steps", type=int, default=300)
    ap.add_argument("--outer", type=int, default=6, help="warmtrain: outer iterations per phantom; recon: T")
    ap.add_argument("--K", type=int, default=4, help="warmtrain, recon: inner FISTA iterations")
    ap.add_argument("--tight", type=int, default=40, help="warmtrain: FISTA iterations of a training target")
    ap.add_argument("--ref-iters", type=int, default=300, help="warmtrain: plain FISTA iterations of x_inf")
    ap.add_argument("--save", default="", help="warmtrain: write the trained network here")
    ap.add_argument("--crops", type=int, default=0, help="warmtrain: train on this many stored 64^3 crops (0 = "
                                                       "a fresh random crop every step)")
    args = ap.parse_args()
    {"nufft": nufft, "normal": normal, "tv": tv, "ablation": ablation, "gfactor": gfactor, "compare": compare,
     "sketch": sketch, "cart2d": cart2d, "batched": batched, "warmnet": warmnet, "warmtrain": warmtrain,
     "recon": recon}[args.what](args)


if __name__ == "__main__":
    main()
