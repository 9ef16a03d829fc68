"""Benchmark: coil-sketched iterative MR reconstruction on GB300.

Metric: time-to-NRMSE per reconstruction (s), coil sketching vs the plain full-coil solver, on
the large 3D cones workload (160x256x256 image, 200x320x320 grid, 40 coils, 20000 x 512 cones
samples, l1-db4 lambda = 2e-3, FISTA, sketch m = 10 = 5 PCA + 5 Gaussian), plus the multicoil
NUFFT forward+adjoint throughput in the roofline object.

A step is one full coil-sketched reconstruction (coil PCA, sketch draws, T outer iterations of
true gradient + sketched FISTA sub-problem) from device-resident inputs.  The iteration count
of the timed reconstructions is the first outer count that reaches the NRMSE target against the
plain full-coil FP32 solution x_inf (found in an untimed logged run); when the target is not
reached within the cap, the timed runs use the cap and the JSON line reports the NRMSE they
reach.  The plain solver is timed for the same NRMSE.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
Multi-GPU (torchrun): each rank reconstructs its own synthetic volume (independent problems,
weak scaling, no collective on the data path); time = max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(name="cones3d_large", img=(160, 256, 256), grid=(200, 320, 320), nc=40, n_int=20000,
                n_read=512, lam=2e-3, V=5, S=5, K=10, T_cap=20, levels=4, nrmse_target=1e-3,
                plain_iters=300, seed=1)
METRIC = "time-to-NRMSE 1e-3 per recon (s), sketched vs full-coil; NUFFT fwd+adj GB/s"


def workload_desc(w):
    return (f"{w['name']}: {w['img'][0]}x{w['img'][1]}x{w['img'][2]} image, grid "
            f"{w['grid'][0]}x{w['grid'][1]}x{w['grid'][2]}, {w['nc']} coils, {w['n_int']}x{w['n_read']} cones "
            f"samples/coil, l1-db4 (lambda {w['lam']}) FISTA K={w['K']}, sketch m={w['V'] + w['S']} "
            f"({w['V']} PCA + {w['S']} Gaussian), sketched maps BF16 split on tensor cores")


def nufft_model_bytes(w, C):
    """Algorithmic bytes of one multicoil forward + adjoint: per coil and direction 8D (maps) +
    2 passes x 3 axes x 8G (FFT) + 8N (samples); per operator 16N (trajectory + dcf) + 16D."""
    D = int(np.prod(w["img"]))
    G = int(np.prod(w["grid"]))
    N = w["n_int"] * w["n_read"]
    return 2 * C * (8 * D + 48 * G + 8 * N) + 2 * (16 * N + 16 * D)


def nufft_compulsory_bytes(w, C):
    """Compulsory bytes of one multicoil forward + adjoint (maps and samples once per coil and
    direction, trajectory + dcf, image in and out): C (8D + 8N) 2 + 16N + 16D."""
    D = int(np.prod(w["img"]))
    N = w["n_int"] * w["n_read"]
    return C * (8 * D + 8 * N) * 2 + 16 * N + 16 * D


# ------------------------------------------------------------------------------------------
def sample_clocks_start(out_path, dev_index):
    cmd = ["nvidia-smi", f"--id={dev_index}",
           "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        f = open(out_path, "w")
        return subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def sample_clocks_stop(proc, f, path):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx = max(mx, float(parts[2]))
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
def cpu_reference_step(w, sub=16):
    """Bounded sample of the workload on the FP64 CPU oracle, extrapolated to one sketched
    reconstruction: one coil forward+adjoint gridding NUFFT at full image/grid size with every
    `sub`-th interleave (gridding time scaled by the sample ratio), one full-grid centred DFT
    pair, one db4 prox at full image size."""
    import synthdata
    from oracle import nufft as onufft
    from oracle import wavelet as owav
    img, grid = w["img"], w["grid"]
    traj = synthdata.cones_trajectory(w["n_int"], w["n_read"]).reshape(w["n_int"], w["n_read"], 3)
    traj_s = np.ascontiguousarray(traj[::sub].reshape(-1, 3))
    frac = traj_s.shape[0] / (w["n_int"] * w["n_read"])
    plan = onufft.Plan(traj_s, img, grid)
    rng = np.random.default_rng(0)
    g = rng.standard_normal(grid) + 1j * rng.standard_normal(grid)
    t0 = time.perf_counter()
    yk = plan.interp(g)
    t1 = time.perf_counter()
    plan.spread(yk)
    t2 = time.perf_counter()
    onufft._cdft(g, (0, 1, 2), False)
    onufft._cdft(g, (0, 1, 2), True)
    t3 = time.perf_counter()
    x = rng.standard_normal(img) + 1j * rng.standard_normal(img)
    owav.prox_l1_wavelet(x, 1e-3, w["levels"])
    t4 = time.perf_counter()
    t_coil = (t1 - t0 + t2 - t1) / frac + (t3 - t2)
    t_prox = t4 - t3
    return t_coil, t_prox, traj_s.shape[0]


def cpu_recon_estimate(w, T, t_coil, t_prox):
    m = w["V"] + w["S"]
    coil_ops = T * (w["nc"] + w["K"] * m) + 20 * m   # gradients, sub-problem iterations, power iteration
    prox = T * w["K"]
    return coil_ops * t_coil + prox * t_prox


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    T_assumed = w["T_cap"]
    cores = 1
    vals = []
    for i in range(args.warmup + args.steps):
        t_coil, t_prox, nsub = cpu_reference_step(w)
        est = cpu_recon_estimate(w, T_assumed, t_coil, t_prox)
        if i >= args.warmup:
            vals.append(est)
    v = float(np.mean(vals))
    sample = (f"1 coil fwd+adj gridding NUFFT at full size with every 16th interleave ({nsub} samples, "
              f"gridding time scaled x16), one full-grid DFT pair, one db4 prox; extrapolated to a "
              f"sketched recon with T={T_assumed}, K={w['K']}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(w), "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
def run_native(args, w, rank, world, local_rank):
    import torch
    import paper_2305_06482_gb300 as cs
    import synthdata
    from paper_2305_06482_gb300 import build as _build
    from paper_2305_06482_gb300 import replicas

    if not os.path.exists(cs.LIB_PATH):
        _build.build()
    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    img, grid, C = w["img"], w["grid"], w["nc"]
    m = w["V"] + w["S"]
    seed = replicas.replica_seed(w["seed"], rank)
    t_setup = time.perf_counter()
    traj = synthdata.cones_trajectory(w["n_int"], w["n_read"])
    dcf = synthdata.cones_dcf(traj, img, w["n_int"], w["n_read"])
    maps = synthdata.coil_maps_torch(img, C, device=dev)
    x_true = synthdata.phantom_torch(img, seed=seed, device=dev)
    traj_d = torch.from_numpy(traj).to(dev)
    dcf_d = torch.from_numpy(dcf).to(dev)
    torch.cuda.synchronize()
    t_plan = time.perf_counter()
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=traj_d, dcf=dcf_d, grid=grid)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t_plan
    del traj_d, dcf_d
    y = cs.sense_fwd(plan, x_true, maps)
    gen = torch.Generator(device=dev).manual_seed(seed + 3)
    sig = 1e-3 * y.abs().max().item()
    y += (sig / math.sqrt(2)) * torch.complex(torch.randn(y.shape, generator=gen, device=dev),
                                              torch.randn(y.shape, generator=gen, device=dev))
    v0 = synthdata.phantom_torch(img, seed=seed + 5, device=dev)   # power-iteration start vector
    torch.cuda.synchronize()

    def nrmse(a, b):
        return float((a - b).norm() / b.norm())

    # x_inf: plain full-coil FISTA, untimed, iterates kept to find its time-to-NRMSE
    K_inf = w["plain_iters"]
    its = torch.empty((K_inf,) + img, dtype=torch.complex64, device=dev)
    x_inf, st_inf = cs.recon_solve(plan, y, maps, w["lam"], cs.REG_L1_WAVELET,
                                   cs.SolveParams(K=K_inf, sketch=False, do_pca=False, power_v0=v0, iterates=its),
                                   wavelet_levels=w["levels"])
    plain_curve = [nrmse(its[k], x_inf) for k in range(K_inf)]
    del its
    torch.cuda.empty_cache()
    # logged sketched run: NRMSE after every outer iteration
    T_cap = w["T_cap"]
    sk_its = torch.empty((T_cap,) + img, dtype=torch.complex64, device=dev)
    sparams = dict(K=w["K"], V=w["V"], S=w["S"], seed=seed + 4, power_v0=v0, precision=cs.PREC_BF16_SPLIT)
    cs.recon_solve(plan, y, maps, w["lam"], cs.REG_L1_WAVELET, cs.SolveParams(T=T_cap, iterates=sk_its, **sparams),
                   wavelet_levels=w["levels"])
    sk_curve = [nrmse(sk_its[t], x_inf) for t in range(T_cap)]
    del sk_its
    target = w["nrmse_target"]
    reached = [t for t, e in enumerate(sk_curve) if e <= target]
    T_star = reached[0] + 1 if reached else T_cap
    eps = target if reached else sk_curve[T_star - 1]
    plain_hit = [k for k, e in enumerate(plain_curve) if e <= eps]
    k_star = plain_hit[0] + 1 if plain_hit else K_inf
    setup_s = time.perf_counter() - t_setup

    # ---- timed region: W warm-up + K timed sketched reconstructions ----
    params_t = cs.SolveParams(T=T_star, **sparams)
    for _ in range(args.warmup):
        cs.recon_solve(plan, y, maps, w["lam"], cs.REG_L1_WAVELET, params_t, wavelet_levels=w["levels"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk_path = os.environ.get("CS_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(), f"cs_clocks_rank{rank}.csv")
    proc, fh = sample_clocks_start(clk_path, local_rank)
    cs.profile(True)
    launches0 = cs.launch_count()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("cs_timed")
    e0.record(stream)
    x_last = None
    for _ in range(args.steps):
        x_last, _ = cs.recon_solve(plan, y, maps, w["lam"], cs.REG_L1_WAVELET, params_t, wavelet_levels=w["levels"])
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    launches = cs.launch_count() - launches0
    ms_total = e0.elapsed_time(e1)
    prof = {k: cs.profile_read(k) for k in cs.STAGES}
    cs.profile(False)
    clocks = sample_clocks_stop(proc, fh, clk_path)
    ms_total = replicas.slowest_ms(ms_total, dist, dev)
    ms_step = ms_total / args.steps
    value = replicas.seconds_per_recon(ms_total, args.steps, world)   # seconds per recon, whole job
    nrmse_timed = nrmse(x_last, x_inf)

    # plain full-coil solver for the same NRMSE (k_star iterations), timed
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    pparams = cs.SolveParams(K=k_star, sketch=False, do_pca=False, power_v0=v0)
    e2.record(stream)
    cs.recon_solve(plan, y, maps, w["lam"], cs.REG_L1_WAVELET, pparams, wavelet_levels=w["levels"])
    e3.record(stream)
    torch.cuda.synchronize()
    plain_s = e2.elapsed_time(e3) / 1e3

    # multicoil NUFFT forward + adjoint throughput (all coils)
    xa = torch.empty(img, dtype=torch.complex64, device=dev)
    yk = torch.empty((C, traj.shape[0]), dtype=torch.complex64, device=dev)
    for _ in range(2):
        cs.sense_fwd(plan, x_true, maps, yk)
        cs.sense_adj(plan, yk, maps, xa)
    torch.cuda.synchronize()
    e4 = torch.cuda.Event(enable_timing=True)
    e5 = torch.cuda.Event(enable_timing=True)
    reps = 5
    e4.record(stream)
    for _ in range(reps):
        cs.sense_fwd(plan, x_true, maps, yk)
        cs.sense_adj(plan, yk, maps, xa)
    e5.record(stream)
    torch.cuda.synchronize()
    op_ms = e4.elapsed_time(e5) / reps
    op_gbs = nufft_model_bytes(w, C) / (op_ms * 1e-3) / 1e9
    del yk, xa

    # dominant kernel of the timed region (by summed device time) and its roofline
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    dom_bytes, dom_n_model = stage_bytes(dom, w, T_star, args.steps)
    avg_ms = dom_ms / max(dom_n, 1)
    per_launch_bytes = dom_bytes / max(dom_n_model, 1)
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 else None
    ratio = TRAFFIC_RATIO.get(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": (achieved / hbm_peak) if achieved else None,
                "traffic": ratio * per_launch_bytes if ratio else None,
                "traffic_source": ("ncu DRAM read+write / algorithmic bytes of one launch on the 128^3 cones, "
                                   f"10-coil case ({ratio}), scaled to this launch size") if ratio else None,
                "launches": dom_n, "launches_model": dom_n_model, "avg_launch_ms": avg_ms,
                "bytes_per_launch": per_launch_bytes,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback",
                "nufft_fwd_adj_gbs": op_gbs, "nufft_fwd_adj_frac": op_gbs / hbm_peak,
                "nufft_fwd_adj_ms": op_ms, "nufft_fwd_adj_model_gb": nufft_model_bytes(w, C) / 1e9,
                "nufft_fwd_adj_compulsory_gb": nufft_compulsory_bytes(w, C) / 1e9,
                "stage_ms": {k: v[0] / args.steps for k, v in prof.items()}}

    # end to end: pinned host inputs -> device, recon through the C ABI, result back to the host
    y_h = y.to("cpu").pin_memory()
    maps_h = maps.to("cpu").pin_memory()
    x_h = torch.empty(img, dtype=torch.complex64).pin_memory()
    y_d = torch.empty_like(y)
    maps_d = torch.empty_like(maps)

    def e2e_step():
        y_d.copy_(y_h, non_blocking=True)
        maps_d.copy_(maps_h, non_blocking=True)
        xo, _ = cs.recon_solve(plan, y_d, maps_d, w["lam"], cs.REG_L1_WAVELET, params_t, wavelet_levels=w["levels"])
        x_h.copy_(xo, non_blocking=True)
        torch.cuda.synchronize()

    # one untimed step: the outer-iteration graph is captured for these buffers once, as for the
    # device-resident runs above
    e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = y.numel() * 8 + maps.numel() * 8
    d2h = int(np.prod(img)) * 8

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        t_coil, t_prox, nsub = cpu_reference_step(w)
        est = cpu_recon_estimate(w, T_star, t_coil, t_prox)
        cpu = {"value": est, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"1 coil fwd+adj gridding NUFFT at full size on every 16th interleave ({nsub} samples, "
                         f"gridding scaled x16) + one full-grid DFT pair + one db4 prox, extrapolated to a "
                         f"sketched recon with T={T_star}, K={w['K']}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_desc(w), "parallelism": f"replicas{world}" if world > 1 else "single",
                           "l2": "inputs larger than L2 (k-space 3.3 GB, maps 3.4 GB per recon)",
                           "nrmse_target": target, "sketched_reached_target": bool(reached),
                           "sketched_outer_iters": T_star, "sketched_nrmse": nrmse_timed,
                           "sketched_nrmse_curve": [round(e, 6) for e in sk_curve],
                           "plain_iters_to_same_nrmse": k_star, "plain_time_to_same_nrmse_s": plain_s,
                           "sketched_over_plain_time": value * world / plain_s if plain_s > 0 else None,
                           "x_inf": f"plain FISTA, {K_inf} iterations",
                           "plan_s": plan_s, "setup_s": setup_s, "L_full": st_inf["L"]},
                "roofline": roofline,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# DRAM bytes (read + write) over algorithmic bytes of one launch, measured with ncu on the 128^3
# cones, 10-coil sketched normal operator (spread and interpolation: the whole launch; strided
# passes: mean of the forward y and z passes; writes still dirty in L2 at kernel end are not
# counted there).  Traffic grows in proportion to the algorithmic bytes, so the bench scales it.
TRAFFIC_RATIO = {"spread": 1.043, "interp": 0.823, "fft_plain": 0.90}


def stage_bytes(stage, w, T, steps):
    """Algorithmic bytes moved by all launches of one stage during the timed reconstructions.

    Per call with c coils (coil-interleaved buffers, complex64 = 8 B):
      interp / spread : c (8G + 8N) + 64N per launch (the 64-byte per-sample record: rotated
                        weights, box start, sqrt(w), user index) and one launch per chunk of
                        <= 16 coils;
      fft_plain       : the four strided passes of a forward + adjoint read and write
                        2 c 8 (nz ny Gx + 2 nz Gy Gx + G);
      expand / reduce : 8D + c (8D + 8 nz ny Gx).
    A sketched reconstruction makes, per outer iteration, one true gradient with C coils and K
    sub-problem normal operators with m coils, plus 20 power iterations with m coils once."""
    nz, ny, nx = w["img"]
    Gz, Gy, Gx = w["grid"]
    D, G = nz * ny * nx, Gz * Gy * Gx
    N = w["n_int"] * w["n_read"]
    C, m, K = w["nc"], w["V"] + w["S"], w["K"]
    calls = [(C, T), (m, T * K + 20)]          # (coils, calls) per reconstruction
    tot, launches = 0, 0
    for c, n in calls:
        if stage in ("interp", "spread"):
            nl = -(-c // 16)
            tot += n * (c * (8 * G + 8 * N) + nl * 64 * N)
            launches += n * nl
        elif stage == "fft_plain":
            tot += n * 2 * c * 8 * (nz * ny * Gx + 2 * nz * Gy * Gx + G)
            launches += n * 4
        elif stage in ("expand", "reduce"):
            tot += n * (8 * D + c * (8 * D + 8 * nz * ny * Gx))
            launches += n
    return tot * steps, launches * steps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if "RANK" in os.environ else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    w = dict(WORKLOAD)
    if args.impl == "reference":
        run_reference(args, w, rank, world)
    else:
        run_native(args, w, rank, world, local_rank)


if __name__ == "__main__":
    main()
