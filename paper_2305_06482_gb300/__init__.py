"""Python binding of libcoilsketch (coil-sketched SENSE reconstruction on sm_103a).

Argument marshalling only: every function forwards torch tensors (device memory, streams) to
the C ABI declared in ``include/coilsketch.h``; every step of the computation runs in the
library's CUDA kernels.  There is no CPU fallback: importing works without a GPU, but any
compute call raises if the compiled library or a CUDA device is missing.

Complex tensors are ``torch.complex64`` (interleaved float2), maps ``[C, *img]``, k-space
``[C, N]``, trajectories ``float32 [N, ndim]`` in cycles/pixel ordered (z, y, x).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcoilsketch.so")

CS_OK = 0
CS_ERR = {1: "CS_ERR_INVALID_ARG", 2: "CS_ERR_UNSUPPORTED_SIZE", 3: "CS_ERR_CUDA", 4: "CS_ERR_OOM",
          5: "CS_ERR_NONFINITE", 6: "CS_ERR_TIMEOUT", 7: "CS_ERR_BOUNDS"}
CARTESIAN, NONCARTESIAN = 0, 1
GAUSSIAN, RADEMACHER = 0, 1
NORM_UNIT_VAR, NORM_PAPER_LITERAL = 0, 1
PREC_FP32, PREC_BF16_SPLIT = 0, 1
REG_L2, REG_L1_WAVELET, REG_L1_TV = 0, 1, 2
# fields of a recon_solve trace record (include/coilsketch.h, CS_TRACE_*)
TRACE_GRAD2, TRACE_OBJECTIVE, TRACE_ACCEPT, TRACE_DIST2, TRACE_TIME_NS, TRACE_STEP_L, TRACE_FIELDS = 0, 1, 2, 3, 4, 5, 6


class CoilSketchError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{CS_ERR.get(code, code)}: {msg}")
        self.code = code


class _Geom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ndim", ctypes.c_int), ("img", ctypes.c_int * 3),
                ("max_coils", ctypes.c_int), ("mask_idx", ctypes.c_void_p), ("nsamples", ctypes.c_int64),
                ("grid", ctypes.c_int * 3), ("alpha", ctypes.c_float), ("traj", ctypes.c_void_p),
                ("dcf", ctypes.c_void_p), ("tile", ctypes.c_int * 3)]


class _Problem(ctypes.Structure):
    _fields_ = [("y", ctypes.c_void_p), ("maps", ctypes.c_void_p), ("C", ctypes.c_int),
                ("lam", ctypes.c_float), ("reg", ctypes.c_int), ("wavelet_levels", ctypes.c_int)]


class _Params(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("K", ctypes.c_int), ("sketch", ctypes.c_int), ("V", ctypes.c_int),
                ("S", ctypes.c_int), ("dist", ctypes.c_int), ("norm", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("sketches", ctypes.c_void_p), ("do_pca", ctypes.c_int), ("precision", ctypes.c_int),
                ("step", ctypes.c_float), ("power_iters", ctypes.c_int), ("power_v0", ctypes.c_void_p),
                ("use_graph", ctypes.c_int), ("iterates", ctypes.c_void_p), ("cg_iters", ctypes.c_int),
                ("tv_tau", ctypes.c_float), ("tv_sigma", ctypes.c_float), ("init", ctypes.c_int),
                ("keep", ctypes.c_int), ("sgd_batch", ctypes.c_int), ("sgd_coils", ctypes.c_void_p),
                ("sgd_beta", ctypes.c_float), ("sgd_min", ctypes.c_float), ("warm", ctypes.c_void_p),
                ("x_ref", ctypes.c_void_p), ("trace", ctypes.c_void_p), ("trace_objective", ctypes.c_int),
                ("step_per_outer", ctypes.c_int)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("problem", _Problem), ("x_inout", ctypes.c_void_p),
                ("power_v0", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("final_rr", ctypes.c_double), ("outer_done", ctypes.c_int),
                ("graph_used", ctypes.c_int), ("ms_total", ctypes.c_double), ("ms_pca", ctypes.c_double),
                ("warm_accepted", ctypes.c_int)]


EXPORTED = [
    "cs_last_error", "cs_version", "cs_plan_create", "cs_plan_destroy", "cs_plan_binning", "sense_fwd",
    "sense_adj", "sense_grad", "sketched_normal_apply", "coil_pca", "coil_rotate", "sketch_draw",
    "cs_philox4x32_10", "sketched_maps", "recon_solve", "wavelet_fwd", "wavelet_inv", "soft_threshold",
    "cs_hermitian_eig_host", "cs_launch_count", "cs_profile", "cs_profile_read", "coil_pca_noalloc", "cs_device_status", "recon_solve_batched",
    "sketched_subproblem_solve", "cs_subproblem_objective", "cs_power_iteration", "cs_nn_pack_weights",
    "cs_nn_conv3d", "cs_nn_conv3d_wgrad", "cs_nn_relu_bwd", "cs_nn_conv1", "cs_nn_conv1_bwd", "cs_nn_mse",
    "cs_nn_adam", "cs_nn_features", "cs_nn_target", "cs_nn_apply", "cs_nn_status", "tv_dual_update", "tv_rhs",
    "cs_nn_maxpool2", "cs_nn_maxpool2_bwd", "cs_nn_upconv2", "cs_nn_upconv2_bwd", "cs_nn_slice",
    "ws_net_create", "ws_net_destroy", "ws_net_infer", "ws_net_train_step", "ws_net_param", "ws_net_save",
    "ws_net_load", "cs_crop3d", "cs_wait_selftest", "cs_plan_set_gridding", "cs_plan_autotune",
    "cs_plan_set_deterministic", "cs_noise_std", "cs_inverse_gfactor", "cs_plan_set_tile", "cs_plan_autotune_tile",
]
STAGES = {"spread": 0, "interp": 1, "fft_plain": 2, "expand": 3, "reduce": 4}

_lib = None


def lib():
    """Load libcoilsketch.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcoilsketch.so not found at {LIB_PATH}; run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, i64, f, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_uint64
        sig = {
            "cs_last_error": ([], ctypes.c_char_p), "cs_version": ([], ctypes.c_char_p),
            "cs_plan_create": ([vp, vp, vp], i), "cs_plan_destroy": ([vp], i),
            "cs_plan_binning": ([vp, vp, vp, vp, vp, vp], i),
            "sense_fwd": ([vp, vp, vp, i, vp, vp], i), "sense_adj": ([vp, vp, vp, i, vp, i, vp], i),
            "sense_grad": ([vp, vp, vp, i, vp, vp, vp], i),
            "sketched_normal_apply": ([vp, vp, vp, i, vp, i, f, vp, vp], i),
            "coil_pca": ([vp, i, i64, vp, vp, vp], i), "coil_rotate": ([vp, vp, i, i, i64, vp, vp], i),
            "sketch_draw": ([u64, i, i, i, i, i, i, i, vp, vp], i), "cs_philox4x32_10": ([vp, vp, vp], i),
            "sketched_maps": ([vp, vp, i64, i, i, i, i, vp, vp], i),
            "recon_solve": ([vp, vp, vp, vp, vp, vp], i),
            "wavelet_fwd": ([vp, i, vp, i, vp, vp], i), "wavelet_inv": ([vp, i, vp, i, vp, vp], i),
            "soft_threshold": ([vp, i64, f, vp], i), "cs_hermitian_eig_host": ([vp, i, vp, vp], i),
            "cs_launch_count": ([], ctypes.c_longlong), "cs_profile": ([i], i),
            "cs_profile_read": ([i, vp, vp], i), "coil_pca_noalloc": ([vp, i, i64, vp, vp, vp], i),
            "cs_device_status": ([vp], i), "recon_solve_batched": ([i, vp, vp, vp, vp], i),
            "sketched_subproblem_solve": ([vp, vp, vp, vp, vp, i, vp, i, f, i, i, i, f, vp], i),
            "cs_subproblem_objective": ([vp, vp, vp, vp, vp, i, vp, i, f, i, i, vp, vp], i),
            "cs_power_iteration": ([vp, vp, vp, i, vp, i, i, vp, vp], i),
            "cs_nn_pack_weights": ([vp, i, i, i, vp, i, i, vp], i),
            "cs_nn_conv3d": ([vp, i, i, i, i, vp, i, i, i, vp, i, i, vp, i, i, vp], i),
            "cs_nn_conv3d_wgrad": ([vp, vp, i, i, i, i, i, vp, vp, vp], i),
            "cs_nn_relu_bwd": ([vp, vp, i64, vp], i), "cs_nn_conv1": ([vp, i64, i, i, vp, vp, vp, vp], i),
            "cs_nn_conv1_bwd": ([vp, vp, i64, i, i, vp, vp, vp, vp, vp], i),
            "cs_nn_mse": ([vp, vp, i64, vp, vp, vp], i), "cs_nn_adam": ([vp, vp, vp, vp, i64, f, f, f, f, i, vp], i),
            "cs_nn_features": ([vp, vp, i64, f, vp, vp, vp], i), "cs_nn_target": ([vp, vp, i64, vp, vp, vp], i),
            "cs_nn_apply": ([vp, vp, i64, vp, vp, vp], i), "cs_nn_status": ([vp], i),
            "tv_dual_update": ([vp, vp, vp, i, vp, f, f, vp], i),
            "cs_nn_maxpool2": ([vp, i, i, i, i, vp, vp, vp], i), "cs_nn_maxpool2_bwd": ([vp, vp, i, i, i, i, vp, vp], i),
            "cs_nn_upconv2": ([vp, i, i, i, i, vp, vp, i, vp, i, i, vp], i),
            "cs_nn_upconv2_bwd": ([vp, vp, i, i, i, i, i, i, vp, i, vp, vp, vp, vp], i),
            "cs_nn_slice": ([vp, i, i, i, vp, i, i, i64, i, vp], i),
            "tv_rhs": ([vp, vp, vp, i, vp, f, vp, vp, vp], i),
            "ws_net_create": ([i, i, i, u64, vp], i), "ws_net_destroy": ([vp], i),
            "ws_net_infer": ([vp, vp, vp, vp, f, vp, vp], i),
            "ws_net_train_step": ([vp, vp, vp, vp, vp, f, f, vp, vp], i),
            "ws_net_param": ([vp, i, i, vp, vp, vp, vp], i),
            "ws_net_save": ([vp, ctypes.c_char_p], i), "ws_net_load": ([vp, ctypes.c_char_p], i),
            "cs_crop3d": ([vp, vp, vp, vp, vp, vp], i), "cs_wait_selftest": ([i, i64, vp], i),
            "cs_plan_set_gridding": ([vp, i, i, i, i], i), "cs_plan_autotune": ([vp, i, i, vp, vp, vp], i),
            "cs_plan_set_deterministic": ([vp, i, i], i),
            "cs_plan_set_tile": ([vp, vp, vp], i), "cs_plan_autotune_tile": ([vp, i, i, vp, i, vp, vp, vp], i),
            "cs_noise_std": ([vp, i, i64, vp, vp], i), "cs_inverse_gfactor": ([vp, vp, i, i64, f, vp, vp], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(rc):
    if rc != CS_OK:
        raise CoilSketchError(rc, lib().cs_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors passed to libcoilsketch must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _dev(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    return t


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A cs_plan: image geometry + sampling operator (Cartesian mask or non-Cartesian NUFFT)."""

    def __init__(self, kind, img, max_coils, mask_idx=None, traj=None, dcf=None, grid=None, alpha=1.25,
                 tile=None, stream=None):
        g = _Geom()
        g.kind = kind
        g.ndim = len(img)
        for a, v in enumerate(img):
            g.img[a] = int(v)
        g.max_coils = int(max_coils)
        self._keep = []
        if kind == CARTESIAN:
            m = _dev(mask_idx, "mask_idx").to(torch.int32).contiguous()
            self._keep.append(m)
            g.mask_idx = m.data_ptr()
            g.nsamples = m.numel()
        else:
            tr = _dev(traj, "traj").to(torch.float32).contiguous()
            w = _dev(dcf, "dcf").to(torch.float32).contiguous()
            self._keep += [tr, w]
            g.traj, g.dcf = tr.data_ptr(), w.data_ptr()
            g.nsamples = tr.shape[0]
            for a, v in enumerate(grid):
                g.grid[a] = int(v)
            g.alpha = float(alpha)
            for a, v in enumerate(tile or (0,) * len(img)):
                g.tile[a] = int(v)
        self.kind, self.img, self.ndim = kind, tuple(int(v) for v in img), len(img)
        self.grid = tuple(int(v) for v in grid) if grid is not None else self.img
        self.nsamples = int(g.nsamples)
        self.max_coils = int(max_coils)
        h = ctypes.c_void_p()
        _check(lib().cs_plan_create(ctypes.byref(g), _stream(stream), ctypes.byref(h)))
        self._h = h
        self._keep = []

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().cs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gridding(self, interp_coils, interp_chunk, spread_coils, spread_chunk):
        """Coils and samples per warp of the gridding kernels (non-Cartesian plans)."""
        _check(lib().cs_plan_set_gridding(self._h, interp_coils, interp_chunk, spread_coils, spread_chunk))

    def set_deterministic(self, on=True, item_visits=0):
        """Owner-computes (atomics-free, bit-reproducible) spreading on or off; item_visits caps the
        sample visits of one spreading work item (0 = keep)."""
        _check(lib().cs_plan_set_deterministic(self.handle, int(bool(on)), int(item_visits)))

    def autotune(self, ncoils, reps=3, stream=None):
        """Time the gridding candidates for `ncoils` coils and keep the fastest; returns
        ((interp coils, interp chunk, spread coils, spread chunk), (best interp ms, best spread ms,
        interp ms before, spread ms before))."""
        choice = (ctypes.c_int * 4)()
        ms = (ctypes.c_float * 4)()
        _check(lib().cs_plan_autotune(self._h, ncoils, reps, choice, ms, _stream(stream)))
        return tuple(choice), tuple(float(v) for v in ms)

    def set_tile(self, tile, stream=None):
        """Re-bin a non-Cartesian plan for new tile sizes (one per axis, z y x order)."""
        t = (ctypes.c_int * len(tile))(*[int(v) for v in tile])
        _check(lib().cs_plan_set_tile(self._h, t, _stream(stream)))

    def autotune_tile(self, ncoils, candidates=(8, 16, 32), reps=3, stream=None):
        """Time interpolation + spreading of `ncoils` coils for each cubic tile candidate and keep
        the fastest; returns (best tile, ms per candidate)."""
        cand = (ctypes.c_int * len(candidates))(*[int(v) for v in candidates])
        ms = (ctypes.c_float * len(candidates))()
        best = ctypes.c_int(0)
        _check(lib().cs_plan_autotune_tile(self._h, ncoils, reps, cand, len(candidates), ctypes.byref(best), ms,
                                           _stream(stream)))
        return best.value, tuple(float(v) for v in ms)

    def binning(self):
        N = self.nsamples
        dev = torch.device("cuda")
        perm = torch.empty(N, dtype=torch.int32, device=dev)
        j0 = torch.empty((N, self.ndim), dtype=torch.int32, device=dev)
        nt = (ctypes.c_int * 3)()
        _check(lib().cs_plan_binning(self._h, None, None, None, nt, _stream()))
        ntot = nt[0] * nt[1] * nt[2]
        off = torch.empty(ntot + 1, dtype=torch.int32, device=dev)
        _check(lib().cs_plan_binning(self._h, _ptr(perm), _ptr(off), _ptr(j0), nt, _stream()))
        return perm, off, j0, tuple(nt)


def sense_fwd(plan: Plan, x, maps, y=None, stream=None):
    C = maps.shape[0]
    if y is None:
        y = torch.empty((C, plan.nsamples), dtype=torch.complex64, device=x.device)
    _check(lib().sense_fwd(plan.handle, _ptr(x), _ptr(maps), C, _ptr(y), _stream(stream)))
    return y


def sense_adj(plan: Plan, y, maps, x=None, accumulate=False, stream=None):
    C = maps.shape[0]
    if x is None:
        x = torch.empty(plan.img, dtype=torch.complex64, device=y.device)
    _check(lib().sense_adj(plan.handle, _ptr(y), _ptr(maps), C, _ptr(x), int(accumulate), _stream(stream)))
    return x


def sense_grad(plan: Plan, x, maps, y, d=None, stream=None):
    C = maps.shape[0]
    if d is None:
        d = torch.empty(plan.img, dtype=torch.complex64, device=x.device)
    _check(lib().sense_grad(plan.handle, _ptr(x), _ptr(maps), C, _ptr(y), _ptr(d), _stream(stream)))
    return d


def sketched_normal_apply(plan: Plan, v, maps_v, maps_s, lam, z=None, stream=None):
    V = 0 if maps_v is None else maps_v.shape[0]
    S = 0 if maps_s is None else maps_s.shape[0]
    if z is None:
        z = torch.empty(plan.img, dtype=torch.complex64, device=v.device)
    _check(lib().sketched_normal_apply(plan.handle, _ptr(v), _ptr(maps_v), V, _ptr(maps_s), S,
                                       ctypes.c_float(lam), _ptr(z), _stream(stream)))
    return z


def coil_pca(y, stream=None):
    C, N = y.shape
    U = torch.empty((C, C), dtype=torch.complex64, device=y.device)
    eig = torch.empty(C, dtype=torch.float64, device=y.device)
    _check(lib().coil_pca(_ptr(y), C, N, _ptr(U), _ptr(eig), _stream(stream)))
    return U, eig


def coil_pca_noalloc(y, U=None, eig=None, stream=None):
    """coil_pca without any device allocation inside the library (static 64 KiB scratch,
    at most 64 coils; concurrent calls race).  U and eig may be preallocated by the caller."""
    C, N = y.shape
    if U is None:
        U = torch.empty((C, C), dtype=torch.complex64, device=y.device)
    if eig is None:
        eig = torch.empty(C, dtype=torch.float64, device=y.device)
    _check(lib().coil_pca_noalloc(_ptr(y), C, N, _ptr(U), _ptr(eig), _stream(stream)))
    return U, eig


def coil_rotate(U, a, c_out=None, stream=None):
    C = a.shape[0]
    c_out = C if c_out is None else c_out
    L = a[0].numel()
    out = torch.empty((c_out,) + tuple(a.shape[1:]), dtype=torch.complex64, device=a.device)
    _check(lib().coil_rotate(_ptr(U), _ptr(a), C, c_out, L, _ptr(out), _stream(stream)))
    return out


def sketch_draw(seed, t0, T, C, V, S, dist=GAUSSIAN, norm=NORM_UNIT_VAR, device="cuda", stream=None):
    out = torch.empty((T, S, C - V), dtype=torch.float32, device=device)
    _check(lib().sketch_draw(ctypes.c_uint64(seed), t0, T, C, V, S, dist, norm, _ptr(out), _stream(stream)))
    return out


def philox4x32_10(ctr: Sequence[int], key: Sequence[int]):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    _check(lib().cs_philox4x32_10(c, k, o))
    return tuple(o)


def sketched_maps(S, maps_rot, V, precision=PREC_FP32, out=None, stream=None):
    C = maps_rot.shape[0]
    Sn = S.shape[0]
    D = maps_rot[0].numel()
    if out is None:
        out = torch.empty((Sn,) + tuple(maps_rot.shape[1:]), dtype=torch.complex64, device=maps_rot.device)
    _check(lib().sketched_maps(_ptr(S), _ptr(maps_rot), D, C, V, Sn, precision, _ptr(out), _stream(stream)))
    return out


def device_status(stream=None):
    """Synchronise the stream; raise CoilSketchError(CS_ERR_TIMEOUT) if a bounded device wait gave up."""
    _check(lib().cs_device_status(_stream(stream)))


def wavelet_fwd(x, levels=4, stream=None):
    dims = (ctypes.c_int * 3)(*x.shape)
    c = torch.empty_like(x)
    _check(lib().wavelet_fwd(_ptr(x), x.dim(), dims, levels, _ptr(c), _stream(stream)))
    return c


def wavelet_inv(c, levels=4, stream=None):
    dims = (ctypes.c_int * 3)(*c.shape)
    x = torch.empty_like(c)
    _check(lib().wavelet_inv(_ptr(c), c.dim(), dims, levels, _ptr(x), _stream(stream)))
    return x


def soft_threshold_(z, tau, stream=None):
    _check(lib().soft_threshold(_ptr(z), z.numel(), ctypes.c_float(tau), _stream(stream)))
    return z


def _require_c64(*ts):
    for v in ts:
        if v is not None and (v.dtype != torch.complex64 or not v.is_contiguous() or not v.is_cuda):
            raise ValueError("expected contiguous complex64 CUDA tensors")


def _dims(x, ndim):
    return (ctypes.c_int * ndim)(*[int(v) for v in x.shape[-ndim:]])


def tv_dual_update(x, z, sigma, lam, x_prev=None, stream=None):
    """In place: z <- proj_lam(z + sigma T (2 x - x_prev)) (x_prev None: T x); z [ndim, *x.shape]."""
    nd = x.dim()
    _require_c64(x, z, x_prev)
    if tuple(z.shape) != (nd,) + tuple(x.shape) or (x_prev is not None and x_prev.shape != x.shape):
        raise ValueError("tv_dual_update: z must be [ndim, *x.shape] and x_prev like x")
    _check(lib().tv_dual_update(_ptr(x), None if x_prev is None else _ptr(x_prev), _ptr(z), nd, _dims(x, nd),
                                float(sigma), float(lam), _stream(stream)))
    return z


def tv_rhs(x, z, inv_tau, b0=None, x_prev_out=None, stream=None):
    """rhs = b0 + inv_tau x - T^H z (b0 None: zero); x_prev_out (if given) receives x."""
    nd = x.dim()
    _require_c64(x, z, b0, x_prev_out)
    if tuple(z.shape) != (nd,) + tuple(x.shape) or any(v is not None and v.shape != x.shape for v in (b0, x_prev_out)):
        raise ValueError("tv_rhs: z must be [ndim, *x.shape], b0 and x_prev_out like x")
    rhs = torch.empty_like(x)
    _check(lib().tv_rhs(None if b0 is None else _ptr(b0), _ptr(x), _ptr(z), nd, _dims(x, nd), float(inv_tau),
                        _ptr(rhs), None if x_prev_out is None else _ptr(x_prev_out), _stream(stream)))
    return rhs


def hermitian_eig_host(A):
    """Run the library's FP64 Jacobi eigensolver on the host (numpy complex128 [n, n])."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    V = np.zeros((n, n), dtype=np.complex128)
    ev = np.zeros(n, dtype=np.float64)
    _check(lib().cs_hermitian_eig_host(A.ctypes.data_as(ctypes.c_void_p), n, V.ctypes.data_as(ctypes.c_void_p),
                                       ev.ctypes.data_as(ctypes.c_void_p)))
    return V, ev


def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(lib().cs_launch_count())


def profile(enable=True):
    """Reset the per-stage timers and turn CUDA-event recording on or off."""
    _check(lib().cs_profile(int(enable)))


def profile_read(stage):
    """(total device ms, launches) of a stage ('spread', 'interp', 'fft_plain', 'expand', 'reduce')."""
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(lib().cs_profile_read(STAGES[stage], ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


@dataclass
class SolveParams:
    T: int = 5
    K: int = 10
    sketch: bool = True
    V: int = 2
    S: int = 2
    dist: int = GAUSSIAN
    norm: int = NORM_UNIT_VAR
    seed: int = 4
    sketches: Optional[torch.Tensor] = None
    do_pca: bool = True
    precision: int = PREC_FP32
    step: float = 0.0
    power_iters: int = 20
    power_v0: Optional[torch.Tensor] = None
    use_graph: bool = False
    iterates: Optional[torch.Tensor] = None
    cg_iters: int = 0          # l1-TV: CG iterations per PDHG data step (0 = 5)
    tv_tau: float = 0.0        # l1-TV: PDHG steps (0 = 0.99 / sqrt(4 ndim))
    tv_sigma: float = 0.0
    init: bool = False         # classical-sketch initialisation (sketch block T; sketches hold T + 1)
    keep: int = 0              # plain solver on the first `keep` (virtual) coils (aggressive compression)
    sgd_batch: int = 0         # > 0: AccProxSGD with coil batches of this size (l1-wavelets)
    sgd_coils: Optional[torch.Tensor] = None   # int32 [K, sgd_batch] device coil indices
    sgd_beta: float = 0.0      # step decay (0 = 0.99)
    sgd_min: float = 0.0       # step floor as a fraction of alpha_0 (0 = 0.1)
    warm: Optional[object] = None          # warmstart.UNet: learned warm start (sketched l1-wavelet, 3D)
    x_ref: Optional[torch.Tensor] = None   # reference image for the trace's distance field
    trace: bool = False                    # record one trace row per outer iteration (plain: per iteration)
    trace_objective: bool = False          # add the objective to the trace (one extra forward per row)
    step_per_outer: int = 0                # sketched FISTA: re-estimate L with this many power iterations per outer


def recon_solve(plan: Plan, y, maps, lam, reg=REG_L2, params: SolveParams = None, x0=None, wavelet_levels=4,
                stream=None):
    """Algorithm 1 (params.sketch) or the plain full-coil solver; returns (x, stats dict)."""
    params = params or SolveParams()
    C = maps.shape[0]
    x = torch.zeros(plan.img, dtype=torch.complex64, device=y.device) if x0 is None else x0.clone()
    pr = _Problem(y=y.data_ptr(), maps=maps.data_ptr(), C=C, lam=float(lam), reg=int(reg),
                  wavelet_levels=int(wavelet_levels))
    sp = _params_struct(params)
    tr = None
    if params.trace:
        import numpy as np
        rows = params.T if params.sketch else params.K
        tr = np.full((max(rows, 1), TRACE_FIELDS), np.nan, dtype=np.float64)
        sp.trace = tr.ctypes.data
    st = _Stats()
    _check(lib().recon_solve(plan.handle, ctypes.byref(pr), ctypes.byref(sp), _ptr(x), ctypes.byref(st),
                             _stream(stream)))
    return x, {"L": st.L, "final_rr": st.final_rr, "outer_done": st.outer_done, "graph_used": st.graph_used,
               "ms_total": st.ms_total, "ms_pca": st.ms_pca, "warm_accepted": st.warm_accepted, "trace": tr}


def _params_struct(params: SolveParams):
    return _Params(T=params.T, K=params.K, sketch=int(params.sketch), V=params.V, S=params.S, dist=params.dist,
                   norm=params.norm, seed=params.seed,
                   sketches=None if params.sketches is None else params.sketches.data_ptr(),
                   do_pca=int(params.do_pca), precision=params.precision, step=float(params.step),
                   power_iters=params.power_iters,
                   power_v0=None if params.power_v0 is None else params.power_v0.data_ptr(),
                   use_graph=int(params.use_graph),
                   iterates=None if params.iterates is None else params.iterates.data_ptr(),
                   cg_iters=int(params.cg_iters), tv_tau=float(params.tv_tau), tv_sigma=float(params.tv_sigma),
                   init=int(params.init), keep=int(params.keep), sgd_batch=int(params.sgd_batch),
                   sgd_coils=None if params.sgd_coils is None else params.sgd_coils.data_ptr(),
                   sgd_beta=float(params.sgd_beta), sgd_min=float(params.sgd_min),
                   warm=None if params.warm is None else params.warm._h.value,
                   x_ref=None if params.x_ref is None else params.x_ref.data_ptr(),
                   trace=None, trace_objective=int(params.trace_objective),
                   step_per_outer=int(params.step_per_outer))


def recon_solve_batched(items, lam, reg=REG_L2, params: SolveParams = None, wavelet_levels=4, stream=None):
    """Independent reconstructions (plan, y, maps[, x0][, power_v0]) in one call; with
    params.use_graph all of them run as one cached CUDA graph.  Returns (list of x, list of stats)."""
    params = params or SolveParams()
    n = len(items)
    arr = (_BatchItem * n)()
    xs = []
    for i, it in enumerate(items):
        plan, y, maps = it["plan"], it["y"], it["maps"]
        x = it.get("x0")
        x = torch.zeros(plan.img, dtype=torch.complex64, device=y.device) if x is None else x.clone()
        xs.append(x)
        v0 = it.get("power_v0")
        arr[i].plan = plan.handle.value
        arr[i].problem = _Problem(y=y.data_ptr(), maps=maps.data_ptr(), C=maps.shape[0], lam=float(lam), reg=int(reg),
                                  wavelet_levels=int(wavelet_levels))
        arr[i].x_inout = x.data_ptr()
        arr[i].power_v0 = None if v0 is None else v0.data_ptr()
    sp = _params_struct(params)
    st = (_Stats * n)()
    _check(lib().recon_solve_batched(n, arr, ctypes.byref(sp), st, _stream(stream)))
    return xs, [{"L": s.L, "final_rr": s.final_rr, "graph_used": s.graph_used} for s in st]


def sketched_subproblem_solve(plan: Plan, d, xt, x, maps_v, maps_s, lam, reg, K, step=0.0, wavelet_levels=4,
                              stream=None):
    """K solver iterations on the sketched sub-problem (Eq. 9-10) from x (in place); x^t = xt."""
    V = 0 if maps_v is None else maps_v.shape[0]
    S = 0 if maps_s is None else maps_s.shape[0]
    _check(lib().sketched_subproblem_solve(plan.handle, _ptr(d), _ptr(xt), _ptr(x), _ptr(maps_v), V, _ptr(maps_s), S,
                                           ctypes.c_float(lam), int(reg), int(wavelet_levels), int(K),
                                           ctypes.c_float(step), _stream(stream)))
    return x


def subproblem_objective(plan: Plan, u, xt, d, maps_v, maps_s, lam, reg, wavelet_levels=4, stream=None):
    V = 0 if maps_v is None else maps_v.shape[0]
    S = 0 if maps_s is None else maps_s.shape[0]
    out = ctypes.c_double()
    _check(lib().cs_subproblem_objective(plan.handle, _ptr(u), _ptr(xt), _ptr(d), _ptr(maps_v), V, _ptr(maps_s), S,
                                         ctypes.c_float(lam), int(reg), int(wavelet_levels), ctypes.byref(out),
                                         _stream(stream)))
    return out.value


def power_iteration(plan: Plan, v0, maps_v, maps_s, iters=20, stream=None):
    V = 0 if maps_v is None else maps_v.shape[0]
    S = 0 if maps_s is None else maps_s.shape[0]
    out = ctypes.c_double()
    _check(lib().cs_power_iteration(plan.handle, _ptr(v0), _ptr(maps_v), V, _ptr(maps_s), S, int(iters),
                                    ctypes.byref(out), _stream(stream)))
    return out.value
