"""Inverse g-factor by Monte Carlo pseudo-replicas (the paper's Sec. 3.2 noise analysis, after
Pruessmann et al. 1999 and Robson et al. 2008): one Cartesian acquisition plus independent
noise realisations, every replica reconstructed by one batched solve (one plan per replica; with
``use_graph`` all replicas run as one captured CUDA graph), then the per-pixel noise standard
deviation over replicas, g = std_R / (std_full sqrt(R)).

The noise realisations are inputs (device tensors [replicas][C][N]); the solver is whatever
``params`` selects (coil sketching or the plain full-coil solver, l2 regularisation).
"""
from __future__ import annotations

import ctypes

import torch

from . import CARTESIAN, REG_L2, Plan, SolveParams, _check, _ptr, _stream, lib, recon_solve_batched


def replicas(y, noise):
    """The noisy copies y + noise[k] (kept: a captured graph refers to their addresses)."""
    return [(y + noise[k]).contiguous() for k in range(noise.shape[0])]


def replica_reconstructions(shape, maps, mask_idx, ys, lam, params: SolveParams, plans=None):
    """Reconstruct every replica in ys; returns ([replicas, *shape] complex64, plans).  Passing the
    plans of an earlier call with the same replicas replays its cached graph."""
    C = maps.shape[0]
    if plans is None:
        plans = [Plan(CARTESIAN, shape, C, mask_idx=mask_idx) for _ in range(len(ys))]
    items = [dict(plan=pl, y=yk, maps=maps) for pl, yk in zip(plans, ys)]
    xs, _ = recon_solve_batched(items, lam, REG_L2, params)
    return torch.stack(xs), plans


def noise_std(recons, stream=None):
    """Per-pixel sqrt(mean_k |x_k - mean|^2) over the first axis (library kernel, FP64 per pixel)."""
    K = recons.shape[0]
    D = recons[0].numel()
    out = torch.empty(recons.shape[1:], dtype=torch.float32, device=recons.device)
    _check(lib().cs_noise_std(_ptr(recons), K, D, _ptr(out), _stream(stream)))
    return out


def inverse_gfactor(recons_R, recons_full, R, stream=None):
    """1/g = std_full sqrt(R) / std_R (library kernel)."""
    K = recons_R.shape[0]
    D = recons_R[0].numel()
    out = torch.empty(recons_R.shape[1:], dtype=torch.float32, device=recons_R.device)
    _check(lib().cs_inverse_gfactor(_ptr(recons_R.contiguous()), _ptr(recons_full.contiguous()), K, D,
                                    ctypes.c_float(R), _ptr(out), _stream(stream)))
    return out
