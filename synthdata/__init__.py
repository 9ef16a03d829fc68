"""Seeded synthetic inputs for coil-sketched MR reconstruction.

Stand-ins for the paper's datasets (Sec. 3.1: a Cartesian knee, a 2D radial liver and
two 3D cones abdominal acquisitions), none of which is available here.  Every generator
is seeded and returns plain NumPy arrays; this module contains no step of the
reconstruction method itself (no Fourier transform, no sensitivity product, no solver),
so both the CPU oracle and the GPU path can consume its outputs without sharing any of
the method's arithmetic.

Recipes (shapes follow the paper's workloads and the benchmark configurations):

* phantom: 12 random ellipses/ellipsoids (3 of them negative "holes"), centres uniform
  inside 0.8 FOV, semi-axes 0.05-0.4 FOV, random rotation, intensities U[0.1, 1];
  smooth random phase built from low-order Fourier modes, bounded by pi/2;
  scaled to max |x| = 1.
* maps: Gaussian profiles (width 0.35 FOV) centred on a ring of radius 0.75 FOV/2
  (3D: nc/8 rings of 8 stacked evenly in z), coil phase 2 pi c / nc, normalised to a
  root-sum-of-squares of 1 in every voxel (an ESPIRiT-like normalisation).
* Poisson-disc variable-density mask with a fully sampled centre (2D Cartesian, R=4).
* line mask: fully sampled centre lines plus lines drawn without replacement with
  density (1 - |ky|/(n/2))^2 (2D Cartesian, R=6).
* cones: a spiral-cones stand-in. Interleave i has axis polar angle
  arccos(1 - (2i+1)/n_int) and azimuth i*pi*(3-sqrt 5); readout point p has radius
  0.5 p/(n_read-1) and azimuth offset 2 pi t s^2 (s = p/(n_read-1)) with t = 0.25 turns, so
  consecutive samples along a readout stay below one pixel (1/FOV) apart, as on a scanner
  readout; a faster twist would undersample the readout itself.
* dcf: analytic radial density compensation w = D 4 pi max(|f|, kmin)^2 / (n_int
  dk^-1), i.e. the inverse of the sample density of the cones stand-in, so that A^H A is
  close to the identity on the sampled ball.
* noise: complex Gaussian with a given standard deviation.
"""
from __future__ import annotations

import math
import numpy as np

__all__ = [
    "phantom", "phantom_torch", "coil_maps", "coil_maps_torch", "poisson_disc_mask", "line_mask", "regular_mask",
    "cones_trajectory", "cones_dcf", "radial_trajectory", "radial_dcf", "complex_noise", "random_complex",
    "slice_sizes", "CONFIGS",
]


def _rng(seed):
    return np.random.default_rng(seed)


def _phantom_params(shape, seed, n_obj, n_holes):
    nd = len(shape)
    rng = _rng(seed)
    objs = []
    for k in range(n_obj):
        centre = rng.uniform(-0.8, 0.8, size=nd)
        semi = rng.uniform(0.05, 0.4, size=nd) * 2.0  # FOV spans 2 in these units
        q, r = np.linalg.qr(rng.standard_normal((nd, nd)))
        q = q * np.sign(np.diag(r))
        amp = rng.uniform(0.1, 1.0)
        if k >= n_obj - n_holes:
            amp = -amp
        objs.append((centre, semi, q, amp))
    rng_m = _rng(seed + 1000)
    modes = []
    for m in np.stack(np.meshgrid(*([range(-2, 3)] * nd), indexing="ij"), -1).reshape(-1, nd):
        a = rng_m.standard_normal() + 1j * rng_m.standard_normal()
        modes.append((m, a))
    return objs, modes


def phantom(shape, seed=1, n_obj=12, n_holes=3):
    """Random-ellipse (2D) or random-ellipsoid (3D) phantom, complex128, max|x| = 1."""
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    objs, modes = _phantom_params(shape, seed, n_obj, n_holes)
    # normalised coordinates in [-1, 1) per axis, axis order (z, y, x) / (y, x)
    grids = np.meshgrid(*[(np.arange(n) - n / 2) / (n / 2) for n in shape], indexing="ij")
    coords = np.stack(grids, axis=-1)  # [..., nd]
    mag = np.zeros(shape)
    for centre, semi, q, amp in objs:
        rel = (coords - centre) @ q
        inside = np.sum((rel / semi) ** 2, axis=-1) <= 1.0
        mag = mag + amp * inside
    mag = np.abs(mag)
    phase = np.zeros(shape)
    for m, a in modes:
        arg = sum(m[i] * grids[i] * 0.5 for i in range(nd))  # grids in [-1,1): r/n = g/2
        phase = phase + np.real(a * np.exp(2j * np.pi * arg))
    phase = phase * (math.pi / 2) / max(np.abs(phase).max(), 1e-30)
    x = mag * np.exp(1j * phase)
    x = x / np.abs(x).max()
    return x.astype(np.complex128)


def phantom_torch(shape, seed=1, device="cuda", n_obj=12, n_holes=3):
    """phantom() evaluated with torch on a device in float32/complex64 (large volumes)."""
    import torch
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    objs, modes = _phantom_params(shape, seed, n_obj, n_holes)
    axes = [(torch.arange(n, device=device, dtype=torch.float32) - n / 2) / (n / 2) for n in shape]
    grids = torch.meshgrid(*axes, indexing="ij")
    mag = torch.zeros(shape, device=device)
    for centre, semi, q, amp in objs:
        acc = torch.zeros(shape, device=device)
        for j in range(nd):
            relj = sum((grids[i] - float(centre[i])) * float(q[i, j]) for i in range(nd))
            acc += (relj / float(semi[j])) ** 2
        mag += float(amp) * (acc <= 1.0).float()
    mag = mag.abs()
    phase = torch.zeros(shape, device=device)
    for m, a in modes:
        arg = sum(float(m[i]) * grids[i] * 0.5 for i in range(nd))
        phase += float(a.real) * torch.cos(2 * math.pi * arg) - float(a.imag) * torch.sin(2 * math.pi * arg)
    phase = phase * (math.pi / 2) / phase.abs().max().clamp_min(1e-30)
    x = torch.polar(mag, phase)
    return (x / x.abs().max()).to(torch.complex64)


def _coil_centres(nd, nc):
    radius = 0.75 * 0.5
    out = []
    for c in range(nc):
        if nd == 2:
            ang = 2 * math.pi * c / nc
            out.append((radius * math.sin(ang), radius * math.cos(ang)))
        else:
            per_ring = 8
            n_rings = max(1, nc // per_ring)
            ring = min(c // per_ring, n_rings - 1)
            k = c % per_ring
            ang = 2 * math.pi * k / per_ring + (math.pi / per_ring) * (ring % 2)
            pz = ((ring + 0.5) / n_rings - 0.5) * 0.8
            out.append((pz, radius * math.sin(ang), radius * math.cos(ang)))
    return out


def coil_maps(shape, nc, width=0.35):
    """Gaussian-profile coil sensitivities on a ring, RSS-normalised. complex128 [nc, *shape]."""
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    grids = np.meshgrid(*[(np.arange(n) - n / 2) / n for n in shape], indexing="ij")  # FOV units
    maps = np.empty((nc,) + shape, dtype=np.complex128)
    for c, p in enumerate(_coil_centres(nd, nc)):
        d2 = sum((grids[i] - p[i]) ** 2 for i in range(nd))
        maps[c] = np.exp(-d2 / (2 * width ** 2)) * np.exp(1j * 2 * math.pi * c / nc)
    rss = np.sqrt(np.sum(np.abs(maps) ** 2, axis=0))
    return maps / rss


def coil_maps_torch(shape, nc, width=0.35, device="cuda"):
    """coil_maps() evaluated with torch on a device, complex64 [nc, *shape]."""
    import torch
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    axes = [(torch.arange(n, device=device, dtype=torch.float32) - n / 2) / n for n in shape]
    grids = torch.meshgrid(*axes, indexing="ij")
    maps = torch.empty((nc,) + shape, dtype=torch.complex64, device=device)
    rss = torch.zeros(shape, device=device)
    for c, p in enumerate(_coil_centres(nd, nc)):
        d2 = sum((grids[i] - float(p[i])) ** 2 for i in range(nd))
        mag = torch.exp(-d2 / (2 * width ** 2))
        maps[c] = torch.polar(mag, torch.full_like(mag, 2 * math.pi * c / nc))
        rss += mag * mag
    return maps / rss.sqrt().unsqueeze(0)


def _disc_sample(n, r_of, centre, rng):
    """Dart throwing over grid points in random order with a spatially varying radius."""
    ny, nx = n
    ky = (np.arange(ny) - ny // 2)
    kx = (np.arange(nx) - nx // 2)
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    kr = np.sqrt((KY / (ny / 2)) ** 2 + (KX / (nx / 2)) ** 2)
    rad = r_of(kr)
    mask = np.zeros((ny, nx), dtype=bool)
    c0y, c0x = ny // 2 - centre // 2, nx // 2 - centre // 2
    mask[c0y:c0y + centre, c0x:c0x + centre] = True
    order = rng.permutation(ny * nx)
    rmax = int(math.ceil(rad.max()))
    for idx in order:
        y, x = divmod(int(idx), nx)
        if mask[y, x]:
            continue
        r = rad[y, x]
        ri = int(math.ceil(r))
        y0, y1 = max(0, y - ri), min(ny, y + ri + 1)
        x0, x1 = max(0, x - ri), min(nx, x + ri + 1)
        sub = mask[y0:y1, x0:x1]
        if sub.any():
            yy, xx = np.nonzero(sub)
            d2 = (yy + y0 - y) ** 2 + (xx + x0 - x) ** 2
            if d2.min() < r * r:
                continue
        mask[y, x] = True
    del rmax
    return mask


def poisson_disc_mask(n, R=4.0, centre=24, seed=2, tol=0.01):
    """Variable-density Poisson-disc mask (radius r0 (1 + 3 |k|/kmax)) with a fully sampled
    centre; r0 found by bisection so that the acceleration is R within tol. bool [ny, nx]."""
    n = (int(n[0]), int(n[1])) if not isinstance(n, int) else (n, n)
    target = n[0] * n[1] / R
    lo, hi = 0.3, 4.0
    best = None
    for _ in range(30):
        r0 = 0.5 * (lo + hi)
        m = _disc_sample(n, lambda kr: r0 * (1 + 3 * kr), centre, _rng(seed))
        cnt = m.sum()
        best = m
        if abs(cnt - target) <= tol * target:
            break
        if cnt > target:
            lo = r0
        else:
            hi = r0
    return best


def line_mask(n, R=6.0, centre_lines=24, seed=2):
    """Phase-encode line mask (rows = ky lines, readout along x fully sampled). bool [ny, nx]."""
    ny, nx = (int(n[0]), int(n[1])) if not isinstance(n, int) else (n, n)
    rng = _rng(seed)
    nlines = int(round(ny / R))
    sel = np.zeros(ny, dtype=bool)
    c0 = ny // 2 - centre_lines // 2
    sel[c0:c0 + centre_lines] = True
    ky = np.arange(ny) - ny // 2
    pdf = (1 - np.abs(ky) / (ny / 2)) ** 2
    pdf[sel] = 0
    pdf = pdf / pdf.sum()
    need = max(0, nlines - int(sel.sum()))
    extra = rng.choice(ny, size=need, replace=False, p=pdf)
    sel[extra] = True
    mask = np.zeros((ny, nx), dtype=bool)
    mask[sel, :] = True
    return mask


def cones_trajectory(n_int, n_read=512, turns=0.25):
    """Spiral-cones stand-in, float32 [n_int*n_read, 3] in cycles/pixel, axis order (z, y, x)."""
    i = np.arange(n_int, dtype=np.float64)[:, None]
    p = np.arange(n_read, dtype=np.float64)[None, :]
    theta = np.arccos(1.0 - (2.0 * i + 1.0) / n_int)
    phi0 = i * math.pi * (3.0 - math.sqrt(5.0))
    s = p / (n_read - 1)
    kr = 0.5 * s
    phi = phi0 + 2 * math.pi * turns * s ** 2
    kx = kr * np.sin(theta) * np.cos(phi)
    ky = kr * np.sin(theta) * np.sin(phi)
    kz = kr * np.cos(theta) * np.ones_like(phi)
    traj = np.stack([kz, ky, kx], axis=-1).reshape(-1, 3)
    return traj.astype(np.float32)


def cones_dcf(traj, img_shape, n_int, n_read=512):
    """Analytic radial density compensation of the cones stand-in, float32 [N]."""
    D = float(np.prod(img_shape))
    kr = np.sqrt(np.sum(traj.astype(np.float64) ** 2, axis=-1))
    dk = 0.5 / (n_read - 1)
    kmin = 0.5 * dk
    w = D * 4 * math.pi * np.maximum(kr, kmin) ** 2 * dk / n_int
    return w.astype(np.float32)


def regular_mask(n, R=3, offset=0):
    """Regular undersampling: every R-th phase-encode line (rows), readout fully sampled.
    bool [ny, nx]."""
    ny, nx = (int(n[0]), int(n[1])) if not isinstance(n, int) else (n, n)
    m = np.zeros((ny, nx), dtype=bool)
    m[offset::R, :] = True
    return m


def radial_trajectory(n_spokes, n_read=256):
    """2D golden-angle radial stand-in (full spokes through the centre), float32
    [n_spokes*n_read, 2] in cycles/pixel, axis order (y, x), radius in [-0.5, 0.5)."""
    i = np.arange(n_spokes, dtype=np.float64)[:, None]
    p = np.arange(n_read, dtype=np.float64)[None, :]
    ang = i * math.pi * (math.sqrt(5.0) - 1.0) / 2.0
    kr = (p - n_read / 2) / n_read
    traj = np.stack([kr * np.sin(ang), kr * np.cos(ang)], axis=-1).reshape(-1, 2)
    return traj.astype(np.float32)


def radial_dcf(traj, img_shape, n_spokes, n_read=256):
    """Analytic density compensation of the radial stand-in (ring spacing pi |k| / n_spokes
    times the readout spacing), float32 [N]."""
    D = float(np.prod(img_shape))
    kr = np.sqrt(np.sum(traj.astype(np.float64) ** 2, axis=-1))
    dk = 1.0 / n_read
    w = D * math.pi * np.maximum(kr, 0.25 * dk) * dk / n_spokes
    return w.astype(np.float32)


def complex_noise(shape, sigma, seed=3):
    rng = _rng(seed)
    return (sigma / math.sqrt(2)) * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def random_complex(shape, seed):
    rng = _rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def slice_sizes(n_slices=64, choices=(256, 288, 320, 352, 384), seed=10):
    rng = _rng(seed)
    return [int(v) for v in rng.choice(np.array(choices), size=n_slices)]


# Benchmark configurations (sizes of the paper-shaped synthetic workloads).
CONFIGS = {
    "cart2d_128": dict(kind="cartesian", img=(128, 128), nc=8, R=4.0, centre=24, lam=1e-3,
                        V=2, S=2, T=5, K=10, reg="l2"),
    "cart2d_batched": dict(kind="cartesian_batched", n_slices=64, nc=16, R=6.0, centre=24,
                           lam=5e-3, V=3, S=3, reg="l1wav"),
    "cones3d_128": dict(kind="nufft", img=(128, 128, 128), grid=(160, 160, 160), nc=32,
                        n_int=6000, n_read=512, lam=1e-3, V=4, S=4, reg="l2"),
    "cones3d_large": dict(kind="nufft", img=(160, 256, 256), grid=(200, 320, 320), nc=40,
                          n_int=20000, n_read=512, lam=2e-3, V=5, S=5, reg="l1wav"),
}
