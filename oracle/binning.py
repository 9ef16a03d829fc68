"""Grid coordinates, Kaiser-Bessel kernel boxes and the stable tile sort of NUFFT samples.

The paper implements the non-uniform operator F~_n with gridding (Sec. 2.1, citing Beatty et
al. 2005) and gives no discretisation details; these are the readings used on both sides:

* grid coordinate per axis: g = fmaf(f, G, G/2) computed once-rounded in IEEE float32
  (f in cycles/pixel, G the oversampled grid size), so that integer decisions are identical
  on CPU and GPU;
* kernel box of width W = 4: the W grid indices j0 .. j0+W-1 with j0 = floor(g) - 1
  (= floor(g - W/2) + 1 for even W), wrapped modulo G;
* tile of a sample: floor(wrap(j0) / T) per axis, linearised (z, y, x) with x fastest; an axis
  whose last tile would be narrower than the kernel (G mod T in 1..W-1) folds that remainder
  into the previous tile, so that no box spans more than two tiles;
* halo class of a sample: bit a (z = 4, y = 2, x = 1) is set when its box reaches past its own
  tile into the next tile along axis a (wrapping), i.e. wrap(j0) - tile start >= tile width - W + 1,
  and only on axes with more than one tile.  Each tile's grid points are accumulated from its own
  samples and from the samples of its lower neighbours whose class reaches it;
* samples are ordered by a stable counting sort on the key tile * 8 + class.
"""
from __future__ import annotations

import numpy as np

KB_WIDTH = 4


def fmaf32(a, b, c):
    """Correctly rounded float32 fused multiply-add of float32 inputs (vectorised).

    a*b is exact in float64 (24x24 bits); the float64 sum s = a*b + c carries an exact
    error term e (Knuth TwoSum).  Rounding s to float32 is correct unless s lies exactly on a
    float32 midpoint while e != 0; in that case we round towards the side e points to.
    """
    a = np.asarray(a, dtype=np.float32).astype(np.float64)
    b = np.asarray(b, dtype=np.float32).astype(np.float64)
    c = np.asarray(c, dtype=np.float32).astype(np.float64)
    p = a * b
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)
    r = s.astype(np.float32)
    r64 = r.astype(np.float64)
    towards = np.where(s > r64, np.float32(np.inf), np.float32(-np.inf))
    r2 = np.nextafter(r, towards.astype(np.float32))
    mid = 0.5 * (r64 + r2.astype(np.float64))
    fix = (s != r64) & (s == mid) & (e != 0)
    # exact value lies on the side of e: if e moves towards r2, take r2
    take_r2 = fix & (np.sign(e) == np.sign(r2.astype(np.float64) - s))
    take_r = fix & ~take_r2
    out = np.where(take_r2, r2, r)
    out = np.where(take_r, r, out)
    return out.astype(np.float32)


def grid_coords(traj, grid):
    """g[i, ax] = fmaf32(f[i, ax], G_ax, G_ax/2), float32 [N, nd]."""
    traj = np.asarray(traj, dtype=np.float32)
    G = np.asarray(grid, dtype=np.float32)[None, :]
    return fmaf32(traj, G, G * np.float32(0.5))


def kernel_box_start(g):
    """First grid index j0 = floor(g) - W/2 + 1 of each sample's W-point box (int64, unwrapped)."""
    return np.floor(np.asarray(g, dtype=np.float64)).astype(np.int64) - (KB_WIDTH // 2 - 1)


def tiles_per_axis(grid, tile):
    """Tiles along each axis: ceil(G / T), or floor(G / T) when the remainder is narrower than
    the kernel (it then widens the last tile)."""
    grid = np.asarray(grid, dtype=np.int64)
    tile = np.asarray(tile, dtype=np.int64)
    rem = grid % tile
    return np.where((rem > 0) & (rem < KB_WIDTH) & (grid >= tile), grid // tile, -(-grid // tile))


def _axis_tiles(j0, grid, tile):
    grid = np.asarray(grid, dtype=np.int64)
    tile = np.asarray(tile, dtype=np.int64)
    nt = tiles_per_axis(grid, tile)
    jw = np.mod(j0, grid[None, :])
    t = np.minimum(jw // tile[None, :], nt[None, :] - 1)
    start = t * tile[None, :]
    width = np.where(t == nt[None, :] - 1, grid[None, :] - start, tile[None, :])
    return t, nt, jw, start, width


def tile_ids(j0, grid, tile):
    """Linear tile id of each sample from its wrapped box start, (z, y, x) with x fastest."""
    t, ntiles, _, _, _ = _axis_tiles(j0, grid, tile)
    lin = np.zeros(j0.shape[0], dtype=np.int64)
    for ax in range(j0.shape[1]):
        lin = lin * ntiles[ax] + t[:, ax]
    return lin, ntiles


def halo_class(j0, grid, tile):
    """Bits (z = 4, y = 2, x = 1 for 3D; y = 2, x = 1 for 2D) of the axes along which a sample's box
    reaches into the next tile (only axes with more than one tile)."""
    t, nt, jw, start, width = _axis_tiles(j0, grid, tile)
    nd = j0.shape[1]
    cls = np.zeros(j0.shape[0], dtype=np.int64)
    for ax in range(nd):
        reach = (jw[:, ax] - start[:, ax] >= width[:, ax] - (KB_WIDTH - 1)) & (nt[ax] > 1)
        cls |= reach.astype(np.int64) << (nd - 1 - ax)
    return cls


def sort_keys(j0, grid, tile):
    """Sort key tile * 8 + halo class of every sample, and the tiles per axis."""
    lin, nt = tile_ids(j0, grid, tile)
    return lin * 8 + halo_class(j0, grid, tile), nt


def tile_sort(tid, n_tiles_total):
    """Stable counting sort: permutation (sorted position -> sample index) and tile offsets."""
    counts = np.bincount(tid, minlength=n_tiles_total)
    offsets = np.zeros(n_tiles_total + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    perm = np.empty(tid.shape[0], dtype=np.int64)
    cursor = offsets[:-1].copy()
    for i, t in enumerate(tid):  # literal stable counting sort (slow; test sizes only)
        perm[cursor[t]] = i
        cursor[t] += 1
    return perm, offsets


def tile_sort_fast(tid, n_tiles_total):
    """Same result as tile_sort via a stable library sort (used for larger inputs)."""
    perm = np.argsort(tid, kind="stable")
    counts = np.bincount(tid, minlength=n_tiles_total)
    offsets = np.zeros(n_tiles_total + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    return perm, offsets


def sample_order(j0, grid, tile):
    """The plan's sample order: permutation (sorted position -> sample index) by the stable key
    tile * 8 + halo class, and the per-tile offsets [ntiles + 1]."""
    key, nt = sort_keys(j0, grid, tile)
    ntot = int(np.prod(nt))
    perm = np.argsort(key, kind="stable")
    counts = np.bincount(key // 8, minlength=ntot)
    offsets = np.zeros(ntot + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    return perm, offsets, nt
