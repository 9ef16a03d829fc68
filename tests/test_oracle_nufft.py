"""Pins for the gridding NUFFT oracle: KB transform closed form vs quadrature, gridding vs the
exact non-uniform DFT of Eq. 1 (the gridding error is reported and bounded), exact
adjointness, NUDFT vs the Cartesian DFT on grid frequencies, and bit-level binning checks."""
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate

import synthdata
from oracle import binning, fourier, nufft


def test_kb_transform_closed_form_matches_quadrature():
    beta = nufft.kb_beta()
    assert 6.99 < beta < 7.0
    for nu in [0.0, 0.05, 0.13, 0.27, 0.4, 0.6]:
        re, _ = integrate.quad(lambda u: nufft.kb_phi(u, beta) * np.cos(2 * np.pi * u * nu), -2, 2,
                               limit=200, epsabs=1e-13)
        assert abs(re - nufft.kb_phi_hat(nu, beta)) <= 1e-10


@pytest.mark.parametrize("img,grid,alpha,bound", [
    ((8, 8, 8), (10, 10, 10), 1.25, 1.5e-2), ((16, 12), (20, 15 + 1), 1.25, 1.5e-2),
    ((16, 16, 8), (20, 20, 10), 1.25, 1.5e-2),
    ((8, 8, 8), (16, 16, 16), 2.0, 1.5e-3), ((32, 32), (64, 64), 2.0, 1.5e-3)])
def test_gridding_approximates_exact_nudft(img, grid, alpha, bound):
    rng = np.random.default_rng(11)
    N = 600
    traj = rng.uniform(-0.5, 0.5, size=(N, len(img))).astype(np.float32)
    dcf = rng.uniform(0.5, 1.5, N).astype(np.float32)
    x = synthdata.random_complex(img, 12)
    maps = synthdata.random_complex((2,) + img, 13)
    exact = nufft.nudft_fwd(x, maps, traj, dcf)
    plan = nufft.Plan(traj, img, grid, alpha=alpha)
    approx = nufft.sense_fwd(plan, x, maps, dcf)
    err = np.linalg.norm(approx - exact) / np.linalg.norm(exact)
    # W = 4 Kaiser-Bessel gridding of a white-noise image: below 1e-2 at alpha = 1.25 and
    # an order of magnitude lower at alpha = 2 (a wrong term would give an O(1) error)
    assert err < bound, err


def test_gridding_adjoint_is_exact():
    img, grid = (8, 10, 12), (10, 12, 16)
    rng = np.random.default_rng(21)
    traj = rng.uniform(-0.5, 0.5, size=(500, 3)).astype(np.float32)
    dcf = rng.uniform(0.1, 1, 500).astype(np.float32)
    plan = nufft.Plan(traj, img, grid)
    maps = synthdata.random_complex((3,) + img, 22)
    x = synthdata.random_complex(img, 23)
    y = synthdata.random_complex((3, 500), 24)
    lhs = np.vdot(nufft.sense_fwd(plan, x, maps, dcf), y)
    rhs = np.vdot(x, nufft.sense_adj(plan, y, maps, dcf))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_nudft_on_grid_frequencies_equals_cartesian_dft():
    shape = (6, 8)
    maps = synthdata.random_complex((2,) + shape, 31)
    x = synthdata.random_complex(shape, 32)
    idx = np.arange(48)
    f = fourier.sampled_frequencies(shape, idx)
    a = nufft.nudft_fwd(x, maps, f, np.ones(48))
    b = fourier.cartesian_fwd(x, maps, idx)
    assert np.abs(a - b).max() <= 1e-12


def _fmaf_exact(a, b, c):
    """Brute force: nearest float32 (ties to even) to the exact rational a*b + c."""
    ex = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    r = np.float32(float(ex))
    cands = [np.nextafter(r, np.float32(-np.inf)), r, np.nextafter(r, np.float32(np.inf))]
    dist = [abs(Fraction(float(v)) - ex) for v in cands]
    best = min(dist)
    ties = [v for v, dd in zip(cands, dist) if dd == best]
    if len(ties) == 1:
        return ties[0]
    return [v for v in ties if (np.array(v, np.float32).view(np.uint32) & 1) == 0][0]


def test_fmaf32_is_correctly_rounded():
    rng = np.random.default_rng(41)
    a = np.concatenate([rng.uniform(-0.5, 0.5, 3000), rng.uniform(-1e-6, 1e-6, 500),
                        np.array([0.5, -0.5, 0.0, 2.0 ** -30, -(2.0 ** -30), 0.25 - 2 ** -26])]).astype(np.float32)
    for G in [160.0, 200.0, 320.0, 10.0]:
        got = binning.fmaf32(a, np.float32(G), np.float32(G / 2))
        want = np.array([_fmaf_exact(v, G, G / 2) for v in a], dtype=np.float32)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_box_and_tile_sort():
    traj = synthdata.cones_trajectory(40, 64)
    grid = (20, 20, 20)
    g = binning.grid_coords(traj, grid).astype(np.float64)
    j0 = binning.kernel_box_start(g)
    off = g - j0
    assert np.all(off >= 1) and np.all(off < 2)        # box = the 4 integers with -2 <= g-j < 2
    tid, nt = binning.tile_ids(j0, grid, (8, 8, 8))
    assert tuple(nt) == (3, 3, 3) and tid.max() < 27
    perm, offs = binning.tile_sort(tid, 27)
    p2, o2 = binning.tile_sort_fast(tid, 27)
    assert np.array_equal(perm, p2) and np.array_equal(offs, o2)
    st = tid[perm]
    assert np.all(np.diff(st) >= 0)
    for t in range(27):
        seg = perm[offs[t]:offs[t + 1]]
        assert np.all(np.diff(seg) > 0)                   # stable
        assert np.all(tid[seg] == t)


@pytest.mark.parametrize("grid,tile", [((20, 20, 20), (8, 8, 8)), ((18, 26, 40), (8, 8, 16)), ((16, 12), (16, 8))])
def test_halo_classes_and_tile_owners_by_brute_force(grid, tile):
    """The halo class of every sample against its box's grid indices, tile by tile: every box index
    lies in the sample's own tile or the next one along each axis (remainders narrower than the
    kernel fold into the last tile: 18 = 8 + 10, 26 = 8 + 8 + 10), a class bit is set exactly when
    the box reaches the next tile, and the samples whose box touches a tile are its own samples and
    those of its lower neighbours t - e whose class contains e."""
    import itertools
    nd = len(grid)
    rng = np.random.default_rng(len(grid) * 100 + grid[0])
    traj = rng.uniform(-0.5, 0.5, size=(600, nd)).astype(np.float32)
    traj[:4] = 0.5                                     # on the edge (wraps to index 0)
    g = binning.grid_coords(traj, grid).astype(np.float64)
    j0 = binning.kernel_box_start(g)
    key, nt = binning.sort_keys(j0, grid, tile)
    tid, cls = key // 8, key % 8
    # brute force: owning tile index of every grid index along each axis
    owner = []
    for ax in range(nd):
        G, T, n = grid[ax], tile[ax], nt[ax]
        starts = [k * T for k in range(n)]
        own = np.array([max(k for k in range(n) if starts[k] <= j) for j in range(G)])
        assert own[-1] == n - 1 and min(np.bincount(own)) >= binning.KB_WIDTH
        owner.append(own)
    tix = np.stack([np.unravel_index(t, tuple(nt)) for t in tid])        # per-axis tile of each sample
    for ax in range(nd):
        box = np.mod(j0[:, ax:ax + 1] + np.arange(binning.KB_WIDTH)[None, :], grid[ax])
        bt = owner[ax][box]
        nxt = (tix[:, ax:ax + 1] + 1) % nt[ax]
        assert np.all((bt == tix[:, ax:ax + 1]) | (bt == nxt))
        reach = np.any(bt != tix[:, ax:ax + 1], axis=1)
        assert np.array_equal(reach, ((cls >> (nd - 1 - ax)) & 1).astype(bool))
    # owners: samples touching tile t == own + lower neighbours' reaching classes
    touch = {}
    for i in range(j0.shape[0]):
        boxes = [np.mod(j0[i, ax] + np.arange(binning.KB_WIDTH), grid[ax]) for ax in range(nd)]
        for pt in itertools.product(*boxes):
            t = np.ravel_multi_index(tuple(owner[ax][pt[ax]] for ax in range(nd)), tuple(nt))
            touch.setdefault(int(t), set()).add(i)
    for t in range(int(np.prod(nt))):
        tt = np.unravel_index(t, tuple(nt))
        want = set()
        for e in range(1 << nd):
            bits = [(e >> (nd - 1 - ax)) & 1 for ax in range(nd)]
            if any(b and nt[ax] == 1 for ax, b in enumerate(bits)):
                continue
            src = np.ravel_multi_index(tuple((tt[ax] - bits[ax]) % nt[ax] for ax in range(nd)), tuple(nt))
            want |= set(np.nonzero((tid == src) & ((cls & e) == e))[0].tolist())
        assert touch.get(t, set()) == want, t


def test_sample_order_is_stable_by_tile_then_class():
    traj = synthdata.cones_trajectory(40, 64)
    grid, tile = (20, 20, 20), (8, 8, 8)
    j0 = binning.kernel_box_start(binning.grid_coords(traj, grid).astype(np.float64))
    key, nt = binning.sort_keys(j0, grid, tile)
    perm, offs, nt2 = binning.sample_order(j0, grid, tile)
    assert tuple(nt) == tuple(nt2)
    p_lit, _ = binning.tile_sort(key, int(np.prod(nt)) * 8)          # literal counting sort on the key
    assert np.array_equal(perm, p_lit)
    assert np.all(np.diff(key[perm]) >= 0)
    for t in range(int(np.prod(nt))):
        seg = perm[offs[t]:offs[t + 1]]
        assert np.all(key[seg] // 8 == t)
