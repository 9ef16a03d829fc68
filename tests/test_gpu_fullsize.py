"""Parity at the large 3D cones workload's full size (160x256x256 image, 200x320x320 grid, 40
coils, 20000 x 512 samples), in the launch configuration the benchmark times: forward samples
checked one by one against the FP64 oracle (the oracle grids only the sampled points), and
properties that hold at any size for the adjoint and the sketched normal operator (adjointness,
Hermitian symmetry, lambda-positivity)."""
import numpy as np
import pytest
import torch

import synthdata
from oracle import nufft

pytestmark = pytest.mark.gpu

IMG, GRID, C, NI, NR = (160, 256, 256), (200, 320, 320), 40, 20000, 512


@pytest.fixture(scope="module")
def large():
    import paper_2305_06482_gb300 as cs
    from tests._gpu import ensure_built
    ensure_built()
    dev = torch.device("cuda")
    traj = synthdata.cones_trajectory(NI, NR)
    dcf = synthdata.cones_dcf(traj, IMG, NI, NR)
    plan = cs.Plan(cs.NONCARTESIAN, IMG, C, traj=torch.from_numpy(traj).to(dev), dcf=torch.from_numpy(dcf).to(dev),
                   grid=GRID)
    maps = synthdata.coil_maps_torch(IMG, C, device=dev)
    x = synthdata.phantom_torch(IMG, seed=1, device=dev)
    return plan, traj, dcf, maps, x


def _rand(shape, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return torch.randn(shape, dtype=torch.complex64, device="cuda", generator=g)


def _dot(a, b):
    return complex(torch.vdot(a.reshape(-1).to(torch.complex128), b.reshape(-1).to(torch.complex128)))


def test_large_forward_samples_match_oracle(large):
    import paper_2305_06482_gb300 as cs
    plan, traj, dcf, maps, x = large
    y = cs.sense_fwd(plan, x, maps)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(traj.shape[0], 16, replace=False))
    op = nufft.Plan(traj[idx], IMG, GRID)          # the oracle grids only the sampled points
    xn = x.cpu().numpy().astype(np.complex128)
    scale = float(y.abs().max())
    for c in (0, 27):
        ref = nufft.sense_fwd(op, xn, maps[c:c + 1].cpu().numpy().astype(np.complex128), dcf[idx])[0]
        got = y[c, torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
        assert np.abs(got - ref).max() < 2e-5 * scale, c


def test_large_adjoint_and_normal_operator_properties(large):
    import paper_2305_06482_gb300 as cs
    plan, traj, dcf, maps, x = large
    N = traj.shape[0]
    u = _rand(IMG, 1)
    r = _rand((C, N), 2)
    Au = cs.sense_fwd(plan, u, maps)
    AHr = cs.sense_adj(plan, r, maps)
    lhs, rhs = _dot(Au, r), _dot(u, AHr)
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    # sketched normal operator (m = 10 = 5 + 5): Hermitian and >= lambda
    lam = 1e-3
    mv, ms = maps[:5].contiguous(), (0.4 * maps[5:10] - 0.3 * maps[10:15]).contiguous()
    v = _rand(IMG, 3)
    Nu = cs.sketched_normal_apply(plan, u, mv, ms, lam)
    Nv = cs.sketched_normal_apply(plan, v, mv, ms, lam)
    a, b = _dot(u, Nv), _dot(Nu, v)
    assert abs(a - b) <= 1e-4 * abs(a)
    q = _dot(v, Nv)
    assert abs(q.imag) <= 1e-4 * abs(q.real) and q.real >= lam * _dot(v, v).real * (1 - 1e-4)


def test_large_adjoint_matches_oracle_voxel_by_voxel(large):
    """The full-size adjoint with all 40 coils in the benchmark's launch configuration (three coil
    chunks of 14 / 13 / 13 coils), k-space non-zero in two coils only (one in the first chunk, one in
    the last): the oracle spreads just those two coils over the full 200x320x320 grid.  The whole
    image matches to NRMSE 1e-5 and 500 sampled voxels one by one to 2e-5 of the image maximum, so
    an error localised anywhere in the spreading shows up."""
    import paper_2305_06482_gb300 as cs
    from oracle import solvers
    plan, traj, dcf, maps, x = large
    N = traj.shape[0]
    coils = (3, 31)
    y = torch.zeros((C, N), dtype=torch.complex64, device="cuda")
    for k, c in enumerate(coils):
        y[c] = _rand((N,), 10 + k)
    got = cs.sense_adj(plan, y, maps).cpu().numpy().astype(np.complex128)
    op = nufft.Plan(traj, IMG, GRID)
    yn = y[list(coils)].cpu().numpy().astype(np.complex128)
    mn = maps[list(coils)].cpu().numpy().astype(np.complex128)
    ref = nufft.sense_adj(op, yn, mn, dcf)
    assert solvers.nrmse(got, ref) < 1e-5
    rng = np.random.default_rng(5)
    vox = rng.choice(got.size, 500, replace=False)
    scale = np.abs(ref).max()
    assert np.abs(got.ravel()[vox] - ref.ravel()[vox]).max() < 2e-5 * scale
