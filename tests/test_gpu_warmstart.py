"""Warm-start U-Net on the GPU: tensor-core convolutions (forward and data gradient), max-pools,
transposed convolutions and skip concatenation, forward/backward against the FP64 reference at
the same BF16 operand precision; Adam training lowers the loss; in Algorithm 1 a prediction is
used only when it lowers the sub-problem objective, and the trained network's effect on
convergence is measured."""
import numpy as np
import pytest
import torch

import synthdata
from oracle import cnn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from tests._gpu import ensure_built
    ensure_built()


def _net_params(net):
    return [p.detach().cpu().numpy().astype(np.float64) for p in net.params]


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    dt = np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64
    a, b = a.astype(dt), b.astype(dt)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("cin,cout,flip,dims", [
    (16, 16, 0, (5, 11, 30)),     # brick kernel: ragged tiles in every axis
    (4, 16, 0, (6, 8, 14)),       # 4 input channels (zero-padded to 16)
    (32, 64, 1, (3, 9, 17)),      # data gradient (flipped taps, transposed weights)
    (64, 32, 0, (2, 3, 29)),      # 4 channel pairs, fewer planes than a tile
    (20, 24, 0, (4, 7, 15)),      # channels not a multiple of 16
    (3, 5, 0, (4, 7, 9)),         # channels not a multiple of 4: the im2col kernel
])
def test_conv3d_matches_reference(cin, cout, flip, dims):
    """One 3x3x3 convolution through cs_nn_pack_weights / cs_nn_conv3d against the FP64
    reference on the same BF16 operands, written into a channel slice of a wider output."""
    import ctypes
    import paper_2305_06482_gb300 as cs
    from tests._unet_layers import _kpad, _npad
    rng = np.random.default_rng(cin * 100 + cout)
    x = rng.standard_normal(dims + (cin,)).astype(np.float32)
    # layer weights [co][27][ci]; the data gradient convolves with the layer whose output has cin channels
    w = (rng.standard_normal((cin, 27, cout) if flip else (cout, 27, cin)) * 0.2).astype(np.float32)
    b = None if flip else rng.standard_normal(cout).astype(np.float32)
    if flip:
        wr = cnn._r(w, True)
        gp = np.pad(cnn._r(x, True), ((1, 1), (1, 1), (1, 1), (0, 0)))
        ref = np.zeros(dims + (cout,))
        for t, (dz, dy, dx) in enumerate(cnn.taps()):
            ref += gp[1 - dz:1 - dz + dims[0], 1 - dy:1 - dy + dims[1], 1 - dx:1 - dx + dims[2]] @ wr[:, t, :]
    else:
        ref = np.maximum(cnn.conv3d(x, w, b, bf16=True), 0.0)
    npad = _npad(cout)
    kpad = _kpad(27 * cin)
    wt = torch.from_numpy(w).cuda()
    packed = torch.empty((npad, kpad), dtype=torch.int16, device="cuda")
    rows, cols = (cout, cin) if not flip else (cin, cout)    # cs_nn_pack_weights takes the layer's (cout, cin)
    cs._check(cs.lib().cs_nn_pack_weights(cs._ptr(wt), rows, cols, int(flip), cs._ptr(packed), npad, kpad, None))
    ldo, coff = cout + 8, 4
    out = torch.full((int(np.prod(dims)), ldo), 7.0, device="cuda")
    xt = torch.from_numpy(x.reshape(-1, cin)).cuda()
    bt = None if b is None else torch.from_numpy(b).cuda()
    cs._check(cs.lib().cs_nn_conv3d(cs._ptr(xt), *dims, cin, cs._ptr(packed), npad, kpad, cout, cs._ptr(bt),
                                    0 if flip else 1, int(flip), cs._ptr(out), ldo, coff, None))
    cs._check(cs.lib().cs_nn_status(None))
    o = out.cpu().numpy()
    assert np.all(o[:, :coff] == 7.0) and np.all(o[:, coff + cout:] == 7.0)
    got = o[:, coff:coff + cout].reshape(ref.shape)
    assert _rel(got, ref) < 1e-5
    if not flip:
        # weight gradient of the same layer for a random output gradient (register-tiled kernel
        # when both channel counts are multiples of 4, else the per-pair kernel)
        go = rng.standard_normal(dims + (cout,)).astype(np.float32)
        _, gw_ref, gb_ref = cnn.conv3d_bwd(x, w, go, bf16=True)
        gw = torch.zeros((cout, 27, cin), device="cuda")
        gb = torch.zeros(cout, device="cuda")
        got = torch.from_numpy(go.reshape(-1, cout)).cuda()
        cs._check(cs.lib().cs_nn_conv3d_wgrad(cs._ptr(xt), cs._ptr(got), *dims, cin, cout, cs._ptr(gw), cs._ptr(gb),
                                              None))
        assert _rel(gw.cpu().numpy(), gw_ref) < 1e-5
        assert _rel(gb.cpu().numpy(), gb_ref) < 1e-5


@pytest.mark.parametrize("cin,cout,dims", [
    (16, 16, (5, 11, 30)),      # 4 row tiles, one tile group
    (4, 16, (6, 8, 14)),        # one partial row tile (108 rows)
    (32, 64, (7, 9, 17)),       # 7 row tiles: two tile groups
    (64, 32, (16, 20, 24)),     # 14 row tiles, 120 voxel rounds over many partial-sum slots
    (128, 100, (3, 5, 9)),      # 27 row tiles, 128-column accumulators, ragged channels
    (3, 5, (4, 7, 9)),          # channels not a multiple of 4
])
def test_conv3d_weight_gradient_on_tensor_cores(cin, cout, dims):
    """cs_nn_conv3d_wgrad (BF16 implicit GEMM on tcgen05, voxels as the reduction) against the FP64
    weight gradient of the same BF16-rounded operands, accumulated into a non-zero gw; the bias
    gradient in FP32; two runs bit-identical (partial sums added in slot order)."""
    import paper_2305_06482_gb300 as cs
    rng = np.random.default_rng(cin * 1000 + cout)
    x = rng.standard_normal(dims + (cin,)).astype(np.float32)
    go = rng.standard_normal(dims + (cout,)).astype(np.float32)
    w = np.zeros((cout, 27, cin), np.float32)
    _, gw_ref, gb_ref = cnn.conv3d_bwd(x, w, go, bf16=True)
    gw0 = rng.standard_normal((cout, 27, cin)).astype(np.float32)
    gb0 = rng.standard_normal(cout).astype(np.float32)
    xt = torch.from_numpy(x.reshape(-1, cin)).cuda()
    gt = torch.from_numpy(go.reshape(-1, cout)).cuda()
    outs = []
    for _ in range(2):
        gw = torch.from_numpy(gw0.copy()).cuda()
        gb = torch.from_numpy(gb0.copy()).cuda()
        cs._check(cs.lib().cs_nn_conv3d_wgrad(cs._ptr(xt), cs._ptr(gt), *dims, cin, cout, cs._ptr(gw), cs._ptr(gb),
                                              None))
        cs._check(cs.lib().cs_nn_status(None))
        outs.append((gw.cpu().numpy(), gb.cpu().numpy()))
    assert _rel(outs[0][0] - gw0, gw_ref) < 1e-5
    assert _rel(outs[0][1] - gb0, gb_ref) < 1e-5
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_upconv_and_slice_general_paths():
    """The transposed convolution and the channel slice on channel counts and offsets that are not
    multiples of 4 (their scalar paths), against the reference and numpy."""
    import paper_2305_06482_gb300 as cs
    rng = np.random.default_rng(5)
    cd = (3, 5, 7)
    cin, cout, ldo, coff = 3, 5, 9, 1
    x = rng.standard_normal(cd + (cin,)).astype(np.float32)
    w = rng.standard_normal((cout, 8, cin)).astype(np.float32)
    b = rng.standard_normal(cout).astype(np.float32)
    Vf = 8 * int(np.prod(cd))
    out = torch.full((Vf, ldo), 3.0, device="cuda")
    xt, wt, bt = (torch.from_numpy(a).cuda() for a in (x.reshape(-1, cin), w, b))
    cs._check(cs.lib().cs_nn_upconv2(cs._ptr(xt), *cd, cin, cs._ptr(wt), cs._ptr(bt), cout, cs._ptr(out), ldo, coff,
                                     None))
    o = out.cpu().numpy()
    ref = cnn.upconv2(x, w, b).reshape(Vf, cout)
    assert _rel(o[:, coff:coff + cout], ref) < 1e-6
    assert np.all(o[:, :coff] == 3.0) and np.all(o[:, coff + cout:] == 3.0)
    src = torch.from_numpy(rng.standard_normal((Vf, 6)).astype(np.float32)).cuda()
    before = out.clone()
    cs._check(cs.lib().cs_nn_slice(cs._ptr(src), 6, 2, 3, cs._ptr(out), ldo, 5, Vf, 1, None))
    exp = before.cpu().numpy()
    exp[:, 5:8] += src.cpu().numpy()[:, 2:5]
    assert np.array_equal(out.cpu().numpy(), exp)


def test_network_forward_backward_match_reference():
    """Every layer against the FP64 reference on the GPU's own inputs to that layer (tight: only
    the FP32 accumulation differs), the wiring between layers exactly, and the whole network end
    to end.  End to end the BF16 rounding of an FP32 activation and of its FP64 counterpart
    differs whenever the two straddle a rounding boundary; each such flip moves that operand by a
    BF16 ulp (2^-8 relative) and the differences grow layer by layer (ten 3x3x3 layers deep), so
    that comparison only bounds the result to a few BF16 ulps."""
    import paper_2305_06482_gb300.warmstart as ws
    from tests._unet_layers import LayeredUNet
    c1, c2, c3 = ws.WIDTHS
    d1 = (8, 12, 20)
    d2 = tuple(v // 2 for v in d1)
    d3 = tuple(v // 2 for v in d2)
    net = LayeredUNet(seed=3)
    assert [tuple(p.shape) for p in net.params] == cnn.unet_shapes(*ws.WIDTHS)
    # non-trivial biases and output layer, from a generator of the test's own (the global one's
    # state depends on which tests ran before)
    gen = torch.Generator(device=net.params[1].device).manual_seed(11)
    for i in range(1, 26, 2):
        net.params[i].normal_(0, 0.05, generator=gen)
    net.params[24].normal_(0, 0.3, generator=gen)
    rng = np.random.default_rng(0)
    f = rng.standard_normal(d1 + (4,)).astype(np.float32)
    tgt = rng.standard_normal(d1 + (2,)).astype(np.float32)
    ft = torch.from_numpy(f.reshape(-1, 4)).cuda()
    out = net.forward(ft, d1, keep=True)
    P = _net_params(net)
    level = {n: d1 for n in ("f", "e1a", "e1", "cat1", "d1a", "d1")}
    level.update({n: d2 for n in ("p1", "e2a", "e2", "cat2", "d2a", "d2", "i1")})
    level.update({n: d3 for n in ("p2", "b1", "b2", "i2")})
    A = {n: t.cpu().numpy().reshape(level[n] + (-1,)) for n, t in net._acts.items()}
    relu = lambda v: np.maximum(v, 0.0)

    # ---- forward, layer by layer ----
    pool_idx = []
    for fine, pooled, idx in (("e1", "p1", "i1"), ("e2", "p2", "i2")):
        kids = np.stack([A[fine][dz::2, dy::2, dx::2] for dz, dy, dx in cnn.sub8()])
        ii = A[idx].astype(np.int64)
        assert np.array_equal(ii, np.argmax(kids, axis=0))      # first child reaching the maximum
        assert np.array_equal(A[pooled], kids.max(axis=0))
        pool_idx.append(ii)
    conv = [(0, "f", "e1a"), (2, "e1a", "e1"), (4, "p1", "e2a"), (6, "e2a", "e2"), (8, "p2", "b1"), (10, "b1", "b2"),
            (14, "cat2", "d2a"), (16, "d2a", "d2"), (20, "cat1", "d1a"), (22, "d1a", "d1")]
    for pi, src, dst in conv:
        assert _rel(A[dst], relu(cnn.conv3d(A[src], P[pi], P[pi + 1], bf16=True))) < 2e-5, pi
    for pi, src, cat, skip, c in ((12, "b2", "cat2", "e2", c2), (18, "d2", "cat1", "e1", c1)):
        assert _rel(A[cat][..., :c], cnn.upconv2(A[src], P[pi], P[pi + 1])) < 1e-5, pi
        assert np.array_equal(A[cat][..., c:], A[skip])
    o = out.cpu().numpy().reshape(d1 + (2,))
    assert _rel(o, A["d1"].astype(np.float64) @ P[24].T + P[25]) < 1e-5

    # ---- backward, layer by layer ----
    loss, g = net.loss_and_grad(out, torch.from_numpy(tgt.reshape(-1, 2)).cuda())
    net.backward(g, d1, keep=True)
    gn = g.cpu().numpy().reshape(d1 + (2,)).astype(np.float64)
    Gg = [t.cpu().numpy() for t in net.grads]
    lvl = {24: d1, 22: d1, 20: d1, 18: d2, 16: d2, 14: d2, 12: d3, 10: d3, 8: d3, 6: d2, 4: d2, 2: d1, 0: d1,
           "e2": d2, "e1": d1}
    inlvl = {20: d1, 14: d2, 12: d3, 8: d3, 4: d2}
    gx = {k: t.cpu().numpy().reshape(inlvl.get(k, lvl[k]) + (-1,)) for k, t in net._gx.items()}
    gup = {k: t.cpu().numpy().reshape(lvl[k] + (-1,)) for k, t in net._gup.items()}
    gz = {k: t.cpu().numpy().reshape(lvl[k] + (-1,)) for k, t in net._gz.items()}
    assert _rel(Gg[24], np.einsum("zyxo,zyxc->oc", gn, A["d1"])) < 1e-5
    assert _rel(Gg[25], gn.sum(axis=(0, 1, 2))) < 1e-5
    assert _rel(gx[24], gn @ P[24]) < 1e-5
    # each layer's upstream gradient is exactly what the layer above handed down
    for pi, up in ((22, 24), (20, 22), (16, 18), (14, 16), (10, 12), (8, 10), (6, "e2"), (4, 6), (2, "e1"), (0, 2)):
        assert np.array_equal(gup[pi], gx[up]), pi
    for pi, src, dst in conv:
        assert np.array_equal(gz[pi], gup[pi] * (A[dst] > 0)), pi
        gx_ref, gw_ref, gb_ref = cnn.conv3d_bwd(A[src], P[pi], gz[pi], bf16=True)
        assert _rel(Gg[pi].reshape(gw_ref.shape), gw_ref) < 1e-5, pi
        assert _rel(Gg[pi + 1], gb_ref) < 1e-5, pi
        if pi > 0:
            assert _rel(gx[pi], gx_ref) < 2e-5, pi
    for pi, src, gcat, c in ((12, "b2", 14, c2), (18, "d2", 20, c1)):
        gx_ref, gw_ref, gb_ref = cnn.upconv2_bwd(A[src], P[pi], gx[gcat][..., :c])
        assert _rel(gx[pi], gx_ref) < 1e-5, pi
        assert _rel(Gg[pi].reshape(gw_ref.shape), gw_ref) < 1e-5, pi
        assert _rel(Gg[pi + 1], gb_ref) < 1e-5, pi
    for e, low, idx, gcat, c in (("e2", 8, 1, 14, c2), ("e1", 4, 0, 20, c1)):
        ref = cnn.maxpool2_bwd(gx[low], pool_idx[idx], A[e].shape) + gx[gcat][..., c:]
        assert _rel(gx[e], ref) < 1e-6, e

    # ---- end to end (pool decisions taken from the GPU) ----
    ref, cache = cnn.unet_forward(P, f, bf16=True, pool_idx=pool_idx)
    assert _rel(o, ref) < 2e-2
    _, g_ref = cnn.mse(ref, tgt)
    grads_ref = cnn.unet_backward(P, cache, g_ref, bf16=True)
    for gi, (gg, gr) in enumerate(zip(Gg, grads_ref)):
        assert _rel(gg.reshape(gr.shape), gr) < 5e-2, gi
    with pytest.raises(ValueError):
        net.forward(ft[: 6 * 12 * 20].contiguous(), (6, 12, 20))


def test_library_network_matches_layered_sequence(tmp_path):
    """The library's network object (ws_net_*) against the same kernels sequenced layer by layer
    from Python: inference, one training step (loss, gradients, Adam update), save / load, and
    the size checks."""
    import paper_2305_06482_gb300 as cs
    import paper_2305_06482_gb300.warmstart as ws
    from tests._unet_layers import LayeredUNet
    dims = (8, 12, 20)
    ref = LayeredUNet(seed=3)
    gen = torch.Generator(device="cuda").manual_seed(11)
    for i in range(1, 26, 2):
        ref.params[i].normal_(0, 0.05, generator=gen)
    net = ws.UNet(seed=5)
    for i, p in enumerate(ref.params):
        net.set_param(i, p.reshape(-1))
    rng = np.random.default_rng(4)
    cplx = lambda: torch.from_numpy((rng.standard_normal(dims) + 1j * rng.standard_normal(dims)).astype(np.complex64)).cuda()
    xt, d, xs = cplx(), cplx(), cplx()
    eta = 0.7
    xhat = net.infer(xt, d, eta)
    f, ss = ws.features(xt, d, eta)
    xh_ref = ws.apply(xt, ref.forward(f, dims), ss)
    # same kernels in the same order; only the atomically summed normaliser s can differ in its
    # last bits
    assert _rel(xhat.cpu().numpy(), xh_ref.cpu().numpy()) < 1e-6
    before = [net.param(i).cpu().numpy() for i in range(26)]
    loss = float(net.train_step(xt, d, xs, eta, 1e-3).item())
    out = ref.forward(f, dims, keep=True)
    lref, g = ref.loss_and_grad(out, ws.target(xt, xs, ss))
    ref.backward(g, dims)
    ref.adam(lr=1e-3)
    assert abs(loss - float(lref.item())) <= 1e-5 * abs(float(lref.item()))
    for i in range(26):
        gr = ref.grads[i].reshape(-1).cpu().numpy()
        assert _rel(net.param(i, which=1).cpu().numpy(), gr) < 1e-4, i
        step_n = net.param(i).cpu().numpy() - before[i]
        step_r = ref.params[i].reshape(-1).cpu().numpy() - before[i]
        # Adam's first step is about lr * sign(g): equal wherever the gradient is clearly nonzero;
        # a component whose gradient is ~0 may take the other sign (the sums are atomic)
        assert np.abs(step_n - step_r).max() <= 2.1e-3, i
        gmax = np.abs(gr).max()
        if gmax > 0:
            big = np.abs(gr) > 1e-3 * gmax
            assert np.abs(step_n - step_r)[big].max() <= 1e-6, i
    path = tmp_path / "unet.bin"
    net.save(path)
    other = ws.UNet(seed=9)
    other.load(path)
    for i in range(26):
        for which in (0, 2, 3):
            assert torch.equal(other.param(i, which), net.param(i, which)), (i, which)
    assert torch.equal(other.infer(xt, d, eta), net.infer(xt, d, eta)) or \
        _rel(other.infer(xt, d, eta).cpu().numpy(), net.infer(xt, d, eta).cpu().numpy()) < 1e-6
    with pytest.raises(cs.CoilSketchError):
        net.infer(xt[:6].contiguous(), d[:6].contiguous(), eta)       # 6 is not a multiple of 4
    with pytest.raises(cs.CoilSketchError):
        ws.UNet(seed=0, widths=(8, 16, 32)).load(path)                 # widths differ
    with pytest.raises(cs.CoilSketchError):
        ws.UNet(seed=0, widths=(16, 64, 64))                           # concatenation too wide
    cs._check(cs.lib().cs_nn_status(None))


def test_crop_and_crop_training():
    """cs_crop3d against slicing (and its range check); training steps on random crops run and
    stay finite."""
    import paper_2305_06482_gb300 as cs
    import paper_2305_06482_gb300.warmstart as ws
    rng = np.random.default_rng(2)
    dims = (12, 20, 28)
    vol = lambda: torch.from_numpy((rng.standard_normal(dims) + 1j * rng.standard_normal(dims)).astype(np.complex64)).cuda()
    x = vol()
    c = ws.crop3d(x, (3, 5, 7), (8, 12, 16))
    assert torch.equal(c, x[3:11, 5:17, 7:23])
    with pytest.raises(cs.CoilSketchError):
        ws.crop3d(x, (5, 0, 0), (8, 12, 16))                     # 5 + 8 > 12
    pairs = [(vol(), vol(), vol(), 0.5) for _ in range(2)]
    net = ws.UNet(seed=1)
    hist = ws.train(net, pairs, steps=6, lr=1e-3, crop=(8, 12, 16))
    assert len(hist) == 6 and all(np.isfinite(hist))


def _problem(seed, img=(32, 48, 48), grid=(40, 60, 60), C=8, n_int=1500, n_read=128):
    import paper_2305_06482_gb300 as cs
    dev = torch.device("cuda")
    traj = synthdata.cones_trajectory(n_int, n_read)
    dcf = synthdata.cones_dcf(traj, img, n_int, n_read)
    plan = cs.Plan(cs.NONCARTESIAN, img, C, traj=torch.from_numpy(traj).to(dev), dcf=torch.from_numpy(dcf).to(dev),
                   grid=grid)
    maps = synthdata.coil_maps_torch(img, C, device=dev)
    x_true = synthdata.phantom_torch(img, seed=seed, device=dev)
    y = cs.sense_fwd(plan, x_true, maps)
    return plan, y, maps


def test_training_and_warm_start_in_algorithm_1():
    """Training on the method's own pairs lowers the loss, and on a held-out phantom the trained
    network's accepted predictions bring the first two outer iterates of Algorithm 1 strictly closer
    to x_inf than the method without it (recon_solve, decision on the device).  Everything runs
    bit-reproducibly (fixed-order coil covariance, deterministic spreading, fixed-order weight-
    gradient and loss sums), so the measured gain is the same on every run and in any test order."""
    import paper_2305_06482_gb300 as cs
    import paper_2305_06482_gb300.warmstart as ws
    img = (32, 48, 48)
    lam, V, S, T, K, levels = 2e-3, 2, 2, 6, 4, 2
    pairs = []
    for seed in (101, 102, 103, 104):
        plan, y, maps = _problem(seed)
        plan.set_deterministic(True)
        su = ws.setup(plan, y, maps, lam, V, S, T, seed, synthdata.phantom_torch(img, seed=seed + 50), levels)
        _, pr, _ = ws.run(su, T, K, record_pairs=1, tight_K=40)
        pairs += pr
    net = ws.UNet(seed=0)
    hist = ws.train(net, pairs, steps=300, lr=2e-3)
    first, last = np.mean(hist[:20]), np.mean(hist[-20:])
    assert last < first, (first, last)
    # held-out phantom: convergence with and without the warm start
    plan, y, maps = _problem(999)
    plan.set_deterministic(True)
    v0 = synthdata.phantom_torch(img, seed=1049)
    x_inf, _ = cs.recon_solve(plan, y, maps, lam, cs.REG_L1_WAVELET,
                              cs.SolveParams(K=400, sketch=False, do_pca=False, power_v0=v0), wavelet_levels=levels)
    curves, acc = {}, None
    for name, n in (("plain", None), ("warm", net)):
        _, st = cs.recon_solve(plan, y, maps, lam, cs.REG_L1_WAVELET,
                               cs.SolveParams(T=T, K=K, V=V, S=S, seed=999, power_v0=v0, warm=n, x_ref=x_inf, trace=True),
                               wavelet_levels=levels)
        curves[name] = np.sqrt(st["trace"][:, cs.TRACE_DIST2])
        if n is not None:
            acc = st["trace"][:, cs.TRACE_ACCEPT]
    e_plain, e_warm = curves["plain"], curves["warm"]
    print(f"\nwarm-start training loss {first:.3e} -> {last:.3e}; accepted {int((acc == 1).sum())}/{T}")
    print("NRMSE vs x_inf without warm start:", ["%.3e" % e for e in e_plain])
    print("NRMSE vs x_inf with warm start:   ", ["%.3e" % e for e in e_warm])
    assert acc[0] == 1
    assert e_warm[0] < e_plain[0] and e_warm[1] < e_plain[1]
    assert np.isfinite(e_warm).all()


def test_warm_start_decided_on_the_device_matches_the_host_loop():
    """recon_solve with the network as its warm start (prediction, two sub-problem objectives and
    the choice of FISTA's start all on the device) takes the same accept decisions and reaches the
    same iterates as the host-driven loop that reads the two objectives on the host; the captured
    outer iteration replays to the eager result."""
    import paper_2305_06482_gb300 as cs
    import paper_2305_06482_gb300.warmstart as ws
    img = (32, 48, 48)
    lam, V, S, T, K, levels = 2e-3, 2, 2, 5, 4, 2
    pairs = []
    for seed in (101, 102):
        plan, y, maps = _problem(seed)
        su = ws.setup(plan, y, maps, lam, V, S, T, seed, synthdata.phantom_torch(img, seed=seed + 50), levels)
        pairs += ws.run(su, T, K, record_pairs=1, tight_K=40)[1]
    net = ws.UNet(seed=0)
    ws.train(net, pairs, steps=150, lr=2e-3)
    plan, y, maps = _problem(999)
    plan.set_deterministic(True)          # bit-reproducible spreading: graph replay == eager exactly
    v0 = synthdata.phantom_torch(img, seed=1049)
    su = ws.setup(plan, y, maps, lam, V, S, T, 999, v0, levels)
    host = []
    _, _, acc = ws.run(su, T, K, net=net, callback=lambda t, x: host.append(x.clone()))
    runs = []
    for graph in (False, True):
        iters = torch.empty((T,) + img, dtype=torch.complex64, device="cuda")
        x, st = cs.recon_solve(plan, y, maps, lam, cs.REG_L1_WAVELET,
                               cs.SolveParams(T=T, K=K, V=V, S=S, seed=999, power_v0=v0, warm=net, use_graph=graph,
                                              iterates=iters, trace=True), wavelet_levels=levels)
        dec = st["trace"][:, cs.TRACE_ACCEPT]
        assert list(dec.astype(int)) == [int(a) for a in acc], (dec, acc)
        assert st["warm_accepted"] == sum(acc)
        # the two paths' FP32 steps differ at the 1e-7 level (the host loop passes the step as a
        # float, the spreading sums in a different order); an accepted prediction goes through the
        # network's BF16 convolutions, which amplify that, so the iterates are held to the
        # final-image tolerance
        for k in range(T):
            assert float((iters[k] - host[k]).norm() / host[k].norm()) < 1e-4
        runs.append(x)
    assert torch.equal(runs[0], runs[1])
    print(f"\\nwarm starts accepted {sum(acc)}/{T}")
    with pytest.raises(cs.CoilSketchError):          # the warm start serves sketched FISTA only
        cs.recon_solve(plan, y, maps, lam, cs.REG_L2, cs.SolveParams(T=2, K=2, V=V, S=S, warm=net))
