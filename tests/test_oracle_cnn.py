"""Pins for the FP64 warm-start network reference: the convolution against a direct loop over
voxels and taps, and the backward pass against central finite differences."""
import numpy as np

from oracle import cnn


def test_conv3d_matches_direct_loops():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 4, 5, 2))
    w = rng.standard_normal((3, 27, 2))
    b = rng.standard_normal(3)
    out = cnn.conv3d(x, w, b)
    ref = np.zeros((3, 4, 5, 3))
    for z in range(3):
        for y in range(4):
            for xx in range(5):
                for co in range(3):
                    s = b[co]
                    for t, (dz, dy, dx) in enumerate(cnn.taps()):
                        zz, yy, xq = z + dz, y + dy, xx + dx
                        if 0 <= zz < 3 and 0 <= yy < 4 and 0 <= xq < 5:
                            s += np.dot(x[zz, yy, xq], w[co, t])
                    ref[z, y, xx, co] = s
    assert np.abs(out - ref).max() < 1e-12


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    shape = (4, 3, 5)
    params = [rng.standard_normal((4, 27, 4)) * 0.3, rng.standard_normal(4) * 0.1,
              rng.standard_normal((4, 27, 4)) * 0.3, rng.standard_normal(4) * 0.1,
              rng.standard_normal((4, 27, 4)) * 0.3, rng.standard_normal(4) * 0.1,
              rng.standard_normal((2, 4)), rng.standard_normal(2)]
    f = rng.standard_normal(shape + (4,))
    tgt = rng.standard_normal(shape + (2,))

    def loss(ps):
        out, _ = cnn.forward(ps, f)
        return cnn.mse(out, tgt)[0]

    out, acts = cnn.forward(params, f)
    _, g = cnn.mse(out, tgt)
    grads = cnn.backward(params, acts, g)
    h = 1e-6
    for pi in range(8):
        flat = params[pi].ravel()
        for j in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            pp = [q.copy() for q in params]
            pm = [q.copy() for q in params]
            pp[pi].ravel()[j] += h
            pm[pi].ravel()[j] -= h
            fd = (loss(pp) - loss(pm)) / (2 * h)
            assert abs(fd - grads[pi].ravel()[j]) <= 1e-6 * max(1.0, abs(fd)), (pi, j)


def test_maxpool_and_transposed_convolution_match_loops():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 2, 6, 3))
    out, idx = cnn.maxpool2(x)
    for z in range(2):
        for y in range(1):
            for xx in range(3):
                for ch in range(3):
                    block = [x[2 * z + dz, 2 * y + dy, 2 * xx + dx, ch] for dz, dy, dx in cnn.sub8()]
                    assert out[z, y, xx, ch] == max(block) and idx[z, y, xx, ch] == int(np.argmax(block))
    w = rng.standard_normal((2, 8, 3))
    b = rng.standard_normal(2)
    u = cnn.upconv2(out, w, b)
    for z in range(4):
        for y in range(2):
            for xx in range(6):
                a = 4 * (z % 2) + 2 * (y % 2) + (xx % 2)
                assert np.allclose(u[z, y, xx], b + w[:, a, :] @ out[z // 2, y // 2, xx // 2])


def test_unet_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    shapes = cnn.unet_shapes(2, 3, 4)
    params = [rng.standard_normal(s) * (0.4 if len(s) > 1 else 0.1) for s in shapes]
    f = rng.standard_normal((4, 4, 8, 4))
    tgt = rng.standard_normal((4, 4, 8, 2))
    out, cache = cnn.unet_forward(params, f)
    idx = (cache["i1"], cache["i2"])

    def loss(ps):
        o, _ = cnn.unet_forward(ps, f, pool_idx=idx)     # the pools' decisions held fixed
        return cnn.mse(o, tgt)[0]

    _, g = cnn.mse(out, tgt)
    grads = cnn.unet_backward(params, cache, g)
    h = 1e-6
    for pi in range(26):
        flat = params[pi].ravel()
        for j in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            pp = [q.copy() for q in params]
            pm = [q.copy() for q in params]
            pp[pi].ravel()[j] += h
            pm[pi].ravel()[j] -= h
            fd = (loss(pp) - loss(pm)) / (2 * h)
            assert abs(fd - grads[pi].ravel()[j]) <= 1e-5 * max(1.0, abs(fd)), (pi, j)


def test_unet_parameter_count():
    n = sum(int(np.prod(s)) for s in cnn.unet_shapes())
    assert 330_000 < n < 350_000        # the configured network's ~0.34 M weights


def test_bf16_weight_gradient_is_the_fp64_gradient_of_the_rounded_operands():
    """conv3d_bwd with bf16=True: the weight gradient is the exact gradient taken at the BF16-
    rounded input and output gradient (the tensor-core GEMM's operands), the data gradient uses the
    rounded weights and output gradient, and the bias gradient the unrounded output gradient."""
    from oracle.philox import round_to_bf16
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, 4, 5, 6)).astype(np.float32)
    w = rng.standard_normal((7, 27, 6)).astype(np.float32)
    g = rng.standard_normal((3, 4, 5, 7)).astype(np.float32)
    r = lambda a: round_to_bf16(a).astype(np.float32)
    gx, gw, gb = cnn.conv3d_bwd(x, w, g, bf16=True)
    gx0, gw0, _ = cnn.conv3d_bwd(r(x), r(w), r(g), bf16=False)
    _, _, gb0 = cnn.conv3d_bwd(x, w, g, bf16=False)
    assert np.array_equal(gw, gw0) and np.array_equal(gx, gx0) and np.array_equal(gb, gb0)
    assert np.abs(gw - cnn.conv3d_bwd(x, w, g)[1]).max() > 0       # the rounding is visible
