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
