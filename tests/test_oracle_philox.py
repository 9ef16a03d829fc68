"""Pins for the Philox4x32-10 generator (published known-answer vectors of Salmon et al. 2011,
Random123 distribution; fixture tests/golden/philox4x32_10_kat.txt) and the sketch entry
distributions (Sec. 3.2)."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox


def _kat():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((tuple(w[0:4]), tuple(w[4:6]), tuple(w[6:10])))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_philox_known_answers(ctr, key, want):
    assert philox.philox4x32_10(ctr, key) == want


def test_bf16_rounding_is_nearest_even():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(2000), [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8]]).astype(np.float32)
    r = philox.round_to_bf16(x)
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
    # nearest: no other bf16 value is closer
    up = (r.view(np.uint32) + 0x10000).view(np.float32)
    dn = (r.view(np.uint32) - 0x10000).view(np.float32)
    d = np.abs(x.astype(np.float64) - r)
    assert np.all(d <= np.abs(x.astype(np.float64) - up)) and np.all(d <= np.abs(x.astype(np.float64) - dn))
    assert r[-3] == np.float32(1.0) and r[-2] == np.float32(1.0 + 4 * 2 ** -8) and r[-1] == np.float32(-1.0)


def test_gaussian_sketch_statistics_and_determinism():
    S = 4
    draws = philox.sketch_draw(1234, 0, 40, 40, 5, S)       # 40 x 4 x 35 = 5600 entries
    v = draws.ravel().astype(np.float64)
    n = v.size
    assert abs(v.mean()) < 4 * np.sqrt(1 / S / n)
    assert abs(v.var() - 1 / S) < 4 * (1 / S) * np.sqrt(2 / n) + 1e-3
    assert stats.kstest(v * np.sqrt(S), "norm").pvalue > 1e-3
    again = philox.sketch_draw(1234, 10, 5, 40, 5, S)
    assert np.array_equal(again, draws[10:15])               # counter-based: (seed, t) addressable
    assert not np.array_equal(philox.sketch_draw(1235, 0, 1, 40, 5, S), draws[:1])


def test_rademacher_sketch():
    S = 2
    d = philox.sketch_draw(7, 0, 50, 20, 4, S, dist=philox.RADEMACHER)
    vals = set(np.unique(d).tolist())
    b = float(philox.round_to_bf16(np.float32(1 / np.sqrt(S))))
    assert vals == {b, -b}
    frac = np.mean(d > 0)
    assert abs(frac - 0.5) < 4 * np.sqrt(0.25 / d.size)
    lit = philox.sketch_draw(7, 0, 1, 20, 4, S, dist=philox.RADEMACHER, norm=philox.NORM_PAPER_LITERAL)
    assert set(np.unique(lit).tolist()) <= {1.0, -1.0}
