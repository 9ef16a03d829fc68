"""The DFT library calls of the oracle (a library primitive used as one step, as the survey's
CPU baseline prescribes: scipy.fft where present, else numpy.fft).

``WORKERS`` is the number of threads scipy.fft may use (1 by default, so tests stay
single-threaded and deterministic; the CPU baseline of the benchmark raises it to the host's
core count).  The result is the same DFT either way, up to floating-point rounding order.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

try:
    import scipy.fft as _sfft
except ImportError:   # pragma: no cover - scipy is present on both machines
    _sfft = None

WORKERS = 1


def set_workers(n):
    """Threads for the oracle's FFTs (>= 1); returns the previous value."""
    global WORKERS
    old, WORKERS = WORKERS, max(1, int(n))
    return old


def fftn(a, axes, norm=None):
    if _sfft is not None:
        return _sfft.fftn(a, axes=axes, norm=norm, workers=WORKERS)
    return np.fft.fftn(a, axes=axes, norm=norm)


def ifftn(a, axes, norm=None):
    if _sfft is not None:
        return _sfft.ifftn(a, axes=axes, norm=norm, workers=WORKERS)
    return np.fft.ifftn(a, axes=axes, norm=norm)
