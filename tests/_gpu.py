"""Shared helpers of the GPU parity tests (inputs come from synthdata; expected values from the
oracle; the device results come through the C ABI)."""
import numpy as np
import torch

import paper_2305_06482_gb300 as cs

DEV = torch.device("cuda:0")


def t(a, dtype=None):
    a = np.ascontiguousarray(a)
    if dtype is not None:
        a = a.astype(dtype)
    elif np.iscomplexobj(a):
        a = a.astype(np.complex64)
    elif a.dtype == np.float64:
        a = a.astype(np.float32)
    return torch.from_numpy(a).to(DEV)


def h(x):
    torch.cuda.synchronize()
    return x.detach().cpu().numpy().astype(np.complex128 if x.is_complex() else np.float64)


def nrmse(a, ref):
    return float(np.linalg.norm((a - ref).ravel()) / np.linalg.norm(np.asarray(ref).ravel()))


def ensure_built():
    from paper_2305_06482_gb300 import build
    build.build()
    cs.lib()
