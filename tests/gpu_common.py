"""Helpers shared by the GPU parity tests (imported only by tests)."""
import math

import numpy as np


def bits(a):
    return np.array(a, dtype=np.float64).view(np.uint64)


def same(a: float, b: float) -> bool:
    """Bitwise equality of binary64 values; NaNs compare by NaN-ness only
    (payloads differ between CPU and GPU)."""
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return bits(a)[()] == bits(b)[()]


def same_array(a, b) -> bool:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.shape != b.shape:
        return False
    na, nb = np.isnan(a), np.isnan(b)
    return bool((na == nb).all() and (bits(a)[~na] == bits(b)[~nb]).all())


def cuda_device():
    import torch
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")
