"""Helpers shared by the GPU tests: device copies and bit-level comparisons."""
import numpy as np
import torch


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def bits_equal(a, b) -> bool:
    """Bit-for-bit equality of float64 arrays (distinguishes -0.0 and +0.0)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return a.shape == b.shape and np.array_equal(a.view(np.int64), b.view(np.int64))


def csr_dev(rp, ci, val):
    return dev(rp.astype(np.int32)), dev(ci.astype(np.int32)), dev(val.astype(np.float64))
