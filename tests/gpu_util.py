"""Shared helpers of the GPU tests (imported only by tests marked gpu)."""
import numpy as np
import torch


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def int_matrix(n, d, seed, lo=-8, hi=8):
    """Small integers: every sum in an SRHT/SJLT sketch is exact in FP64, so a GPU result
    equal bit for bit to the oracle's proves the same signs, rows and hash positions."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=(n, d)).astype(np.float64)
