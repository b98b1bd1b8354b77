"""Helpers for the GPU parity tests (device transfer and tolerances)."""
import numpy as np
import torch

from paper_2601_13994_b300 import sla

DEV = "cuda"


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def csr(rp, c):
    return sla.CSRMatrix.from_numpy(rp, c, device=DEV)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (d if d > 0 else 1.0)
