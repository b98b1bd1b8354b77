"""Helpers for the GPU parity tests (device transfer and tolerances)."""
import json
import os

import numpy as np
import pytest
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


def stored_oracle(name):
    """Stored expected values written by tests/golden/make_golden.py (which
    calls only the oracle); the test is skipped when the file is absent."""
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    if not os.path.exists(p):
        pytest.skip("no stored oracle values " + name)
    with open(p) as f:
        return json.load(f)


def sampled_errors(x, g):
    """(max_i |x_i - x*_i| / max |x*|, ||x - x*|| / ||x*||) over the stored
    sample of the oracle's solution."""
    idx = np.asarray(g["sample_idx"], dtype=np.int64)
    xs = np.asarray(g["x_star_sample"], dtype=np.float64)
    d = np.asarray(x)[idx] - xs
    return float(np.abs(d).max() / np.abs(xs).max()), float(np.linalg.norm(d) / np.linalg.norm(xs))


def elementwise_rel(a, b):
    """max_i |a_i - b_i| / max_i |b_i|: an error confined to a few entries
    cannot hide under a norm."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = np.abs(b).max() if b.size else 0.0
    return float(np.abs(a - b).max() / (m if m > 0 else 1.0)) if b.size else 0.0
