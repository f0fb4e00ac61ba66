"""Shared helpers of the GPU parity tests (compare the CUDA path with the oracle)."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import qmc_oracle as O
from paper_2305_11645_gb300 import api
from paper_2305_11645_gb300 import build as B

U32 = 2.0 ** -24          # unit roundoff of float32
U64 = 2.0 ** -53


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def norm_rel(got, want) -> float:
    got, want = np.asarray(got, dtype=np.float64), np.asarray(want, dtype=np.float64)
    scale = max(np.max(np.abs(want)), 1e-300)
    return float(np.max(np.abs(got - want)) / scale)


def fp32_product_bound(X, A):
    """Elementwise forward-error bound of the FP32 product: the points are rounded
    once to float (<= 3u for the inverse normal), and every output is an
    FMA chain of at most s + 8 terms (coarse block products, tree adds), so
    |P - P*| <= (s + 16) u sum_j |x_j a_j| (standard dot-product bound, u = 2^-24)."""
    s = X.shape[1]
    return (s + 16) * U32 * (np.abs(X) @ np.abs(np.asarray(A, dtype=np.float64)))


def oracle_rows(p, r, ks):
    return O.product(O.points(p, r, ks), p.A)


def integrand(p):
    return api.Integrand(p.f_kind, p.f_params)


GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(key):
    """The oracle's stored values for a full-size workload (written by tests/golden/make_full_size.py,
    which calls only the oracle)."""
    with open(os.path.join(GOLDEN_DIR, "full_size_oracle.json")) as fh:
        return json.load(fh)[key]


def golden_grad(key):
    return np.load(os.path.join(GOLDEN_DIR, golden(key)["grad_file"])).astype(np.float64)
