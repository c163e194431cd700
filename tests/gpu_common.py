"""Shared helpers of the GPU parity tests (collected only through -m gpu tests)."""
import numpy as np
import pytest

import oracle as O


def require_gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2304_12465_gb300 as K
    K.load()
    return K


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def f32_product_bound(X, kern, sigma, lam, V, rows=None):
    """Entrywise scale of a float32 product: A|V| + lam|V| (A >= 0)."""
    return O.kmatvec(X, kern, sigma, lam, np.abs(V), rows)
