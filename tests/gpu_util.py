"""Helpers for the GPU tests: build the library once, move arrays between numpy and torch."""

import numpy as np
import pytest
import torch


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_0262_gb300 import build
    build.build()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to("cuda")


def to_np(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rand_eo(n, vh, rng):
    return rng.standard_normal((n, vh, 4, 3)) + 1j * rng.standard_normal((n, vh, 4, 3))
