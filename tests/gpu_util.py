"""Helpers for the GPU tests: build the library once, torch device buffers."""
import os

import numpy as np


def require_lib():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    from paper_1301_1247_gb300 import build, hbs
    if not os.path.exists(hbs.LIB_PATH):
        build.build()
    return hbs


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
