"""Helpers for the GPU parity tests: build + load the CUDA library, device arrays."""
import numpy as np
import pytest


def binding():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2203_00879_gb300 import build
    build.build()
    from paper_2203_00879_gb300 import nopcs
    return nopcs


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a if dtype is None else a.astype(dtype)))
    return t.cuda()


def stream_ptr():
    import torch
    return torch.cuda.current_stream().cuda_stream


def field_rel(a, b):
    """max |a - b| / max |b| per leading component."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.abs(a - b).reshape(a.shape[0], -1).max(axis=1)
    s = np.abs(b).reshape(b.shape[0], -1).max(axis=1)
    return d / np.where(s == 0, 1.0, s)
