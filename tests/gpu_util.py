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


def state_err(Q, ref, p):
    """Per-variable L-inf errors used as gates: rho and E relative to their
    field maximum; momentum relative to max(rho) * max(c), c = sqrt(T)/M the
    sound speed, the natural momentum scale of this compressible flow (the
    flow's own momentum is 1e-4 of it or less, so its field-relative error
    measures FP64 round-off of the O(1/(gamma M^2)) pressure terms, not
    parity)."""
    Q = np.asarray(Q, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    gam, M = p["gamma"], p["M"]
    rho = ref[0]
    pr = (gam - 1) * (ref[4] - 0.5 * (ref[1] ** 2 + ref[2] ** 2 + ref[3] ** 2) / rho)
    T = gam * M * M * pr / rho
    mscale = np.max(np.abs(rho)) * np.sqrt(np.max(T)) / M
    d = np.abs(Q - ref).reshape(5, -1).max(axis=1)
    out = d / np.abs(ref).reshape(5, -1).max(axis=1)
    out[1:4] = d[1:4] / mscale
    return out


def dist_rel(Q, ref, Q0):
    """Disturbance-relative L-inf error per conserved variable:
    max |Q - ref| / max |ref - Q0|, with Q0 the initial state both runs
    started from.  For rho and E the flow changes only ~1e-4 of the field, so
    this is the figure that shows an error of the size of the flow itself."""
    Q = np.asarray(Q, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    Q0 = np.asarray(Q0, dtype=np.float64)
    d = np.abs(Q - ref).reshape(Q.shape[0], -1).max(axis=1)
    s = np.abs(ref - Q0).reshape(Q.shape[0], -1).max(axis=1)
    return d / np.where(s == 0, 1.0, s)
