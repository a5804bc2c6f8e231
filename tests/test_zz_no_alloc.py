"""nopcs_derivative2_noalloc, the allocation-free second derivative.

Callers whose device memory belongs to their own pool allocator, or whose loop
cannot absorb the implicit synchronisation of cudaMalloc/cudaFree, cannot use
nopcs_derivative(order=2), which allocates its scratch on first use.  The
no-allocation variant keeps the intermediate in a fixed 16 MiB array of the
library.  This file is collected last so that a run stopping at its first
failure has already run every other test; it also passes alone in a fresh
process.
"""
import numpy as np
import pytest

import nopcs_synth as S
from gpu_util import binding, stream_ptr, to_dev

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.mark.parametrize("dtype", [0, 1])
def test_noalloc_matches_order2_twice(dtype):
    import torch
    N = binding()
    n = (70, 45, 37)
    p = S.box_params(n, sub_n=(24, 16, 0), perturb_amp=0.0)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, stream=stream_ptr())
    try:
        f = S.sine_field(n, kmax=16, seed=7, noise=1e-3)
        fd = to_dev(f, np.float64 if dtype == 0 else np.float32)
        ref = torch.empty_like(fd)
        got = torch.empty_like(fd)
        for axis in range(3):
            N.nopcs_derivative(ctx, 0, axis, 2, dtype, fd.data_ptr(), ref.data_ptr(), stream_ptr())
            for _ in range(2):  # two calls in a row reuse the same static scratch
                got.fill_(float("nan"))
                N.nopcs_derivative2_noalloc(ctx, 0, axis, dtype, fd.data_ptr(), got.data_ptr(), stream_ptr())
                torch.cuda.synchronize()
                r = ref.double().cpu().numpy()
                g = got.double().cpu().numpy()
                err = np.max(np.abs(g - r)) / np.max(np.abs(r))
                assert np.all(np.isfinite(g)) and err <= TOL[dtype], (axis, err)
    finally:
        N.nopcs_destroy(ctx)


def test_noalloc_rejects_fields_beyond_the_static_scratch():
    import torch
    N = binding()
    n = (129, 128, 128)  # 2,113,536 points: above 2^21 FP64 values
    p = S.box_params(n, sub_n=(64, 64, 64), perturb_amp=0.0)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, stream=stream_ptr())
    try:
        f = torch.zeros(n[::-1], dtype=torch.float64, device="cuda")
        out = torch.empty_like(f)
        with pytest.raises(N.NopcsError) as ei:
            N.nopcs_derivative2_noalloc(ctx, 0, 0, 0, f.data_ptr(), out.data_ptr(), stream_ptr())
        assert ei.value.status == N.NOPCS_EINVAL and "16 MiB" in str(ei.value)
        # the same field in FP32 (4 bytes a point) fits
        f32 = f.float()
        o32 = torch.empty_like(f32)
        N.nopcs_derivative2_noalloc(ctx, 0, 0, 1, f32.data_ptr(), o32.data_ptr(), stream_ptr())
        torch.cuda.synchronize()
        assert torch.all(o32 == 0)
    finally:
        N.nopcs_destroy(ctx)
