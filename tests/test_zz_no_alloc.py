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


def _free_bytes():
    """Free device memory as the driver reports it, plus what torch's caching
    allocator holds."""
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0] + torch.cuda.memory_reserved()


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
                # same kernels in the same form: identical bits
                assert np.array_equal(g, r), axis
    finally:
        N.nopcs_destroy(ctx)


@pytest.mark.parametrize("form", ["GEMM_3XTF32", "GEMM_BF16X3", "BANDED"])
def test_noalloc_takes_the_boxs_derivative_form(form):
    """Under the tensor-core and banded forms the allocation-free call runs the
    same per-axis form as nopcs_derivative(order = 2): identical bits."""
    import torch
    N = binding()
    n = (70, 45, 37)
    p = S.box_params(n, sub_n=(24, 16, 0), perturb_amp=0.0)
    fcode = getattr(N, "NOPCS_FORM_" + form)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, form=fcode, stream=stream_ptr())
    try:
        assert N.nopcs_box_info(ctx, 0)["deriv_form"] == [fcode] * 3
        fd = to_dev(S.sine_field(n, kmax=16, seed=7, noise=1e-3), np.float32)
        ref = torch.empty_like(fd)
        got = torch.empty_like(fd)
        for axis in range(3):
            N.nopcs_derivative(ctx, 0, axis, 2, 1, fd.data_ptr(), ref.data_ptr(), stream_ptr())
            for _ in range(2):
                got.fill_(float("nan"))
                N.nopcs_derivative2_noalloc(ctx, 0, axis, 1, fd.data_ptr(), got.data_ptr(), stream_ptr())
                N.nopcs_synchronize(ctx)
                assert torch.equal(got, ref), (form, axis)
    finally:
        N.nopcs_destroy(ctx)


def test_noalloc_first_call_allocates_nothing():
    """In a fresh context, calls of the allocation-free entry point, the first
    one included, leave the device's free memory unchanged, while the first
    order-2 nopcs_derivative allocates its scratch (so the measurement would
    see an allocation of that size)."""
    import torch
    N = binding()
    n = (128, 96, 80)  # 983,040 points: 7.5 MiB of FP64 scratch
    p = S.box_params(n, sub_n=(64, 32, 40), perturb_amp=0.0)
    fd = to_dev(S.sine_field(n, kmax=8, seed=3, noise=0.0), np.float64)
    got = torch.empty_like(fd)
    ref = torch.empty_like(fd)
    ctx = N.nopcs_init([p], prec=N.NOPCS_FP64, form=N.NOPCS_FORM_THOMAS, stream=stream_ptr())
    try:
        # order 1 first: the line kernels' first launches happen outside the
        # measured window
        N.nopcs_derivative(ctx, 0, 0, 1, 0, fd.data_ptr(), got.data_ptr(), stream_ptr())
        free0 = _free_bytes()
        for axis in (0, 1, 2, 0):
            N.nopcs_derivative2_noalloc(ctx, 0, axis, 0, fd.data_ptr(), got.data_ptr(), stream_ptr())
        assert _free_bytes() == free0
        N.nopcs_derivative(ctx, 0, 0, 2, 0, fd.data_ptr(), ref.data_ptr(), stream_ptr())
        assert free0 - _free_bytes() >= n[0] * n[1] * n[2] * 8
        N.nopcs_derivative2_noalloc(ctx, 0, 0, 0, fd.data_ptr(), got.data_ptr(), stream_ptr())
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
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
