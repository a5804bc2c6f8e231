"""One box split into z-slabs (nopcs_slab_*), on one GPU: the ranks of a
three-way split run one after another (no kernel waits for another); each
slab gets its halo planes copied from the whole field, as exchange_halo would
deliver them, and its own planes must equal nopcs_derivative of the whole box
bit for bit, along z (the split axis) and along x and y, in FP64 and FP32, and
match the FP64 oracle."""
import numpy as np
import pytest

import nopcs_synth as S
import oracle
from gpu_util import binding, field_rel, stream_ptr, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [0, 1])
def test_slabs_equal_the_whole_box(dtype):
    import torch
    from paper_2203_00879_gb300 import halo
    N = binding()
    n = (40, 33, 300)
    p = S.box_params(n, sub_n=(16, 12, 32), perturb_amp=0.0)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, form=N.NOPCS_FORM_THOMAS, stream=stream_ptr())
    f = S.sine_field(n, kmax=12, seed=5, noise=1e-3)
    fd = to_dev(f, np.float64 if dtype == 0 else np.float32)
    h = 1.0 / (n[0] - 1)
    slabs = []
    try:
        whole = []
        for axis in range(3):
            out = torch.empty_like(fd)
            N.nopcs_derivative(ctx, 0, axis, 1, dtype, fd.data_ptr(), out.data_ptr(), stream_ptr())
            whole.append(out)
        torch.cuda.synchronize()
        bounds = halo.slab_bounds(n[2], 32, 3)
        assert len(bounds) == 3 and bounds[0][0] == 0 and bounds[-1][1] == n[2]
        for z0, z1 in bounds:
            sl = N.nopcs_slab_create(p, z0, z1)
            slabs.append(sl)
            lo, hi = N.nopcs_slab_extent(sl, dtype)
            assert (lo, hi) == halo.slab_extent(n[2], 32, dtype, z0, z1)
            loc = fd[lo:hi].clone()  # own planes plus the halo a neighbour sends
            for axis in range(3):
                got = torch.full((z1 - z0, n[1], n[0]), float("nan"), dtype=fd.dtype, device="cuda")
                N.nopcs_slab_derivative(sl, axis, dtype, loc.data_ptr(), got.data_ptr(), stream_ptr())
                torch.cuda.synchronize()
                assert torch.equal(got, whole[axis][z0:z1]), (z0, z1, axis)
        # and the whole against the oracle (FP64: the single-domain NOHAP solve)
        if dtype == 0:
            for axis in range(3):
                ref = oracle.deriv3d(f, axis, h, p["sub_n"][axis])
                assert field_rel(whole[axis].cpu().numpy()[None], ref[None])[0] <= 1e-12
    finally:
        for sl in slabs:
            N.nopcs_slab_destroy(sl)
        N.nopcs_destroy(ctx)


def test_slab_rejects_unaligned_bounds():
    N = binding()
    p = S.box_params((20, 20, 100), sub_n=(8, 8, 32), perturb_amp=0.0)
    with pytest.raises(N.NopcsError) as ei:
        N.nopcs_slab_create(p, 0, 40)
    assert ei.value.status == N.NOPCS_EINVAL and "boundaries" in str(ei.value)
