"""Parity of the banded explicit form of nopcs_derivative (the equivalent
explicit scheme C = A^-1 B, truncated at 1e-8, at every row) with the FP64
oracle's NOHAP derivative: FP32 fields, <= 1e-5 of max |f'| (order 1), 5e-5
(order 2).  Shapes cover lines shorter than one row tile (every row
tabulated), ragged line tiles and row tiles, and lines long enough for the
interior stencil."""
import numpy as np
import pytest

import nopcs_synth as S
import oracle
from gpu_util import binding, field_rel, stream_ptr, to_dev

pytestmark = pytest.mark.gpu


def _ctx(N, n, sub_n, form):
    p = S.box_params(n, sub_n=sub_n, perturb_amp=0.0)
    return N.nopcs_init([p], prec=N.NOPCS_MIXED, form=form, stream=stream_ptr()), p


@pytest.mark.parametrize("n,sub_n", [((40, 36, 33), (16, 16, 16)), ((130, 66, 35), (64, 32, 8)),
                                     ((200, 140, 129), (64, 64, 64)), ((7, 9, 11), (3, 4, 5)),
                                     ((257, 70, 97), (0, 24, 32))])
def test_band_form_parity(n, sub_n):
    import torch
    N = binding()
    ctx, p = _ctx(N, n, sub_n, N.NOPCS_FORM_BANDED)
    try:
        assert N.nopcs_box_info(ctx, 0)["deriv_form"] == [N.NOPCS_FORM_BANDED] * 3
        f = S.sine_field(n, kmax=16, seed=7, noise=1e-3)
        fd = to_dev(f, np.float32)
        fin = fd.cpu().numpy().astype(np.float64)
        h = p["len"][0] / (n[0] - 1)
        out = torch.empty_like(fd)
        for axis in range(3):
            for order in (1, 2):
                out.fill_(float("nan"))
                N.nopcs_derivative(ctx, 0, axis, order, 1, fd.data_ptr(), out.data_ptr(), stream_ptr())
                N.nopcs_synchronize(ctx)
                got = out.cpu().numpy().astype(np.float64)
                ref = oracle.deriv3d(fin, axis, h, sub_n[axis])
                if order == 2:
                    ref = oracle.deriv3d(ref, axis, h, sub_n[axis])
                err = field_rel(got[None], ref[None])[0]
                print("band parity", n, sub_n, "axis", axis, "order", order, "err %.3e" % err)
                assert np.all(np.isfinite(got)), (axis, order)
                assert err <= (1e-5 if order == 1 else 5e-5), (axis, order, err)
    finally:
        N.nopcs_destroy(ctx)


def test_band_form_modified_wavenumber():
    """A single Fourier mode far from the walls: the banded derivative takes
    the OUCS3 modified wavenumber (closed form) to FP32 accuracy."""
    import torch
    N = binding()
    n = (512, 8, 8)
    ctx, p = _ctx(N, n, (64, 8, 8), N.NOPCS_FORM_BANDED)
    try:
        h = p["len"][0] / (n[0] - 1)
        x = np.arange(n[0]) * h
        k = 2 * np.pi * 17
        f = np.broadcast_to(np.sin(k * x), (n[2], n[1], n[0])).copy()
        fd = to_dev(f, np.float32)
        out = torch.empty_like(fd)
        N.nopcs_derivative(ctx, 0, 0, 1, 1, fd.data_ptr(), out.data_ptr(), stream_ptr())
        N.nopcs_synchronize(ctx)
        got = out.cpu().numpy()[3, 3, 60:-60]
        al, b1, b2 = oracle.OUCS3[:3]
        kh = k * h
        keq = (2 * b1 * np.sin(kh) + 2 * b2 * np.sin(2 * kh)) / (1 + 2 * al * np.cos(kh)) / h
        ref = keq * np.cos(k * x[60:-60])
        assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))
    finally:
        N.nopcs_destroy(ctx)


def test_band_form_fp64_fields_use_thomas():
    """FP64 fields keep the Thomas form under a banded context (<= 1e-12)."""
    import torch
    N = binding()
    n = (40, 36, 33)
    ctx, p = _ctx(N, n, (16, 16, 16), N.NOPCS_FORM_BANDED)
    try:
        f = S.sine_field(n, kmax=8, seed=3, noise=0.0)
        fd = to_dev(f)
        out = torch.empty_like(fd)
        N.nopcs_derivative(ctx, 0, 2, 1, 0, fd.data_ptr(), out.data_ptr(), stream_ptr())
        N.nopcs_synchronize(ctx)
        ref = oracle.deriv3d(f, 2, p["len"][0] / 39, 16)
        assert field_rel(out.cpu().numpy()[None], ref[None])[0] <= 1e-12
    finally:
        N.nopcs_destroy(ctx)


def test_band_form_sampled_lines_512():
    """512^3 at the benchmark's launch shape: sampled lines against the oracle
    evaluated one line at a time."""
    import torch
    N = binding()
    n = (512, 512, 512)
    ctx, p = _ctx(N, n, (64, 64, 64), N.NOPCS_FORM_BANDED)
    try:
        px, py, pz = [torch.from_numpy(v).cuda() for v in S.sine_profiles(n, kmax=64, seed=7)]
        fd = (px[None, None, :] + py[None, :, None] + pz[:, None, None]).float().contiguous()
        h = p["len"][0] / (n[0] - 1)
        out = torch.empty_like(fd)
        rng = np.random.default_rng(3)
        for axis in range(3):
            N.nopcs_derivative(ctx, 0, axis, 1, 1, fd.data_ptr(), out.data_ptr(), stream_ptr())
            N.nopcs_synchronize(ctx)
            prof = [px, py, pz][axis].double().cpu().numpy()
            ref = oracle.Op(n[axis], kind=0, sub_n=64).nopcs(prof) / h
            scale = np.max(np.abs(ref))
            for _ in range(6):
                i, j = rng.integers(0, 512, 2)
                if axis == 0:
                    line = out[i, j, :]
                elif axis == 1:
                    line = out[i, :, j]
                else:
                    line = out[:, i, j]
                got = line.double().cpu().numpy()
                assert np.max(np.abs(got - ref)) <= 1e-5 * scale, axis
    finally:
        N.nopcs_destroy(ctx)
