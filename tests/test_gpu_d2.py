"""The compact second derivative (nopcs_derivative order NOPCS_ORDER_D2_COMPACT:
Lele's sixth-order tridiagonal scheme with its own NOHAP closure) against the
oracle on shapes with several sub-domains, ragged tiles and single-sub-domain
axes.  FP64: <= 1e-12 of max |f''|.  FP32: <= 1e-5 of max |f''| plus the
round-off floor of a second difference, 16 eps_32 max |f| / h^2 (the
right-hand side cancels O(|f|) terms down to O(h^2 f''), so FP32 rounding of
|f| reaches f'' amplified by 1/h^2; on fine grids this floor dominates)."""
import numpy as np
import pytest

import nopcs_synth as S
import oracle
from gpu_util import binding, field_rel, stream_ptr, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,sub_n", [((40, 36, 33), (16, 16, 16)), ((130, 66, 35), (64, 32, 0)),
                                     ((7, 9, 11), (3, 4, 5)), ((97, 70, 129), (24, 0, 64))])
def test_d2_compact_parity(n, sub_n):
    import torch
    N = binding()
    p = S.box_params(n, sub_n=sub_n, perturb_amp=0.0)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, form=N.NOPCS_FORM_THOMAS, stream=stream_ptr())
    try:
        h = p["len"][0] / (n[0] - 1)
        f = S.sine_field(n, kmax=8, seed=5, noise=0.0)
        hs = [p["len"][d] / (n[d] - 1) for d in range(3)]
        for dtype, tol in ((0, 1e-12), (1, 1e-5)):
            fd = to_dev(f, np.float64 if dtype == 0 else np.float32)
            fin = fd.cpu().numpy().astype(np.float64)
            out = torch.empty_like(fd)
            for axis in range(3):
                out.fill_(float("nan"))
                N.nopcs_derivative(ctx, 0, axis, N.NOPCS_ORDER_D2_COMPACT, dtype, fd.data_ptr(), out.data_ptr(),
                                   stream_ptr())
                N.nopcs_synchronize(ctx)
                got = out.cpu().numpy().astype(np.float64)
                ref = oracle.deriv3d(fin, axis, h, sub_n[axis], kind=oracle.D2)
                err = field_rel(got[None], ref[None])[0]
                print("d2 parity", n, sub_n, "dtype", dtype, "axis", axis, "err %.3e" % err)
                assert np.all(np.isfinite(got))
                floor = 0.0 if dtype == 0 else 16 * np.finfo(np.float32).eps * np.max(np.abs(fin)) / hs[axis] ** 2
                assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)) + floor, (dtype, axis, err)
    finally:
        N.nopcs_destroy(ctx)


def test_d2_compact_closed_form_on_a_sine():
    """Interior points of sin(kx) take -k_eq^2 sin(kx) with Lele's modified
    wavenumber (FP64 path)."""
    import torch
    N = binding()
    n = (256, 8, 8)
    p = S.box_params(n, sub_n=(64, 8, 8), perturb_amp=0.0)
    ctx = N.nopcs_init([p], prec=N.NOPCS_FP64, stream=stream_ptr())
    try:
        h = p["len"][0] / (n[0] - 1)
        x = np.arange(n[0]) * h
        k = 2 * np.pi * 23
        f = np.broadcast_to(np.sin(k * x), (n[2], n[1], n[0])).copy()
        fd = to_dev(f)
        out = torch.empty_like(fd)
        N.nopcs_derivative(ctx, 0, 0, N.NOPCS_ORDER_D2_COMPACT, 0, fd.data_ptr(), out.data_ptr(), stream_ptr())
        N.nopcs_synchronize(ctx)
        al, a, b = oracle.LELE_D2
        kh = k * h
        keq2 = (2 * a * (1 - np.cos(kh)) + 0.5 * b * (1 - np.cos(2 * kh))) / (1 + 2 * al * np.cos(kh)) / h ** 2
        got = out.cpu().numpy()[4, 4, 40:-40]
        assert np.max(np.abs(got + keq2 * f[4, 4, 40:-40])) <= 1e-10 * keq2
    finally:
        N.nopcs_destroy(ctx)
