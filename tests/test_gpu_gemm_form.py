"""Parity of the tensor-core forms of nopcs_derivative (tcgen05: 3xTF32, and
BF16x3 with three BF16 parts per operand) with the FP64 oracle: FP32 fields,
<= 1e-5 of max |f'| (order 1), 5e-5 (order 2)."""
import numpy as np
import pytest

import nopcs_synth as S
import oracle
from gpu_util import binding, field_rel, stream_ptr, to_dev

pytestmark = pytest.mark.gpu


FORMS = ("3xtf32", "bf16x3")


def _ctx(N, n, sub_n, form="3xtf32"):
    p = S.box_params(n, sub_n=sub_n, perturb_amp=0.0)
    f = N.NOPCS_FORM_GEMM_3XTF32 if form == "3xtf32" else N.NOPCS_FORM_GEMM_BF16X3
    return N.nopcs_init([p], prec=N.NOPCS_MIXED, form=f, stream=stream_ptr()), p


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,sub_n", [((40, 36, 33), (16, 16, 16)), ((130, 66, 35), (64, 32, 8)),
                                     ((200, 140, 129), (64, 64, 64)), ((7, 9, 11), (3, 4, 5))])
def test_gemm_form_parity(n, sub_n, form):
    import torch
    N = binding()
    ctx, p = _ctx(N, n, sub_n, form)
    try:
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
                print("gemm parity", form, n, sub_n, "axis", axis, "order", order, "err %.3e" % err)
                assert np.all(np.isfinite(got)), (axis, order)
                assert err <= (1e-5 if order == 1 else 5e-5), (axis, order, err)
    finally:
        N.nopcs_destroy(ctx)


@pytest.mark.parametrize("form", FORMS)
def test_gemm_form_fp64_fields_use_thomas(form):
    """FP64 fields keep the Thomas form under a tensor-core context (<= 1e-12)."""
    import torch
    N = binding()
    n = (40, 36, 33)
    ctx, p = _ctx(N, n, (16, 16, 16), form)
    try:
        f = S.sine_field(n, kmax=8, seed=3, noise=0.0)
        fd = to_dev(f)
        out = torch.empty_like(fd)
        N.nopcs_derivative(ctx, 0, 1, 1, 0, fd.data_ptr(), out.data_ptr(), stream_ptr())
        N.nopcs_synchronize(ctx)
        ref = oracle.deriv3d(f, 1, p["len"][0] / 39, 16)
        assert field_rel(out.cpu().numpy()[None], ref[None])[0] <= 1e-12
    finally:
        N.nopcs_destroy(ctx)


def test_autotuner_choices_and_parity():
    """sub_n = -1 and NOPCS_FORM_AUTO: the autotuner picks a sub-domain length
    among 32/64/128 and a derivative form per axis; results still match the
    oracle (NOHAP results do not depend on the split)."""
    import torch
    N = binding()
    n = (160, 140, 130)
    p = S.box_params(n, sub_n=(-1, -1, -1), perturb_amp=1e-4)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, form=N.NOPCS_FORM_AUTO, stream=stream_ptr())
    try:
        info = N.nopcs_box_info(ctx, 0)
        assert all(sn in (32, 64, 128) for sn in info["sub_n"]), info
        assert all(fm in (N.NOPCS_FORM_THOMAS, N.NOPCS_FORM_GEMM_3XTF32, N.NOPCS_FORM_GEMM_BF16X3,
                          N.NOPCS_FORM_BANDED) for fm in info["deriv_form"]), info
        f = S.sine_field(n, kmax=16, seed=5, noise=1e-3)
        fd = to_dev(f, np.float32)
        out = torch.empty_like(fd)
        h = p["len"][0] / (n[0] - 1)
        for axis in range(3):
            N.nopcs_derivative(ctx, 0, axis, 1, 1, fd.data_ptr(), out.data_ptr(), stream_ptr())
            N.nopcs_synchronize(ctx)
            ref = oracle.deriv3d(fd.cpu().numpy().astype(np.float64), axis, h, info["sub_n"][axis])
            assert field_rel(out.cpu().numpy()[None], ref[None])[0] <= 1e-5
        print("autotuner", info)
        # a few RK steps with the tuned sub-domains match the oracle
        N.nopcs_rk_step(ctx, 3)
        Q = torch.empty((5, n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
        N.nopcs_get_state(ctx, 0, Q.data_ptr())
        pr = dict(p, sub_n=tuple(info["sub_n"]), base_subtract=1)
        orc = oracle.Solver(pr)
        ref = orc.step(orc.initial_state(), 3)
        assert np.all(field_rel(Q.cpu().numpy(), ref) <= 1e-5)
    finally:
        N.nopcs_destroy(ctx)


def test_bf16x3_reports_its_form_and_matches_3xtf32_on_a_512_line():
    """A full-length 512-point line tile (the microbenchmark's line length):
    both tensor-core forms agree with the oracle on sampled lines."""
    import torch
    N = binding()
    n = (512, 16, 16)
    out = {}
    for form in FORMS:
        ctx, p = _ctx(N, n, (64, 16, 16), form)
        try:
            info = N.nopcs_box_info(ctx, 0)
            want = N.NOPCS_FORM_GEMM_3XTF32 if form == "3xtf32" else N.NOPCS_FORM_GEMM_BF16X3
            assert all(fm == want for fm in info["deriv_form"]), info
            f = S.sine_field(n, kmax=64, seed=9, noise=1e-3)
            fd = to_dev(f, np.float32)
            o = torch.empty_like(fd)
            N.nopcs_derivative(ctx, 0, 0, 1, 1, fd.data_ptr(), o.data_ptr(), stream_ptr())
            N.nopcs_synchronize(ctx)
            out[form] = o.cpu().numpy().astype(np.float64)
            ref = oracle.deriv3d(fd.cpu().numpy().astype(np.float64), 0, p["len"][0] / 511, 64)
            assert field_rel(out[form][None], ref[None])[0] <= 1e-5
        finally:
            N.nopcs_destroy(ctx)
