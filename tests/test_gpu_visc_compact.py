"""Parity of the compact viscous terms (visc_compact = 1: the gradients of u,
v, w, T and the divergence of the viscous fluxes by the NOHAP/OUCS3 operator)
of the CUDA path with the FP64 oracle, through the C ABI.  Gates as for the
explicit viscous terms: FP64 <= 1e-12 (momentum with the round-off floor of
its pressure-gradient residual), mixed <= 1e-4 for one right-hand side and
<= 1e-5 for the state.  A low Reynolds number makes the viscous terms a large
part of the right-hand side, and each test checks that the oracle's compact
and explicit forms differ by far more than its gate."""
import numpy as np
import pytest

import nopcs_synth as S
import oracle
from gpu_util import binding, field_rel, state_err, stream_ptr, to_dev

pytestmark = pytest.mark.gpu


def _state(N, ctx, p, box=0):
    import torch
    Q = torch.empty((5, p["n"][2], p["n"][1], p["n"][0]), dtype=torch.float64, device="cuda")
    N.nopcs_get_state(ctx, box, Q.data_ptr())
    return Q.cpu().numpy()


def _perturbed(orc, seed):
    Q = orc.initial_state()
    rng = np.random.default_rng(seed)
    Q[4] *= 1 + 1e-4 * rng.standard_normal(Q[4].shape)
    Q[0] *= 1 + 1e-4 * rng.standard_normal(Q[0].shape)
    return Q


def _no_slip(R):
    R = R.copy()
    R[1:4][:, [0, -1]] = 0
    R[1:4][:, :, [0, -1]] = 0
    R[1:4][:, :, :, [0, -1]] = 0
    return R


@pytest.mark.parametrize("prec,bs", [(0, 0), (0, 1), (1, 1)])
def test_rhs_compact_viscous_matches_oracle(prec, bs):
    import torch
    N = binding()
    p = S.box_params((26, 23, 30), sub_n=(8, 24, 12), base_subtract=bs, perturb_amp=1e-3, seed=9, Re=5.0,
                     visc_compact=1)
    ctx = N.nopcs_init([p], prec=prec, stream=stream_ptr())
    try:
        orc = oracle.Solver(p)
        Q = _perturbed(orc, 1)
        ref = _no_slip(orc.rhs(Q))
        explicit = _no_slip(oracle.Solver(dict(p, visc_compact=0)).rhs(Q))
        r = torch.empty(Q.shape, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
        N.nopcs_rhs(ctx, 0, to_dev(Q).data_ptr(), r.data_ptr())
        got = r.cpu().numpy().astype(np.float64)
        d = np.abs(got - ref).reshape(5, -1).max(axis=1)
        s_ = np.abs(ref).reshape(5, -1).max(axis=1)
        sep = np.abs(explicit - ref).reshape(5, -1).max(axis=1)
        if prec == 0:
            pr = (p["gamma"] - 1) * (Q[4] - 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0])
            h = p["len"][0] / (p["n"][0] - 1)
            floor = 30 * np.finfo(float).eps * np.abs(pr).max() / h
            gate = 1e-12 * s_ + np.r_[0.0, floor, floor, floor, 0.0]
        else:
            gate = 1e-4 * s_
        assert np.all(d <= gate), (d / s_, gate / s_)
        # the viscous operator matters far beyond the gate
        assert np.all(sep[1:] > 100 * gate[1:]), (sep / s_, gate / s_)
    finally:
        N.nopcs_destroy(ctx)


@pytest.mark.parametrize("prec,bs", [(0, 0), (0, 1), (1, 1)])
def test_compact_viscous_steps_match_oracle(prec, bs):
    """32^3 box with sub-domains of 12, ten RK4 steps with a filter after
    step 5, at a Reynolds number of 50."""
    N = binding()
    p = S.box_params((32, 30, 34), sub_n=(12, 12, 12), base_subtract=bs, perturb_amp=1e-3, seed=4, Re=50.0,
                     filter_every=5, visc_compact=1)
    ctx = N.nopcs_init([p], prec=prec, stream=stream_ptr())
    try:
        N.nopcs_rk_step(ctx, 10)
        Q = _state(N, ctx, p)
        orc = oracle.Solver(p)
        Q0 = orc.initial_state()
        ref = orc.step(Q0.copy(), 10)
        exp = oracle.Solver(dict(p, visc_compact=0)).step(Q0.copy(), 10)
        # the change over the run, against which the viscous operator shows
        dref = np.abs(ref - Q0).reshape(5, -1).max(axis=1)
        dd = np.abs(Q - ref).reshape(5, -1).max(axis=1)
        sep = np.abs(exp - ref).reshape(5, -1).max(axis=1)
        if prec == 0:
            err = state_err(Q, ref, p)
            assert np.all(err <= 1e-12), (err, field_rel(Q, ref))
            # the change over the run itself agrees to 1e-8 of its size
            assert np.all(dd[1:] <= 1e-8 * dref[1:]), dd / dref
            assert np.all(sep[1:] > 1e3 * dd[1:]), (sep / dref, dd / dref)
        else:
            err = field_rel(Q, ref)
            assert np.all(err <= 1e-5), err
            assert np.all(dd[1:4] <= 1e-2 * dref[1:4]), dd / dref
        d = N.nopcs_diagnostics(ctx, 0)
        assert d["step"] == 10 and d["nonfinite"] == 0
    finally:
        N.nopcs_destroy(ctx)


def test_compact_viscous_graph_equals_direct():
    """The captured CUDA graph and direct launches (profiling on) give
    identical bits, and the compact-path kernels are the ones that ran."""
    N = binding()
    p = S.box_params((40, 36, 44), sub_n=(16, 16, 16), filter_every=2, Re=100.0, perturb_amp=1e-3,
                     visc_compact=1)
    outs = []
    for prof in (0, 1):
        ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, stream=stream_ptr())
        try:
            N.nopcs_set_profiling(ctx, prof)
            N.nopcs_rk_step(ctx, 3)
            outs.append(_state(N, ctx, p))
            if prof:
                t = N.nopcs_profile_read(ctx)
                assert t["visc_grad"][1] == 36 and t["visc_div"][1] == 36
                assert t["visc_flux"][1] == 12 and t["source_rk_update"][1] == 12
                assert t["visc_rk_update"][1] == 0
        finally:
            N.nopcs_destroy(ctx)
    assert np.array_equal(outs[0], outs[1])


def test_compact_viscous_rest_state():
    """An isothermal quiescent box with gravity stays at rest with compact
    viscous terms (base-subtracted mixed form).  The FP32 end-row taps of a
    derivative of the uniform temperature sum to zero only to rounding, which
    gives a heat flux of round-off size; the velocity it drives over four
    steps stays below 1e-10, four orders under the paper's 1e-6 seed."""
    N = binding()
    p = S.box_params((48, 40, 56), sub_n=(16, 16, 16), T_lower=1.0, perturb_amp=0.0, visc_compact=1)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, stream=stream_ptr())
    try:
        N.nopcs_rk_step(ctx, 4)
        d = N.nopcs_diagnostics(ctx, 0)
        assert d["max_speed"] < 1e-10 and d["nonfinite"] == 0
    finally:
        N.nopcs_destroy(ctx)


def test_compact_and_explicit_boxes_in_one_context():
    """A context holding a box with compact viscous terms and one with the
    paper's explicit ones (one CUDA graph, a branch per box) advances each
    exactly as a context of its own does."""
    N = binding()
    boxes = [S.box_params((24, 20, 30), sub_n=(8, 8, 8), seed=3, Re=300.0, perturb_amp=1e-3, visc_compact=1),
             S.box_params((17, 33, 21), sub_n=(5, 16, 0), seed=4, T_lower=1.5, perturb_amp=1e-3)]
    ctx = N.nopcs_init(boxes, prec=N.NOPCS_MIXED, stream=stream_ptr())
    try:
        N.nopcs_rk_step(ctx, 3)
        both = [_state(N, ctx, p, b) for b, p in enumerate(boxes)]
    finally:
        N.nopcs_destroy(ctx)
    for b, p in enumerate(boxes):
        c1 = N.nopcs_init([p], prec=N.NOPCS_MIXED, stream=stream_ptr())
        try:
            N.nopcs_rk_step(c1, 3)
            assert np.array_equal(_state(N, c1, p), both[b])
        finally:
            N.nopcs_destroy(c1)


@pytest.mark.parametrize("visc_compact", [1, 0])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,sub_n", [((5, 5, 5), (0, 0, 0)), ((5, 7, 6), (3, 3, 3)), ((9, 5, 11), (3, 0, 4))])
def test_smallest_boxes(prec, n, sub_n, visc_compact):
    """The smallest boxes (5 points per axis) and sub-domains (3 points),
    with compact and with the paper's explicit viscous terms: every line is
    almost all wall-closure rows and sub-domain ends, and the explicit
    viscous kernel's 32 x 8 tile is wider than the box."""
    import torch
    N = binding()
    p = S.box_params(n, sub_n=sub_n, base_subtract=1, perturb_amp=1e-3, seed=6, Re=20.0, visc_compact=visc_compact)
    ctx = N.nopcs_init([p], prec=prec, stream=stream_ptr())
    try:
        orc = oracle.Solver(p)
        Q = _perturbed(orc, 2)
        ref = _no_slip(orc.rhs(Q))
        r = torch.empty(Q.shape, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
        N.nopcs_rhs(ctx, 0, to_dev(Q).data_ptr(), r.data_ptr())
        got = r.cpu().numpy().astype(np.float64)
        d = np.abs(got - ref).reshape(5, -1).max(axis=1)
        s_ = np.abs(ref).reshape(5, -1).max(axis=1)
        if prec == 0:
            pr = (p["gamma"] - 1) * (Q[4] - 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0])
            h = p["len"][0] / (p["n"][0] - 1)
            floor = 30 * np.finfo(float).eps * np.abs(pr).max() / h
            gate = 1e-12 * s_ + np.r_[0.0, floor, floor, floor, 0.0]
        else:
            gate = 1e-4 * s_
        assert np.all(d <= gate), (d / s_, gate / s_)
    finally:
        N.nopcs_destroy(ctx)
