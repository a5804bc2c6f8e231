"""Parity of the CUDA RK path (nopcs_init / nopcs_rhs / nopcs_rk_step /
nopcs_filter / nopcs_diagnostics, through the C ABI) with the FP64 oracle.
FP64 form: <= 1e-12 L-inf per conserved variable (rho and E relative to their
field maximum, momentum relative to max(rho) max(c)); mixed form: <= 1e-5
field-relative against the oracle's base-subtracted FP64 run."""
import numpy as np
import pytest

import nopcs_synth as S
import oracle
from gpu_util import binding, dist_rel, field_rel, state_err, stream_ptr, to_dev

# mixed form, disturbance-relative gate: max |Q_gpu - Q_orc| / max |Q_orc - Q_0|
MIXED_DIST_GATE = 2e-5

pytestmark = pytest.mark.gpu


def _state(N, ctx, p, box=0):
    import torch
    Q = torch.empty((5, p["n"][2], p["n"][1], p["n"][0]), dtype=torch.float64, device="cuda")
    N.nopcs_get_state(ctx, box, Q.data_ptr())
    return Q.cpu().numpy()


def _ctx(N, p, prec):
    return N.nopcs_init([p], prec=prec, stream=stream_ptr())


def test_initial_state_matches_oracle():
    N = binding()
    p = S.box_params((21, 18, 24), sub_n=(8, 8, 8), seed=5)
    ctx = _ctx(N, p, N.NOPCS_FP64)
    try:
        Q = _state(N, ctx, p)
        ref = oracle.Solver(p).initial_state()
        assert np.all(field_rel(Q, ref) <= 1e-15)
        # perturbation identical bit for bit (same generator, same counters)
        assert np.array_equal(Q[1:4] != 0, ref[1:4] != 0)
    finally:
        N.nopcs_destroy(ctx)


@pytest.mark.parametrize("prec,bs", [(0, 0), (0, 1), (1, 1)])
def test_rhs_matches_oracle(prec, bs):
    """One right-hand-side evaluation on a perturbed state."""
    import torch
    N = binding()
    p = S.box_params((26, 23, 30), sub_n=(8, 24, 12), base_subtract=bs, perturb_amp=1e-3, seed=9)
    ctx = _ctx(N, p, prec)
    try:
        orc = oracle.Solver(p)
        Q = orc.initial_state()
        rng = np.random.default_rng(1)
        Q[4] *= 1 + 1e-4 * rng.standard_normal(Q[4].shape)
        Q[0] *= 1 + 1e-4 * rng.standard_normal(Q[0].shape)
        ref = orc.rhs(Q)
        ref[1:4][:, [0, -1]] = 0
        ref[1:4][:, :, [0, -1]] = 0
        ref[1:4][:, :, :, [0, -1]] = 0
        r = torch.empty(Q.shape, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
        N.nopcs_rhs(ctx, 0, to_dev(Q).data_ptr(), r.data_ptr())
        got = r.cpu().numpy().astype(np.float64)
        err = field_rel(got, ref)
        if prec == 0:
            # the momentum right-hand side is a small residual of pressure-gradient
            # terms of size p/h: allow 30 ulps of that on top of 1e-12 of max |R|
            pr = (p["gamma"] - 1) * (Q[4] - 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0])
            h = p["len"][0] / (p["n"][0] - 1)
            floor = 30 * np.finfo(float).eps * np.abs(pr).max() / h
            d = np.abs(got - ref).reshape(5, -1).max(axis=1)
            s_ = np.abs(ref).reshape(5, -1).max(axis=1)
            assert np.all(d[[0, 4]] <= 1e-12 * s_[[0, 4]]), err
            assert np.all(d[1:4] <= 1e-12 * s_[1:4] + floor), (err, d, floor)
        else:
            assert np.all(err <= 1e-4), err
    finally:
        N.nopcs_destroy(ctx)


@pytest.mark.parametrize("prec,bs", [(0, 0), (0, 1), (1, 1)])
def test_config0_50_steps(prec, bs):
    """48^3 two-temperature box, sub-domains of 24, 50 RK4 steps at the paper's
    time step, filter after step 50 (the small workload)."""
    N = binding()
    p = S.box_params((48, 48, 48), sub_n=(24, 24, 24), base_subtract=bs, seed=1)
    ctx = _ctx(N, p, prec)
    try:
        N.nopcs_rk_step(ctx, 50)
        Q = _state(N, ctx, p)
        orc = oracle.Solver(p)
        Q0 = orc.initial_state()
        ref = orc.step(Q0, 50)
        if prec == 0:
            err = state_err(Q, ref, p)
            assert np.all(err <= 1e-12), (err, field_rel(Q, ref))
        else:
            err = field_rel(Q, ref)
            dr = dist_rel(Q, ref, Q0)
            print("config0 mixed: field-relative", err, "disturbance-relative", dr)
            assert np.all(err <= 1e-5), err
            assert np.all(dr <= MIXED_DIST_GATE), dr
        d = N.nopcs_diagnostics(ctx, 0)
        assert d["step"] == 50 and d["nonfinite"] == 0
    finally:
        N.nopcs_destroy(ctx)


def test_filter_matches_oracle():
    N = binding()
    for bs in (0, 1):
        p = S.box_params((30, 27, 33), sub_n=(8, 16, 0), base_subtract=bs, perturb_amp=1e-3)
        ctx = _ctx(N, p, N.NOPCS_FP64)
        try:
            orc = oracle.Solver(p)
            N.nopcs_filter(ctx, 0)
            Q = _state(N, ctx, p)
            ref = orc.filter(orc.initial_state())
            assert np.all(field_rel(Q, ref) <= 1e-13)
        finally:
            N.nopcs_destroy(ctx)


def test_mixed_filter_matches_oracle():
    """Mixed form: the FP32 filter of the base deviation, applied to the FP64
    state as Q += F(D) - D, against the oracle's FP64 base-subtracted filter."""
    N = binding()
    p = S.box_params((30, 27, 33), sub_n=(8, 16, 0), base_subtract=1, perturb_amp=1e-3, seed=4)
    ctx = _ctx(N, p, N.NOPCS_MIXED)
    try:
        orc = oracle.Solver(p)
        Q = orc.initial_state()
        rng = np.random.default_rng(2)
        Q[0] *= 1 + 1e-4 * rng.standard_normal(Q[0].shape)
        Q[4] *= 1 + 1e-4 * rng.standard_normal(Q[4].shape)
        N.nopcs_set_state(ctx, 0, to_dev(Q).data_ptr())
        N.nopcs_filter(ctx, 0)
        got = _state(N, ctx, p)
        ref = orc.filter(Q)
        err = field_rel(got, ref)
        assert np.all(err <= 1e-5), err
        # the filter changed the state by far more than the error
        assert np.all(field_rel(Q, ref)[1:4] > 100 * err[1:4])
        # points within three nodes of a wall along every axis are never
        # filtered: their state keeps its bits
        assert np.array_equal(got[:, :3, :3, :3], Q[:, :3, :3, :3])
        assert np.array_equal(got[:, -3:, -3:, -3:], Q[:, -3:, -3:, -3:])
    finally:
        N.nopcs_destroy(ctx)


def test_diagnostics_match_oracle():
    N = binding()
    p = S.box_params((20, 22, 26), sub_n=(8, 8, 8), perturb_amp=1e-3)
    ctx = _ctx(N, p, N.NOPCS_FP64)
    try:
        N.nopcs_rk_step(ctx, 3)
        Q = _state(N, ctx, p)
        d = N.nopcs_diagnostics(ctx, 0)
        r = oracle.Solver(p).diagnostics(Q)
        for k in ("mass", "energy_total"):
            assert abs(d[k] - r[k]) <= 1e-13 * abs(r[k])
        for k in ("max_speed", "max_dp", "max_mach"):
            assert abs(d[k] - r[k]) <= 1e-12 * abs(r[k])
        assert np.allclose(d["momentum"], r["momentum"], rtol=1e-10, atol=1e-22)
        d2 = N.nopcs_diagnostics(ctx, 0)
        assert d2 == d  # fixed reduction order
    finally:
        N.nopcs_destroy(ctx)


def test_deterministic_and_graph_equals_direct():
    """Two contexts, one replaying the CUDA graph and one launching directly
    with profiling on, give identical bits."""
    N = binding()
    p = S.box_params((40, 36, 44), sub_n=(16, 16, 16), filter_every=2)
    outs = []
    for prof in (0, 1):
        ctx = _ctx(N, p, N.NOPCS_MIXED)
        try:
            N.nopcs_set_profiling(ctx, prof)
            N.nopcs_rk_step(ctx, 5)
            outs.append(_state(N, ctx, p))
            if prof:
                t = N.nopcs_profile_read(ctx)
                assert t["sweep_x"][1] == 20 and t["filter"][1] == 2
                # the mixed form recovers primitives inside the stage kernels:
                # no separate prep launch during steps
                compact_only = ("visc_grad", "visc_flux", "visc_div", "source_rk_update")
                assert all(v[0] > 0 for k, v in t.items() if k not in ("diagnostics", "prep") + compact_only)
                assert all(t[k][1] == 0 for k in compact_only)
        finally:
            N.nopcs_destroy(ctx)
    assert np.array_equal(outs[0], outs[1])


def test_isothermal_rest_state_large():
    """128^3 isothermal quiescent box with gravity, mixed form: stays at rest."""
    N = binding()
    p = S.box_params((128, 128, 128), sub_n=(64, 64, 64), T_lower=1.0, perturb_amp=0.0)
    ctx = _ctx(N, p, N.NOPCS_MIXED)
    try:
        N.nopcs_rk_step(ctx, 4)
        d = N.nopcs_diagnostics(ctx, 0)
        assert d["max_speed"] < 1e-12 and d["nonfinite"] == 0
    finally:
        N.nopcs_destroy(ctx)


def test_mixed_128_against_oracle():
    """128^3 config-0 physics, mixed form vs the FP64 base-subtracted oracle."""
    N = binding()
    p = S.box_params((128, 128, 128), sub_n=(64, 64, 64), base_subtract=1, seed=2, filter_every=5)
    ctx = _ctx(N, p, N.NOPCS_MIXED)
    try:
        N.nopcs_rk_step(ctx, 10)
        Q = _state(N, ctx, p)
        orc = oracle.Solver(p)
        Q0 = orc.initial_state()
        ref = orc.step(Q0, 10)
        err = field_rel(Q, ref)
        dr = dist_rel(Q, ref, Q0)
        print("128^3 mixed, 10 steps, 2 filters: field-relative", err, "disturbance-relative", dr)
        assert np.all(err <= 1e-5), err
        assert np.all(dr <= MIXED_DIST_GATE), dr
    finally:
        N.nopcs_destroy(ctx)


def test_batched_uneven_boxes():
    """Several independent boxes of different shapes in one context advance
    exactly as they do alone."""
    N = binding()
    boxes = [S.box_params((24, 20, 30), sub_n=(8, 8, 8), seed=3),
             S.box_params((17, 33, 21), sub_n=(5, 16, 0), seed=4, T_lower=1.5)]
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


def test_set_get_state_host_roundtrip():
    N = binding()
    p = S.box_params((12, 13, 14))
    ctx = _ctx(N, p, N.NOPCS_FP64)
    try:
        q = np.random.default_rng(0).standard_normal((5, 14, 13, 12)) + 2.0
        N.nopcs_set_state(ctx, 0, q.ctypes.data)
        back = np.empty_like(q)
        N.nopcs_get_state(ctx, 0, back.ctypes.data)
        assert np.array_equal(q, back)
    finally:
        N.nopcs_destroy(ctx)


_CFG2 = {}


def _config2_reference(p):
    """(initial state, state after 200 steps) of the oracle, cached per box."""
    key = tuple(sorted((k, str(v)) for k, v in p.items()))
    if key not in _CFG2:
        orc = oracle.Solver(p)
        Q0 = orc.initial_state()
        _CFG2[key] = (Q0, orc.step(Q0, 200))
    return _CFG2[key]


@pytest.mark.parametrize("prec", [1, 0])
def test_config2_128_200_steps(prec):
    """The full-RK-step workload's parity case: 128^3 two-temperature box,
    200 RK4 steps (filter after steps 50, 100, 150, 200), base-subtracted
    formulation, FP64 oracle.  Mixed form <= 1e-5 field-relative; FP64 form
    <= 1e-12 (momentum relative to rho c)."""
    N = binding()
    p = S.box_params((128, 128, 128), sub_n=(64, 64, 64), base_subtract=1, seed=2)
    ctx = _ctx(N, p, prec)
    try:
        N.nopcs_rk_step(ctx, 200)
        Q = _state(N, ctx, p)
    finally:
        N.nopcs_destroy(ctx)
    Q0, ref = _config2_reference(p)
    fr = field_rel(Q, ref)
    dr = dist_rel(Q, ref, Q0)
    print("config2 prec", prec, "field-relative L-inf", fr, "disturbance-relative", dr, "L2",
          np.sqrt(((Q - ref) ** 2).reshape(5, -1).sum(1) / (ref ** 2).reshape(5, -1).sum(1)))
    if prec == 1:
        assert np.all(fr <= 1e-5), fr
        assert np.all(dr <= MIXED_DIST_GATE), dr
    else:
        err = state_err(Q, ref, p)
        assert np.all(err <= 1e-12), (err, fr)


def test_fp64_momentum_spread_is_roundoff():
    """FP64 form, 48^3, 50 steps: sizes of the momentum differences between
    runs that differ only in rounding -- the sub-domain split (GPU and oracle),
    the oracle source compiled with multiply-adds fused, the GPU against the
    oracle, and the GPU started from the oracle's own initial state (set
    through nopcs_set_state) against the oracle.  The momentum (1e-4 of rho c)
    is a small residual of O(1/(gamma M^2)) pressure terms, so its
    field-relative differences are large while all stay ~1e-15 of rho c, the
    gate's scale.  Reports the spreads field-relative and relative to rho c."""
    N = binding()
    outs, refs = {}, {}
    for sn in (24, 16):
        p = S.box_params((48, 48, 48), sub_n=(sn, sn, sn), base_subtract=0, seed=1)
        ctx = _ctx(N, p, N.NOPCS_FP64)
        try:
            N.nopcs_rk_step(ctx, 50)
            outs[sn] = _state(N, ctx, p)
        finally:
            N.nopcs_destroy(ctx)
        orc = oracle.Solver(p)
        refs[sn] = orc.step(orc.initial_state(), 50)
    p = S.box_params((48, 48, 48), sub_n=(24, 24, 24), base_subtract=0, seed=1)
    orc = oracle.Solver(p)
    Q0 = orc.initial_state()
    ctx = _ctx(N, p, N.NOPCS_FP64)
    try:
        Qg0 = _state(N, ctx, p)
        N.nopcs_set_state(ctx, 0, to_dev(Q0).data_ptr())
        N.nopcs_rk_step(ctx, 50)
        from_orc = _state(N, ctx, p)
    finally:
        N.nopcs_destroy(ctx)
    fused = oracle.Solver(p, contracted=True)
    ref_fused = fused.step(fused.initial_state(), 50)
    gpu_split = field_rel(outs[24], outs[16])[1:4].max()
    orc_split = field_rel(refs[24], refs[16])[1:4].max()
    orc_fused = field_rel(ref_fused, refs[24])[1:4].max()
    gpu_orc = max(field_rel(outs[24], refs[24])[1:4].max(), field_rel(outs[16], refs[16])[1:4].max())
    gpu_orc_same_init = field_rel(from_orc, refs[24])[1:4].max()
    init_gap = np.abs(Qg0 - Q0).max(axis=(1, 2, 3)) / np.abs(Q0).max(axis=(1, 2, 3))
    rc = [state_err(outs[24], refs[24], p)[1:4].max(), state_err(from_orc, refs[24], p)[1:4].max()]
    print("FP64 momentum spread, field-relative: GPU split 24 vs 16 %.2e, oracle split %.2e, oracle fused vs "
          "plain %.2e, GPU vs oracle %.2e, GPU from the oracle's initial state vs oracle %.2e; relative to rho c: "
          "%.2e, %.2e; initial-state gap per field %s" % (gpu_split, orc_split, orc_fused, gpu_orc,
                                                          gpu_orc_same_init, *rc, init_gap))
    assert max(rc) <= 1e-12
    # the initial state is not where the gap comes from: starting the GPU from
    # the oracle's own initial state leaves it within a factor of 2
    assert 0.5 * gpu_orc <= gpu_orc_same_init <= 2 * gpu_orc, (gpu_orc, gpu_orc_same_init)
