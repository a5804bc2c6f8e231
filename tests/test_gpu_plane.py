"""Plane diagnostics of Sec. 4 through the C ABI (nopcs_plane_fields) against
the FP64 oracle, and the paper's front-speed check: the disturbance-pressure
pulses that leave the interface travel at the local sound speed sqrt(T)/M
(the slopes the paper reads off its (y, t) diagram)."""
import numpy as np
import pytest

import nopcs_synth as S
import oracle
from gpu_util import binding, stream_ptr, to_dev
from test_oracle_plane import _quadratic_state

pytestmark = pytest.mark.gpu


def _plane(N, ctx, p, axis, index, what):
    import torch
    n = p["n"]
    a, b = [d for d in range(3) if d != axis]
    out = torch.full((9 if what else 1, n[b], n[a]), float("nan"), dtype=torch.float64, device="cuda")
    N.nopcs_plane_fields(ctx, 0, axis, index, what, out.data_ptr())
    N.nopcs_synchronize(ctx)
    o = out.cpu().numpy()
    return o[0] if what == 0 else o


def _rel(a, b):
    """max |a - b| / max |b| per field ((nb, na) planes or (9, nb, na) stacks)."""
    a, b = np.asarray(a), np.asarray(b)
    if a.ndim == 2:
        a, b = a[None], b[None]
    a, b = a.reshape(a.shape[0], -1), b.reshape(b.shape[0], -1)
    return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)


def test_plane_fields_match_oracle_on_a_quadratic_state():
    N = binding()
    p = S.box_params((9, 8, 10), sub_n=(0, 0, 0), perturb_amp=0.0)
    ctx = N.nopcs_init([p], prec=N.NOPCS_FP64, stream=stream_ptr())
    try:
        Q, _, _ = _quadratic_state(p)
        N.nopcs_set_state(ctx, 0, to_dev(Q).data_ptr())
        orc = oracle.Solver(p)
        for axis in range(3):
            for index in (0, p["n"][axis] // 2, p["n"][axis] - 1):
                for what in (0, 1):
                    got = _plane(N, ctx, p, axis, index, what)
                    ref = orc.plane_fields(Q, axis, index, what)
                    assert np.all(_rel(got, ref) <= 1e-12), (axis, index, what)
    finally:
        N.nopcs_destroy(ctx)


def test_plane_fields_match_oracle_after_steps():
    """A perturbed state after five RK4 steps, both precisions' state.  The
    pressure gradients difference the O(1/(gamma M^2)) = 6e4 pressure over
    one cell, so the two sides' FP64 round-off in p (operation order, fused
    multiply-adds) reaches the baroclinic terms amplified by ~1/h: they are
    gated at 1e-12 of their maximum plus that round-off floor; the
    disturbance pressure at 1e-9 of its maximum, the other terms at 1e-12."""
    N = binding()
    for prec in (N.NOPCS_FP64, N.NOPCS_MIXED):
        p = S.box_params((20, 18, 24), sub_n=(8, 8, 8), perturb_amp=1e-3, base_subtract=1)
        ctx = N.nopcs_init([p], prec=prec, stream=stream_ptr())
        try:
            N.nopcs_rk_step(ctx, 5)
            import torch
            Qd = torch.empty((5, 24, 18, 20), dtype=torch.float64, device="cuda")
            N.nopcs_get_state(ctx, 0, Qd.data_ptr())
            Q = Qd.cpu().numpy()
            orc = oracle.Solver(p)
            # round-off floor of the baroclinic terms: a few ulps of p over one
            # cell, times the largest density gradient over rho^2
            h = p["len"][0] / (p["n"][0] - 1)
            rho = Q[0]
            grad_rho = max(np.abs(np.diff(rho, axis=k)).max() for k in range(3)) / h
            pmax = np.max(np.abs(Q[4])) * (p["gamma"] - 1)
            baro_floor = 16 * np.finfo(float).eps * pmax / h * grad_rho / rho.min() ** 2
            for axis, index in ((2, 12), (0, 0), (1, 9)):
                for what in (0, 1):
                    got = _plane(N, ctx, p, axis, index, what)
                    ref = orc.plane_fields(Q, axis, index, what)
                    err = _rel(got, ref)
                    if what == 0:
                        assert err[0] <= 1e-9, (prec, axis, index, err)
                    else:
                        assert np.all(err[:6] <= 1e-12), (prec, axis, index, err)
                        d = np.abs(got[6:] - ref[6:]).max()
                        assert d <= 1e-12 * np.abs(ref[6:]).max() + baro_floor, (prec, axis, index, d, baro_floor)
        finally:
            N.nopcs_destroy(ctx)


def test_bad_plane_requests():
    N = binding()
    p = S.box_params((9, 8, 10), sub_n=(0, 0, 0))
    ctx = N.nopcs_init([p], prec=N.NOPCS_FP64, stream=stream_ptr())
    try:
        import torch
        out = torch.empty(100, dtype=torch.float64, device="cuda")
        for args in ((3, 0, 0), (0, 9, 0), (0, -1, 0), (0, 0, 2)):
            with pytest.raises(N.NopcsError) as ei:
                N.nopcs_plane_fields(ctx, 0, *args, out.data_ptr())
            assert ei.value.status == N.NOPCS_EINVAL
    finally:
        N.nopcs_destroy(ctx)


def test_pressure_fronts_travel_at_the_local_sound_speed():
    """Unperturbed two-temperature box, h = 1/128, gravity along z: the
    leading disturbance-pressure peaks above and below the interface move at
    sqrt(T)/M of their side (T = 1 above, 5/3 below), within 5%."""
    N = binding()
    n = (33, 33, 129)
    p = S.box_params(n, sub_n=(0, 0, 64), length=(0.25, 0.25, 1.0), perturb_amp=0.0, base_subtract=1,
                     filter_every=50)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, stream=stream_ptr())
    try:
        h = 1.0 / 128
        z = np.arange(n[2]) * h
        upper, lower = z > 0.5 + 4 * h, z < 0.5 - 4 * h
        times, zu, zl = [], [], []
        steps_per_sample, samples = 150, 8
        for k in range(samples):
            N.nopcs_rk_step(ctx, steps_per_sample)
            prof = _plane(N, ctx, p, 0, n[0] // 2, 0)[:, n[1] // 2]  # p - p_h along z at the centre
            t = (k + 1) * steps_per_sample * p["dt"]

            def peak(mask):
                i = np.where(mask)[0]
                j = i[np.argmax(np.abs(prof[i]))]
                # parabolic refinement of the peak position
                y0, y1, y2 = np.abs(prof[j - 1]), np.abs(prof[j]), np.abs(prof[j + 1])
                den = y0 - 2 * y1 + y2
                return z[j] + (0.5 * (y0 - y2) / den * h if den != 0 else 0.0)

            times.append(t)
            zu.append(peak(upper))
            zl.append(peak(lower))
        t = np.array(times)
        su = np.polyfit(t[2:], np.array(zu)[2:], 1)[0]
        sl = -np.polyfit(t[2:], np.array(zl)[2:], 1)[0]
        au, al = np.sqrt(p["T_upper"]) / p["M"], np.sqrt(p["T_lower"]) / p["M"]
        print("front speeds %.1f (a = %.1f) above, %.1f (a = %.1f) below" % (su, au, sl, al))
        assert abs(su / au - 1) < 0.05 and abs(sl / al - 1) < 0.05, (su, au, sl, al)
    finally:
        N.nopcs_destroy(ctx)
