"""Pins of the oracle's plane diagnostics (Sec. 4; Eq. eqn12_1): the
disturbance pressure and the three right-hand-side terms of the inviscid
vorticity transport equation.  The gradients are second-order explicit
differences, exact for quadratic fields (central inside, one-sided on the
walls), so for quadratic rho, V and p every term has a closed form."""
import numpy as np
import pytest

import nopcs_synth as S
import oracle

GAMMA = 1.4


def _quadratic_state(p):
    n = p["n"]
    h = [p["len"][d] / (n[d] - 1) for d in range(3)]
    z, y, x = np.meshgrid(np.arange(n[2]) * h[2], np.arange(n[1]) * h[1], np.arange(n[0]) * h[0], indexing="ij")
    # quadratic fields and their exact gradients (d/dx, d/dy, d/dz)
    rho = 1.0 + 0.10 * x + 0.05 * y * y + 0.02 * z + 0.03 * x * z
    g_rho = [0.10 + 0.03 * z, 0.10 * y, 0.02 + 0.03 * x]
    u = 0.20 + 0.30 * y + 0.10 * z * z - 0.05 * x * y
    g_u = [-0.05 * y, 0.30 - 0.05 * x, 0.20 * z]
    v = -0.10 + 0.25 * x * x + 0.15 * z + 0.04 * y * z
    g_v = [0.50 * x, 0.04 * z, 0.15 + 0.04 * y]
    w = 0.05 + 0.12 * x * y - 0.08 * y + 0.06 * z * z
    g_w = [0.12 * y, 0.12 * x - 0.08, 0.12 * z]
    pr = 50.0 + 1.5 * x * x - 0.7 * y * z + 2.0 * z
    g_p = [3.0 * x, -0.7 * z, -0.7 * y + 2.0]
    Q = np.stack([rho, rho * u, rho * v, rho * w, pr / (GAMMA - 1) + 0.5 * rho * (u * u + v * v + w * w)])
    G = np.array([g_u, g_v, g_w])  # G[i][j] = dV_i/dx_j
    om = np.array([G[2][1] - G[1][2], G[0][2] - G[2][0], G[1][0] - G[0][1]])
    div = G[0][0] + G[1][1] + G[2][2]
    stretch = np.array([om[0] * G[i][0] + om[1] * G[i][1] + om[2] * G[i][2] for i in range(3)])
    dil = -om * div
    gr, gp = np.array(g_rho), np.array(g_p)
    baro = np.cross(gr, gp, axis=0) / rho ** 2
    return Q, np.concatenate([stretch, dil, baro]), pr


def _plane(f, axis, index):
    """(..., nz, ny, nx) -> the plane normal to axis, laid out (b, a), a fastest."""
    sl = [slice(None)] * f.ndim
    sl[f.ndim - 1 - axis] = index
    return f[tuple(sl)]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_vorticity_terms_exact_for_quadratic_fields(axis):
    p = S.box_params((9, 8, 10), perturb_amp=0.0)
    orc = oracle.Solver(p)
    Q, terms, _ = _quadratic_state(p)
    n = p["n"]
    for index in (0, n[axis] // 2, n[axis] - 1):  # both walls (one-sided) and the inside
        got = orc.plane_fields(Q, axis, index, 1)
        ref = _plane(terms, axis, index)
        scale = np.abs(terms).reshape(9, -1).max(axis=1)
        err = np.abs(got - ref).reshape(9, -1).max(axis=1) / scale
        assert np.all(err <= 1e-11), (index, err)


def test_vorticity_terms_fail_on_a_planted_sign_error():
    """The closed form separates the terms: a sign flip of the baroclinic
    cross product is far outside the tolerance."""
    p = S.box_params((9, 8, 10), perturb_amp=0.0)
    orc = oracle.Solver(p)
    Q, terms, _ = _quadratic_state(p)
    got = orc.plane_fields(Q, 2, 4, 1)
    ref = _plane(terms, 2, 4)
    assert np.max(np.abs(got[6:] + ref[6:])) > 1e-3 * np.max(np.abs(ref[6:]))
    assert np.max(np.abs(got[6:] - ref[6:])) <= 1e-11 * np.max(np.abs(ref[6:]))


def test_disturbance_pressure_plane():
    p = S.box_params((9, 8, 10), perturb_amp=0.0)
    orc = oracle.Solver(p)
    Q, _, pr = _quadratic_state(p)
    _, p_h = oracle.base_profile(p)
    for axis in range(3):
        got = orc.plane_fields(Q, axis, 3, 0)
        ref = _plane(pr - p_h[:, None, None], axis, 3)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(pr))
    # the hydrostatic initial state has no disturbance pressure
    Q0 = orc.initial_state()
    d = orc.plane_fields(Q0, 0, 4, 0)
    assert np.max(np.abs(d)) <= 1e-10 * np.max(p_h)


def test_plane_request_errors():
    p = S.box_params((9, 8, 10), perturb_amp=0.0)
    orc = oracle.Solver(p)
    Q = orc.initial_state()
    with pytest.raises(ValueError):
        orc.plane_fields(Q, 3, 0, 0)
    with pytest.raises(ValueError):
        orc.plane_fields(Q, 0, 9, 0)
