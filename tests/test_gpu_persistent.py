"""One persistent kernel per RK step for all boxes of a context
(nopcs_set_launch): it runs the same device code as the per-box CUDA graph
with the same launch geometry and matches the graph and the oracle; its
bounded waits give up, return and leave the context usable when a dependency
is withheld (no fault, no hang)."""
import numpy as np
import pytest

import nopcs_synth as S
from gpu_util import binding, stream_ptr

pytestmark = pytest.mark.gpu


def _boxes():
    return [S.box_params((24, 20, 30), sub_n=(8, 8, 8), seed=3, filter_every=2),
            S.box_params((17, 33, 21), sub_n=(5, 16, 0), seed=4, T_lower=1.5, filter_every=2),
            S.box_params((96, 64, 128), sub_n=(32, 32, 64), seed=5, T_lower=1.4, perturb_amp=1e-4),
            S.box_params((40, 40, 72), sub_n=(-1, -1, -1), seed=6)]


def _states(N, ctx, boxes):
    import torch
    out = []
    for b, p in enumerate(boxes):
        Q = torch.empty((5, p["n"][2], p["n"][1], p["n"][0]), dtype=torch.float64, device="cuda")
        N.nopcs_get_state(ctx, b, Q.data_ptr())
        out.append(Q.cpu().numpy())
    return out


def _run(N, boxes, mode, steps):
    ctx = N.nopcs_init(boxes, prec=N.NOPCS_MIXED, stream=stream_ptr())
    try:
        if mode is not None:
            N.nopcs_set_launch(ctx, mode)
        N.nopcs_rk_step(ctx, steps)
        N.nopcs_synchronize(ctx)
        return _states(N, ctx, boxes)
    finally:
        N.nopcs_destroy(ctx)


def _interior_visc_tiles(n):
    """True if some 32 x 8 viscous tile of an n box lies off the x and y walls
    (the tile placement of the stage kernel)."""
    for x0 in range(0, n[0], 32):
        x0 = min(x0, max(n[0] - 32, 0))
        for y0 in range(0, n[1], 8):
            y0 = min(y0, max(n[1] - 8, 0))
            if x0 - 1 > 0 and x0 + 32 < n[0] - 1 and y0 - 1 > 0 and y0 + 8 < n[1] - 1:
                return True
    return False


def test_persistent_step_equals_graph():
    """Every box against the per-box graph: identical bits where all viscous
    tiles touch an x or y wall; where some lie in the interior the compiler
    rounds one of their approximate FP32 operations (reciprocal square root
    or fast division) differently inside the persistent kernel, and the two
    agree to FP32 rounding.  Every box against the FP64 oracle within the
    mixed-form gates."""
    import oracle
    from gpu_util import dist_rel, field_rel
    N = binding()
    boxes = _boxes()
    ref = _run(N, boxes, None, 5)
    got = _run(N, boxes, N.NOPCS_LAUNCH_PERSISTENT, 5)
    for b, p in enumerate(boxes):
        if _interior_visc_tiles(p["n"]):
            fr = field_rel(got[b], ref[b])
            print("box", p["n"], "persistent vs graph, field-relative", fr)
            assert np.all(fr <= 1e-8), (b, fr)
        else:
            assert np.array_equal(got[b], ref[b]), b
        assert not np.array_equal(got[b][1:4], 0 * got[b][1:4])
        if p["sub_n"][0] >= 0:
            pb = dict(p, base_subtract=1)
            orc = oracle.Solver(pb)
            Q0 = orc.initial_state()
            want = orc.step(Q0, 5)
            assert np.all(field_rel(got[b], want) <= 1e-5)
            assert np.all(dist_rel(got[b], want, Q0) <= 2e-5), (b, dist_rel(got[b], want, Q0))
    assert any(_interior_visc_tiles(p["n"]) for p in boxes)
    assert any(not _interior_visc_tiles(p["n"]) for p in boxes)


def test_persistent_wait_gives_up_and_context_recovers():
    N = binding()
    boxes = _boxes()[:2]
    ctx = N.nopcs_init(boxes, prec=N.NOPCS_MIXED, stream=stream_ptr())
    try:
        N.nopcs_set_launch(ctx, N.NOPCS_LAUNCH_PERSISTENT_WITHHOLD, 0.05)
        N.nopcs_rk_step(ctx, 1)
        with pytest.raises(N.NopcsError) as ei:
            N.nopcs_synchronize(ctx)
        assert ei.value.status == N.NOPCS_ETIMEOUT and "persistent" in str(ei.value)
        N.nopcs_synchronize(ctx)  # the error word was cleared
        # usable again: reset the states, step normally, match the graph
        N.nopcs_set_launch(ctx, N.NOPCS_LAUNCH_PERSISTENT, 2.0)
        for b in range(len(boxes)):
            N.nopcs_reset_state(ctx, b)
        N.nopcs_rk_step(ctx, 3)
        N.nopcs_synchronize(ctx)
        got = _states(N, ctx, boxes)
    finally:
        N.nopcs_destroy(ctx)
    ref = _run(N, boxes, None, 3)
    for b in range(len(boxes)):
        assert np.array_equal(got[b], ref[b]), b


def test_persistent_rejects_unsupported_boxes():
    N = binding()
    p = S.box_params((16, 16, 16), sub_n=(8, 8, 8))
    ctx = N.nopcs_init([p], prec=N.NOPCS_FP64, stream=stream_ptr())
    try:
        with pytest.raises(N.NopcsError) as ei:
            N.nopcs_set_launch(ctx, N.NOPCS_LAUNCH_PERSISTENT)
        assert ei.value.status == N.NOPCS_EUNSUPPORTED
        with pytest.raises(N.NopcsError) as ei:
            N.nopcs_set_launch(ctx, 7)
        assert ei.value.status == N.NOPCS_EINVAL
    finally:
        N.nopcs_destroy(ctx)
