"""Failure behaviour and checkpoint/resume of the C ABI, made on the host:
a non-finite state written through nopcs_set_state, an allocation cap that
nopcs_init cannot meet, a run split at a checkpoint, a call from the wrong
device, and the library's initial state against the SplitMix64 published test
vector.  No test here faults, traps or hangs the GPU."""
import numpy as np
import pytest

import nopcs_synth as S
from gpu_util import binding, stream_ptr, to_dev
from test_splitmix64 import expected_velocity, shifted_seed

pytestmark = pytest.mark.gpu


def _state(N, ctx, p, box=0):
    import torch
    Q = torch.empty((5, p["n"][2], p["n"][1], p["n"][0]), dtype=torch.float64, device="cuda")
    N.nopcs_get_state(ctx, box, Q.data_ptr())
    return Q.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_state_is_reported_unstable(prec, bad):
    N = binding()
    p = S.box_params((20, 18, 22), sub_n=(8, 8, 8))
    ctx = N.nopcs_init([p], prec=prec, stream=stream_ptr())
    try:
        assert N.nopcs_diagnostics(ctx, 0)["nonfinite"] == 0
        Q = _state(N, ctx, p)
        Q[4, 11, 9, 7] = bad
        N.nopcs_set_state(ctx, 0, to_dev(Q).data_ptr())
        with pytest.raises(N.NopcsError) as ei:
            N.nopcs_diagnostics(ctx, 0)
        assert ei.value.status == N.NOPCS_EUNSTABLE
        d = N.nopcs_diagnostics(ctx, 0, allow_unstable=True)
        assert d["nonfinite"] == 1
        # the context stays usable: a finite state clears the flag
        Q[4, 11, 9, 7] = 1.0 / (p["gamma"] - 1) / (p["gamma"] * p["M"] ** 2)
        N.nopcs_set_state(ctx, 0, to_dev(Q).data_ptr())
        assert N.nopcs_diagnostics(ctx, 0)["nonfinite"] == 0
    finally:
        N.nopcs_destroy(ctx)


def _free_bytes():
    """Free device memory as the driver reports it, plus what torch's caching
    allocator holds (so tensors created and freed in between do not count)."""
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0] + torch.cuda.memory_reserved()


def test_memory_limit_gives_enomem_and_leaks_nothing():
    N = binding()
    p = S.box_params((96, 80, 72), sub_n=(32, 32, 32))
    # a first context runs every path the test takes, so that the modules
    # loaded on first launch and the driver's own pools are in place before
    # the baseline, whatever ran earlier in the process
    import torch
    c0 = N.nopcs_init([p], prec=N.NOPCS_MIXED, form=N.NOPCS_FORM_THOMAS, stream=stream_ptr())
    f0 = torch.zeros((72, 80, 96), dtype=torch.float32, device="cuda")
    o0 = torch.empty_like(f0)
    N.nopcs_derivative(c0, 0, 0, 1, 1, f0.data_ptr(), o0.data_ptr(), stream_ptr())
    N.nopcs_derivative(c0, 0, 0, 2, 1, f0.data_ptr(), o0.data_ptr(), stream_ptr())
    N.nopcs_rk_step(c0, 1)
    N.nopcs_synchronize(c0)
    N.nopcs_destroy(c0)
    del f0, o0
    free0 = _free_bytes()
    np_ = 96 * 80 * 72
    try:
        for limit in (1 << 20, 100 * np_):  # below the tables, below the registers (148 B/pt)
            N.nopcs_set_memory_limit(limit)
            with pytest.raises(N.NopcsError) as ei:
                N.nopcs_init([p], prec=N.NOPCS_MIXED, form=N.NOPCS_FORM_THOMAS, stream=stream_ptr())
            assert ei.value.status == N.NOPCS_ENOMEM, str(ei.value)
            assert _free_bytes() == free0
        # enough for the context, not for the order-2 scratch (8 B/pt)
        N.nopcs_set_memory_limit(155 * np_)
        ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, form=N.NOPCS_FORM_THOMAS, stream=stream_ptr())
        try:
            import torch
            f = torch.zeros((72, 80, 96), dtype=torch.float32, device="cuda")
            out = torch.empty_like(f)
            N.nopcs_derivative(ctx, 0, 0, 1, 1, f.data_ptr(), out.data_ptr(), stream_ptr())
            with pytest.raises(N.NopcsError) as ei:
                N.nopcs_derivative(ctx, 0, 0, 2, 1, f.data_ptr(), out.data_ptr(), stream_ptr())
            assert ei.value.status == N.NOPCS_ENOMEM
            N.nopcs_rk_step(ctx, 1)  # still usable
            N.nopcs_synchronize(ctx)
            del f, out
        finally:
            N.nopcs_destroy(ctx)
    finally:
        N.nopcs_set_memory_limit(0)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED, form=N.NOPCS_FORM_THOMAS, stream=stream_ptr())
    N.nopcs_destroy(ctx)
    assert _free_bytes() == free0


@pytest.mark.parametrize("prec", [0, 1])
def test_checkpoint_resume_is_bitwise(prec):
    """k + m steps in one run equal k steps, a checkpoint (state and step
    counter), a fresh context restored from it, and m more steps: bit for bit,
    with the filter firing inside both halves."""
    N = binding()
    p = S.box_params((30, 28, 26), sub_n=(12, 12, 12), filter_every=3, perturb_amp=1e-3, seed=8)
    k, m = 4, 5
    ctx = N.nopcs_init([p], prec=prec, stream=stream_ptr())
    try:
        N.nopcs_rk_step(ctx, k)
        Qk = _state(N, ctx, p)
        step_k = N.nopcs_diagnostics(ctx, 0)["step"]
        N.nopcs_rk_step(ctx, m)
        Qa = _state(N, ctx, p)
    finally:
        N.nopcs_destroy(ctx)
    assert step_k == k
    ctx = N.nopcs_init([p], prec=prec, stream=stream_ptr())
    try:
        N.nopcs_set_state(ctx, 0, to_dev(Qk).data_ptr())
        N.nopcs_set_step(ctx, 0, step_k)
        N.nopcs_rk_step(ctx, m)
        Qb = _state(N, ctx, p)
        assert N.nopcs_diagnostics(ctx, 0)["step"] == k + m
    finally:
        N.nopcs_destroy(ctx)
    assert np.array_equal(Qa, Qb)
    assert not np.array_equal(Qa, Qk)


def test_calls_from_another_device_are_rejected():
    import torch
    N = binding()
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    p = S.box_params((16, 16, 16), sub_n=(8, 8, 8))
    torch.cuda.set_device(0)
    ctx = N.nopcs_init([p], prec=N.NOPCS_MIXED)
    try:
        torch.cuda.set_device(1)
        with pytest.raises(N.NopcsError) as ei:
            N.nopcs_rk_step(ctx, 1)
        assert ei.value.status == N.NOPCS_EINVAL and "device" in str(ei.value)
    finally:
        N.nopcs_destroy(ctx)  # frees on device 0 and switches back
        assert torch.cuda.current_device() == 1
        torch.cuda.set_device(0)


def test_initial_state_draws_the_published_splitmix_vector():
    """The library's generator against the SplitMix64 published test vector:
    with the seed shifted so that node p draws values 0..4 of the stream seeded
    with 1234567, node p's u, v, w and node p+1's u, v are those values."""
    N = binding()
    n = (9, 8, 7)
    i, j, k = 3, 4, 2
    pidx = i + n[0] * (j + n[1] * k)
    amp = 1e-3
    p = S.box_params(n, sub_n=(0, 0, 0), perturb_amp=amp, seed=shifted_seed(3 * pidx))
    ctx = N.nopcs_init([p], prec=N.NOPCS_FP64, stream=stream_ptr())
    try:
        Q = _state(N, ctx, p)
    finally:
        N.nopcs_destroy(ctx)
    V = [Q[c + 1, k, j, i] / Q[0, k, j, i] for c in range(3)] + \
        [Q[c + 1, k, j, i + 1] / Q[0, k, j, i + 1] for c in range(2)]
    np.testing.assert_allclose(V, expected_velocity(amp), rtol=1e-14, atol=0)


@pytest.mark.parametrize("prec", [0, 1])
def test_staged_state_equals_set_state(prec):
    """nopcs_stage_state + nopcs_commit_state give the state nopcs_set_state
    gives, bit for bit, from pinned host memory: a state staged while a step
    runs does not reach that step, and becomes current only at its commit."""
    import torch
    N = binding()
    p = S.box_params((30, 28, 26), sub_n=(12, 12, 12), perturb_amp=1e-3, seed=9)
    ctx = N.nopcs_init([p], prec=prec, stream=stream_ptr())
    try:
        N.nopcs_rk_step(ctx, 2)
        QA = _state(N, ctx, p)
        N.nopcs_rk_step(ctx, 3)
        QB = _state(N, ctx, p)
        hA = torch.from_numpy(QA.copy()).pin_memory()
        hB = torch.from_numpy(QB.copy()).pin_memory()
        # reference: set_state(A), one step
        N.nopcs_set_state(ctx, 0, hA.data_ptr())
        N.nopcs_rk_step(ctx, 1)
        ref1 = _state(N, ctx, p)
        # staged: A staged and committed; B staged while the step on A runs
        N.nopcs_stage_state(ctx, 0, hA.data_ptr())
        N.nopcs_commit_state(ctx, 0)
        N.nopcs_stage_state(ctx, 0, hB.data_ptr())
        N.nopcs_rk_step(ctx, 1)
        got1 = _state(N, ctx, p)
        N.nopcs_commit_state(ctx, 0)
        gotB = _state(N, ctx, p)
        # a commit needs a staged state
        with pytest.raises(N.NopcsError) as ei:
            N.nopcs_commit_state(ctx, 0)
        assert ei.value.status == N.NOPCS_EINVAL
        with pytest.raises(N.NopcsError) as ei:
            N.nopcs_stage_state(ctx, 0, 0)
        assert ei.value.status == N.NOPCS_EINVAL
        # the derived fields were refreshed too: stepping from the committed B
        # equals stepping from set_state(B)
        N.nopcs_rk_step(ctx, 1)
        gotB1 = _state(N, ctx, p)
        N.nopcs_set_state(ctx, 0, hB.data_ptr())
        N.nopcs_rk_step(ctx, 1)
        refB1 = _state(N, ctx, p)
    finally:
        N.nopcs_destroy(ctx)
    assert np.array_equal(got1, ref1)
    assert np.array_equal(gotB, QB)
    assert np.array_equal(gotB1, refB1)
    assert not np.array_equal(ref1, QA)


def test_split_state_copies_are_exact():
    """States of 64 MB and more cross the host link in four parts on four
    streams: set_state and stage + commit of an 84 MB state (128^3) from pinned
    host memory give back exactly the state that was sent."""
    import torch
    N = binding()
    n = 128
    p = S.box_params((n, n, n), sub_n=(64, 64, 64), perturb_amp=1e-3, seed=21)
    ctx = N.nopcs_init([p], prec=N.NOPCS_FP64, stream=stream_ptr())
    try:
        Q = _state(N, ctx, p)
        g = np.random.default_rng(3)
        send = torch.from_numpy(Q * (1.0 + 1e-6 * g.standard_normal(Q.shape))).pin_memory()
        assert send.numel() * 8 >= 64 << 20
        N.nopcs_set_state(ctx, 0, send.data_ptr())
        back1 = _state(N, ctx, p)
        N.nopcs_reset_state(ctx, 0)
        N.nopcs_stage_state(ctx, 0, send.data_ptr())
        N.nopcs_commit_state(ctx, 0)
        back2 = _state(N, ctx, p)
    finally:
        N.nopcs_destroy(ctx)
    ref = send.numpy()
    assert np.array_equal(back1, ref)
    assert np.array_equal(back2, ref)
    assert not np.array_equal(ref, Q)
