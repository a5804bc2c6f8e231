"""Known-answer pins of the counter-based SplitMix64 generator of the initial
velocity perturbation, against the generator's published test vector
(tests/golden/splitmix64_seed1234567.txt).  The oracle, the seeded input
module and the CUDA library each implement the generator from its published
definition; a constant mistyped the same way in two of them would still fail
here.  CPU only; the library's copy is checked in tests/test_gpu_rk.py with
the same seed shift."""
import os

import numpy as np

import nopcs_synth as S
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")
SEED = 1234567
GOLDEN_RATIO_64 = 0x9E3779B97F4A7C15


def published():
    with open(GOLDEN) as fh:
        return [int(l) for l in fh if l.strip() and not l.startswith("#")]


def shifted_seed(counter: int) -> int:
    """Seed s' with value number `counter` of stream s' equal to value 0 of the
    stream seeded with SEED: the state after c + 1 steps is s + (c + 1) * golden,
    so s' = SEED - counter * golden (mod 2^64)."""
    return (SEED - counter * GOLDEN_RATIO_64) % (1 << 64)


def expected_velocity(amp):
    """The five published values as the perturbation u, v, w of one node and
    u, v of the next: amp (2 U - 1), U = (z >> 11) 2^-53."""
    z = published()
    return [amp * (2.0 * ((v >> 11) * (1.0 / 2.0 ** 53)) - 1.0) for v in z]


def test_synth_generator_matches_published_vector():
    got = S.splitmix64(SEED, np.arange(5, dtype=np.uint64))
    assert [int(v) for v in got] == published()


def test_oracle_initial_state_draws_the_published_vector():
    n = (9, 8, 7)
    i, j, k = 3, 4, 2  # interior node, and its interior x-neighbour
    pidx = i + n[0] * (j + n[1] * k)
    amp = 1e-3
    p = S.box_params(n, perturb_amp=amp, seed=shifted_seed(3 * pidx))
    s = oracle.Solver(p)
    Q = s.initial_state()
    V0 = [Q[c + 1, k, j, i] / Q[0, k, j, i] for c in range(3)]
    V1 = [Q[c + 1, k, j, i + 1] / Q[0, k, j, i + 1] for c in range(2)]
    want = expected_velocity(amp)
    np.testing.assert_allclose(V0 + V1, want, rtol=1e-14, atol=0)
    # a different seed gives other values (the shift is what selects them)
    p2 = dict(p, seed=SEED)
    Q2 = oracle.Solver(p2).initial_state()
    assert abs(Q2[1, k, j, i] / Q2[0, k, j, i] - want[0]) > 1e-9
