"""Pins of the oracle's one-dimensional operators against what the paper and the
mathematics fix (arXiv 2203.00879, Sec. 3 and Appendix).  CPU only."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oucs3_equivalent_explicit_row.txt")
ALPHA, B1, B2, BETA = oracle.OUCS3


def _appendix():
    d = np.loadtxt(GOLDEN)
    return d[:, 0].astype(int), d[:, 1]


def test_appendix_equivalent_explicit_row():
    """Interior row of C = A^-1 B equals the Appendix table (97 values)."""
    k, c = _appendix()
    assert list(k) == list(range(-48, 49))
    op = oracle.Op(301)
    _, Cm = op.matrices()
    i = 150
    got = Cm[i, i + k]
    assert np.max(np.abs(got - c)) < 2e-16
    # semi-bandwidth n_b = 48: the next coefficient is below 1e-16 (Sec. 3)
    assert abs(Cm[i, i + 49]) < 1e-16 and abs(Cm[i, i - 49]) < 1e-16
    assert abs(Cm[i, i + 48]) >= 1e-16


def test_appendix_row_rejects_planted_sign_error():
    """A plausible transcription mistake (sign of the b2 term) breaks the pin."""
    k, c = _appendix()
    op = oracle.Op(301, coef=(ALPHA, B1, -B2, BETA))
    _, Cm = op.matrices()
    assert np.max(np.abs(Cm[150, 150 + k] - c)) > 1e-3


def test_consistency_of_printed_coefficients():
    """Antisymmetric B with the printed magnitudes is consistent: 2 b1 + 4 b2 = 1 + 2 alpha."""
    assert abs(2 * B1 + 4 * B2 - (1 + 2 * ALPHA)) < 1e-15


@pytest.mark.parametrize("kh", [0.1, 0.5, 1.0, 1.7, 2.392, 2.9])
@pytest.mark.parametrize("sub_n", [0, 24, 64])
def test_modified_wavenumber_closed_form(kh, sub_n):
    """Sine waves are eigenfunctions of the interior scheme:
    k_eq h = (2 b1 sin kh + 2 b2 sin 2kh) / (1 + 2 alpha cos kh)."""
    N, h = 257, 0.01
    x = np.arange(N) * h
    k = kh / h
    f = np.sin(k * x + 0.3)
    op = oracle.Op(N, sub_n=sub_n)
    d = op.nopcs(f, 1.0 / h)
    keq = (2 * B1 * np.sin(kh) + 2 * B2 * np.sin(2 * kh)) / (1 + 2 * ALPHA * np.cos(kh))
    exact = keq / h * np.cos(k * x + 0.3)
    inner = slice(80, N - 80)  # wall closures decay like 0.46^distance
    assert np.max(np.abs(d[inner] - exact[inner])) < 1e-13 * max(1.0, keq / h)


def test_modified_wavenumber_peak():
    """max k_eq h = 2.209 at kh = 2.392 (spectral resolution of OUCS3)."""
    N, h = 257, 1.0
    best = (0, 0)
    for kh in np.linspace(2.2, 2.6, 81):
        x = np.arange(N)
        d = oracle.Op(N).nopcs(np.sin(kh * x))
        # amplitude of the interior response
        c = np.cos(kh * x)[100:150]
        amp = float(np.dot(d[100:150], c) / np.dot(c, c))
        if amp > best[0]:
            best = (amp, kh)
    assert abs(best[0] - 2.209) < 2e-3 and abs(best[1] - 2.392) < 0.01


@pytest.mark.parametrize("N", [5, 6, 7, 9, 13, 24, 37, 48, 101])
@pytest.mark.parametrize("sub_n", [3, 4, 5, 8, 24, 0])
def test_global_system_residual(N, sub_n):
    """NOHAP result solves the global system [A]{f'} = [B]{f} to machine
    precision for any sub-domain split (Sec. 3: no parallelisation error)."""
    rng = np.random.default_rng(N * 100 + sub_n)
    f = rng.standard_normal(N)
    op = oracle.Op(N, sub_n=sub_n)
    B, _ = op.matrices()
    g = op.nopcs(f)
    Bf = B @ f
    res = np.zeros(N)
    for i in range(N):
        if i < 2 or i > N - 3:
            res[i] = g[i] - Bf[i]
        else:
            res[i] = ALPHA * g[i - 1] + g[i] + ALPHA * g[i + 1] - Bf[i]
    assert np.max(np.abs(res)) < 2e-14 * max(1.0, np.max(np.abs(Bf)))


@pytest.mark.parametrize("N", [48, 101, 257])
def test_subdomain_independence(N):
    """Results do not depend on the number of sub-domains (Sec. 3)."""
    rng = np.random.default_rng(N)
    f = rng.standard_normal(N)
    ref = oracle.Op(N).dense(f)
    for sub_n in (3, 5, 8, 24, 64, N):
        g = oracle.Op(N, sub_n=sub_n).nopcs(f)
        assert np.max(np.abs(g - ref)) < 1e-14 * np.max(np.abs(ref))


def test_truncated_fp32_rows_error_bound():
    """Dropping |C| < 1e-8 (24 taps each side) changes results by < 1e-8 relative."""
    N = 257
    rng = np.random.default_rng(3)
    f = rng.standard_normal(N)
    ref = oracle.Op(N).dense(f)
    g = oracle.Op(N, sub_n=32, thresh=1e-8).nopcs(f)
    assert np.max(np.abs(g - ref)) < 1e-8 * np.max(np.abs(f))


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_exact_for_quadratics(deg):
    """Interior OUCS3 rows and the wall closures are exact for polynomials up to
    degree 2, so the whole operator differentiates them exactly."""
    N, h = 41, 0.05
    x = np.arange(N) * h - 0.3
    f = x ** deg
    fp = deg * x ** (deg - 1) if deg else np.zeros(N)
    for sub_n in (0, 7, 16):
        d = oracle.Op(N, sub_n=sub_n).nopcs(f, 1.0 / h)
        assert np.max(np.abs(d - fp)) < 1e-12


def test_near_wall_row_exact_for_cubics():
    """The beta-family closure next to the wall is fourth-order: exact for cubics."""
    N, h = 21, 0.1
    x = np.arange(N) * h
    B, _ = oracle.Op(N).matrices()
    for deg in range(4):
        f = x ** deg
        fp = deg * x ** (deg - 1) if deg else np.zeros(N)
        assert abs(B[1] @ f / h - fp[1]) < 1e-11
        assert abs(B[N - 2] @ f / h - fp[N - 2]) < 1e-11


def test_convergence_order():
    """Max-norm error of the derivative of a smooth function falls at least like h^2."""
    errs = []
    for N in (33, 65, 129, 257):
        h = 1.0 / (N - 1)
        x = np.arange(N) * h
        f = np.sin(3.0 * x + 0.2) + np.cos(5.0 * x)
        fp = 3 * np.cos(3.0 * x + 0.2) - 5 * np.sin(5.0 * x)
        d = oracle.Op(N, sub_n=16).nopcs(f, 1.0 / h)
        errs.append(np.max(np.abs(d - fp)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9), rates


def test_partition_rule():
    st = oracle.partition(48, 24)
    assert list(st) == [0, 24, 48]
    assert list(oracle.partition(50, 24)) == [0, 24, 50]   # remainder 2 joins
    assert list(oracle.partition(51, 24)) == [0, 24, 48, 51]  # remainder 3 stands
    assert list(oracle.partition(10, 64)) == [0, 10]
    assert list(oracle.partition(1024, 64)) == list(range(0, 1025, 64))


# ----------------------------------------------------------------------------- filter

def _filter_response(theta, N=257):
    x = np.arange(N)
    f = np.cos(theta * x)
    g = oracle.Op(N, kind=oracle.FILTER, sub_n=32).nopcs(f)
    c = f[100:160]
    return float(np.dot(g[100:160], c) / np.dot(c, c)), g, f


def test_filter_transfer_properties():
    """The 6th-order tridiagonal filter with alpha_f = 0.135 keeps constants,
    removes the odd-even mode, and 1 - T(kh) = O((kh)^6); those three facts fix
    its four right-hand-side coefficients."""
    t0, g, f = _filter_response(0.0)
    assert abs(t0 - 1.0) < 1e-14
    tpi, g, f = _filter_response(np.pi)
    assert abs(tpi) < 1e-14
    d1 = 1 - _filter_response(0.2)[0]
    d2 = 1 - _filter_response(0.1)[0]
    rate = np.log2(d1 / d2)
    assert 5.8 < rate < 6.2, rate
    # response at kh = pi/2 is strictly between 0 and 1 (low-pass)
    tm = _filter_response(np.pi / 2)[0]
    assert 0.5 < tm < 1.0


def test_filter_walls_untouched_and_subdomain_independent():
    N = 97
    rng = np.random.default_rng(5)
    f = rng.standard_normal(N)
    ref = oracle.Op(N, kind=oracle.FILTER).dense(f)
    assert np.all(ref[:3] == f[:3]) and np.all(ref[-3:] == f[-3:])
    for sub_n in (4, 9, 24, 50):
        g = oracle.Op(N, kind=oracle.FILTER, sub_n=sub_n).nopcs(f)
        assert np.max(np.abs(g - ref)) < 1e-14 * np.max(np.abs(ref))


def test_axis_application_matches_lines():
    """The 3-D driver applies the line operator along the requested axis."""
    rng = np.random.default_rng(9)
    f = rng.standard_normal((7, 9, 11))  # (nz, ny, nx)
    h = 0.1
    for axis, N in ((0, 11), (1, 9), (2, 7)):
        d = oracle.deriv3d(f, axis, h, sub_n=4)
        op = oracle.Op(N, sub_n=4)
        line = np.moveaxis(f, 2 - axis, -1)[3, 2]
        got = np.moveaxis(d, 2 - axis, -1)[3, 2]
        assert np.max(np.abs(got - op.nopcs(line, 1 / h))) < 1e-14


def test_explicit_second_order_operator():
    """2nd-order explicit derivative: exact for quadratics, order 2."""
    x = np.arange(12) * 0.1
    f = np.broadcast_to(x ** 2, (3, 4, 12)).copy()
    d = oracle.explicit2(f, 0, 0.1)
    assert np.max(np.abs(d - 2 * x)) < 1e-12


# ---- the compact second derivative (Lele's sixth-order tridiagonal scheme) ----

def test_d2_coefficients_are_consistent():
    """The Taylor conditions of the tridiagonal second-derivative family at
    orders 2, 4 and 6: a + b = 1 + 2 alpha, a + 4b = 12 alpha, a + 16b = 30 alpha."""
    al, a, b = oracle.LELE_D2
    assert abs((a + b) - (1 + 2 * al)) < 1e-15
    assert abs((a + 4 * b) - 12 * al) < 1e-14
    assert abs((a + 16 * b) - 30 * al) < 1e-14


@pytest.mark.parametrize("sub_n", [0, 3, 5, 8])
def test_d2_exact_for_cubics(sub_n):
    N = 30
    x = np.linspace(0.0, 1.0, N)
    h = x[1] - x[0]
    f = 1 + 2 * x - 3 * x ** 2 + 0.7 * x ** 3
    g = oracle.Op(N, kind=oracle.D2, sub_n=sub_n).nopcs(f) / h ** 2
    assert np.max(np.abs(g - (-6 + 4.2 * x))) < 1e-11


def test_d2_modified_wavenumber_in_the_interior():
    """Away from the walls sin(kx) gets -k_eq^2 sin(kx) with
    k_eq^2 h^2 = [2a (1 - cos kh) + (b/2)(1 - cos 2kh)] / (1 + 2 alpha cos kh)."""
    al, a, b = oracle.LELE_D2
    N = 200
    x = np.arange(N) * 1.0
    for kh in (0.3, 1.0, 2.0, 2.9):
        f = np.sin(kh * x + 0.4)
        g = oracle.Op(N, kind=oracle.D2, sub_n=0).nopcs(f)
        keq2 = (2 * a * (1 - np.cos(kh)) + 0.5 * b * (1 - np.cos(2 * kh))) / (1 + 2 * al * np.cos(kh))
        i = slice(40, N - 40)
        assert np.max(np.abs(g[i] + keq2 * f[i])) < 1e-12


def test_d2_sixth_order_in_the_interior():
    errs = []
    for N in (41, 81):
        x = np.linspace(0, 1, N)
        h = x[1] - x[0]
        f = np.sin(2 * np.pi * x + 0.3)
        g = oracle.Op(N, kind=oracle.D2, sub_n=0).nopcs(f) / h ** 2
        c = N // 2
        errs.append(abs(g[c] + (2 * np.pi) ** 2 * f[c]))
    assert 50 < errs[0] / errs[1] < 80  # 2^6 = 64


def test_d2_subdomain_independence():
    N = 61
    rng = np.random.default_rng(5)
    f = np.cumsum(rng.standard_normal(N)) * 0.1
    ref = oracle.Op(N, kind=oracle.D2, sub_n=0).dense(f)
    for sub_n in (3, 5, 8, 24, 0):
        g = oracle.Op(N, kind=oracle.D2, sub_n=sub_n).nopcs(f)
        assert np.max(np.abs(g - ref)) <= 1e-13 * np.max(np.abs(ref))
