"""The C-ABI library loads, exports every symbol include/nopcs.h declares, and its
host-side logic (argument checks, NOHAP operator tables) is right.  No GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nopcs.h")


@pytest.fixture(scope="module")
def N():
    from paper_2203_00879_gb300 import build
    build.build()
    from paper_2203_00879_gb300 import nopcs
    return nopcs


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nopcs_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_four_entry_points():
    names = declared_functions()
    for n in ("nopcs_init", "nopcs_derivative", "nopcs_rk_step", "nopcs_diagnostics"):
        assert n in names


def test_library_exports_every_declared_symbol(N):
    lib = ctypes.CDLL(N.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_same_names(N):
    for n in declared_functions():
        assert hasattr(N, n), n


def test_init_rejects_bad_arguments_before_device_work(N):
    import nopcs_synth as S
    good = S.box_params((8, 8, 8))
    cases = [dict(good, n=(4, 8, 8)), dict(good, sub_n=(2, 8, 8)), dict(good, gravity_axis=3),
             dict(good, dt=0.0), dict(good, gamma=1.0), dict(good, filter_every=-1)]
    for c in cases:
        with pytest.raises(N.NopcsError) as ei:
            N.nopcs_init([c])
        assert ei.value.status == N.NOPCS_EINVAL
    with pytest.raises(N.NopcsError):
        N.nopcs_init([good], prec=7)
    for form in (-1, N.NOPCS_FORM_BANDED + 1):
        with pytest.raises(N.NopcsError) as ei:
            N.nopcs_init([good], form=form)
        assert ei.value.status == N.NOPCS_EINVAL
    with pytest.raises(N.NopcsError) as ei:
        N.nopcs_init([dict(good, visc_compact=2)])
    assert ei.value.status == N.NOPCS_EINVAL


def test_kernel_names(N):
    names = [N.nopcs_kernel_name(k) for k in range(N.NOPCS_NUM_KERNELS)]
    assert all(names) and len(set(names)) == len(names)
    assert N.nopcs_kernel_name(N.NOPCS_NUM_KERNELS) is None


@pytest.mark.parametrize("Nn,sub_n", [(5, 3), (7, 3), (48, 24), (50, 24), (101, 24), (257, 64), (129, 0)])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_operator_tables_match_oracle(N, Nn, sub_n, kind):
    """The library's end rows (C = A^-1 B via transposed tridiagonal solves)
    equal the oracle's dense C rows, and everything dropped is below 1e-16."""
    starts, rows = N.nopcs_operator_rows(Nn, sub_n, kind=kind, alpha_f=0.135, thresh=1e-16)
    assert list(starts) == list(oracle.partition(Nn, sub_n))
    op = oracle.Op(Nn, kind=kind, sub_n=sub_n)
    _, Cm = op.matrices()
    for b in range(len(starts) - 1):
        for which, i in ((0, starts[b]), (1, starts[b + 1] - 1)):
            j0, c = rows[2 * b + which]
            if which == 1 and starts[b + 1] - 1 == starts[b]:
                continue
            c = np.array(c)
            assert np.max(np.abs(c - Cm[i, j0:j0 + len(c)])) < 1e-15
            rest = np.ones(Nn, bool)
            rest[j0:j0 + len(c)] = False
            assert np.all(np.abs(Cm[i][rest]) < 1e-16)


def test_fp32_tables_have_24_taps_each_side(N):
    starts, rows = N.nopcs_operator_rows(1024, 64, kind=0, thresh=1e-8)
    j0, c = rows[2 * 8]  # start of a sub-domain far from both walls
    assert starts[8] == 512 and j0 == 512 - 24 and len(c) == 49
    k = np.loadtxt(os.path.join(ROOT, "tests", "golden", "oucs3_equivalent_explicit_row.txt"))
    ref = k[24:73, 1]
    assert np.max(np.abs(np.array(c) - ref)) < 2e-16


@pytest.mark.parametrize("Nn,sub_n", [(5, 3), (9, 4), (48, 24), (50, 24), (101, 24), (257, 64), (129, 0)])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_host_line_algorithm_matches_oracle(N, Nn, sub_n, kind):
    """The library's own FP64 line algorithm (end rows, tabulated Thomas
    factors) equals the oracle's NOHAP evaluation."""
    rng = np.random.default_rng(Nn + 7 * sub_n + kind)
    f = rng.standard_normal(Nn)
    g = N.nopcs_operator_apply(Nn, sub_n, f, kind=kind)
    ref = oracle.Op(Nn, kind=kind, sub_n=sub_n).nopcs(f)
    assert np.max(np.abs(g - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("Nn", [5, 9, 40, 64, 129, 512])
@pytest.mark.parametrize("kind,thresh", [(0, 1e-16), (0, 1e-8), (1, 1e-16)])
def test_band_form_matches_oracle(N, Nn, kind, thresh):
    """The banded explicit form (every row from the truncated global C) equals
    the oracle's NOHAP evaluation to within the truncation."""
    rng = np.random.default_rng(Nn + kind)
    f = rng.standard_normal(Nn)
    g, h, lo, hi = N.nopcs_band_apply(Nn, f, kind=kind, thresh=thresh)
    ref = oracle.Op(Nn, kind=kind, sub_n=0).nopcs(f)
    tol = 1e-14 if thresh < 1e-12 else 2e-7
    assert np.max(np.abs(g - ref)) <= tol * max(1.0, np.max(np.abs(ref)))
    if Nn >= 129:
        # one interior stencil for all rows away from the walls
        assert lo <= 60 and hi >= Nn - 61 and h == (24 if thresh == 1e-8 else h)


def test_band_fp32_stencil_is_the_appendix_row(N):
    """The interior stencil at the FP32 threshold is the printed equivalent
    explicit row (Appendix table), 24 taps each side."""
    Nn = 256
    f = np.zeros(Nn)
    k = np.loadtxt(os.path.join(ROOT, "tests", "golden", "oucs3_equivalent_explicit_row.txt"))
    _, h, lo, hi = N.nopcs_band_apply(Nn, f, kind=0, thresh=1e-8)
    assert h == 24
    # apply to unit vectors at an interior row to read the stencil back
    i = Nn // 2
    taps = []
    for j in range(i - h, i + h + 1):
        e = np.zeros(Nn)
        e[j] = 1.0
        taps.append(N.nopcs_band_apply(Nn, e, kind=0, thresh=1e-8)[0][i])
    assert np.max(np.abs(np.array(taps) - k[24:73, 1])) < 2e-16
