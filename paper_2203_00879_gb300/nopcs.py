"""ctypes binding of libnopcs (include/nopcs.h): argument marshalling only.

Every function here has the name and arguments of the C entry point it wraps
and raises NopcsError on a non-OK status.  All computation happens in the CUDA
library; if the library is missing this module raises at import time.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnopcs.so")

NOPCS_OK, NOPCS_EINVAL, NOPCS_ENOMEM, NOPCS_ECUDA, NOPCS_EUNSTABLE, NOPCS_ETIMEOUT, NOPCS_EUNSUPPORTED = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EUNSTABLE", "ETIMEOUT", "EUNSUPPORTED"]
NOPCS_FP64, NOPCS_MIXED = 0, 1
NOPCS_FORM_AUTO, NOPCS_FORM_THOMAS, NOPCS_FORM_GEMM_3XTF32, NOPCS_FORM_GEMM_BF16X3, NOPCS_FORM_BANDED = range(5)
NOPCS_NUM_KERNELS = 12


class NopcsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("NOPCS_%s: %s" % (name, msg))


class nopcs_box_desc(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("len", C.c_double * 3), ("gravity_axis", C.c_int),
                ("sub_n", C.c_int * 3), ("Re", C.c_double), ("M", C.c_double), ("Pr", C.c_double),
                ("gamma", C.c_double), ("suth_S", C.c_double), ("mub_scale", C.c_double),
                ("mu_s_si", C.c_double), ("Ts_kelvin", C.c_double), ("T_upper", C.c_double),
                ("T_lower", C.c_double), ("g", C.c_double), ("dt", C.c_double),
                ("filter_every", C.c_int), ("filter_alpha", C.c_double), ("base_subtract", C.c_int),
                ("seed", C.c_ulonglong), ("perturb_amp", C.c_double), ("visc_compact", C.c_int)]


class nopcs_diag(C.Structure):
    _fields_ = [("mass", C.c_double), ("momentum", C.c_double * 3), ("energy_total", C.c_double),
                ("max_speed", C.c_double), ("max_dp", C.c_double), ("max_mach", C.c_double),
                ("step", C.c_longlong), ("nonfinite", C.c_int)]


if not os.path.exists(LIB_PATH):
    raise ImportError("libnopcs.so is not built (run __graft_entry__.build()); there is no fallback")

_L = C.CDLL(LIB_PATH)
_vp, _i, _d = C.c_void_p, C.c_int, C.c_double
_L.nopcs_init.argtypes = [C.POINTER(nopcs_box_desc), _i, _i, _i, _vp, C.POINTER(_vp)]
_L.nopcs_destroy.argtypes = [_vp]
_L.nopcs_destroy.restype = None
_L.nopcs_last_error.argtypes = [_vp]
_L.nopcs_last_error.restype = C.c_char_p
_L.nopcs_set_state.argtypes = [_vp, _i, _vp]
_L.nopcs_get_state.argtypes = [_vp, _i, _vp]
_L.nopcs_stage_state.argtypes = [_vp, _i, _vp]
_L.nopcs_commit_state.argtypes = [_vp, _i]
_L.nopcs_reset_state.argtypes = [_vp, _i]
_L.nopcs_set_step.argtypes = [_vp, _i, C.c_longlong]
_L.nopcs_set_memory_limit.argtypes = [C.c_ulonglong]
_L.nopcs_set_launch.argtypes = [_vp, _i, _d]
_L.nopcs_derivative.argtypes = [_vp, _i, _i, _i, _i, _vp, _vp, _vp]
_L.nopcs_derivative2_noalloc.argtypes = [_vp, _i, _i, _i, _vp, _vp, _vp]
_L.nopcs_rk_step.argtypes = [_vp, _i]
_L.nopcs_rhs.argtypes = [_vp, _i, _vp, _vp]
_L.nopcs_filter.argtypes = [_vp, _i]
_L.nopcs_diagnostics.argtypes = [_vp, _i, C.POINTER(nopcs_diag)]
_L.nopcs_synchronize.argtypes = [_vp]
_L.nopcs_box_info.argtypes = [_vp, _i, _vp, _vp, _vp]
_L.nopcs_set_profiling.argtypes = [_vp, _i]
_L.nopcs_profile_read.argtypes = [_vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), _i]
_L.nopcs_kernel_name.argtypes = [_i]
_L.nopcs_kernel_name.restype = C.c_char_p
_L.nopcs_operator_rows.argtypes = [_i, _i, _i, _d, _d, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i),
                                   C.POINTER(_i), C.POINTER(_d), _i]
_L.nopcs_operator_apply.argtypes = [_i, _i, _i, _d, _d, C.c_void_p, C.c_void_p]
_L.nopcs_plane_fields.argtypes = [_vp, _i, _i, _i, _i, _vp]
_L.nopcs_band_apply.argtypes = [_i, _i, _d, _d, C.c_void_p, C.c_void_p, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)]
_L.nopcs_slab_create.argtypes = [C.POINTER(nopcs_box_desc), _i, _i, C.POINTER(_vp)]
_L.nopcs_slab_destroy.argtypes = [_vp]
_L.nopcs_slab_destroy.restype = None
_L.nopcs_slab_last_error.argtypes = [_vp]
_L.nopcs_slab_last_error.restype = C.c_char_p
_L.nopcs_slab_extent.argtypes = [_vp, _i, C.POINTER(_i), C.POINTER(_i)]
_L.nopcs_slab_derivative.argtypes = [_vp, _i, _i, _vp, _vp, _vp]
_L.nopcs_slab_line_apply.argtypes = [_i, _i, _d, _i, _i, C.c_void_p, C.c_void_p, C.POINTER(_i), C.POINTER(_i)]
for _name in ("nopcs_slab_create", "nopcs_slab_extent", "nopcs_slab_derivative", "nopcs_slab_line_apply"):
    getattr(_L, _name).restype = _i
for _name in ("nopcs_operator_apply", "nopcs_band_apply", "nopcs_plane_fields", "nopcs_init", "nopcs_set_state",
              "nopcs_get_state", "nopcs_stage_state", "nopcs_commit_state", "nopcs_reset_state", "nopcs_set_step", "nopcs_set_memory_limit", "nopcs_set_launch",
              "nopcs_derivative",
              "nopcs_derivative2_noalloc",
              "nopcs_rk_step", "nopcs_rhs", "nopcs_filter", "nopcs_diagnostics", "nopcs_synchronize",
              "nopcs_set_profiling", "nopcs_profile_read", "nopcs_operator_rows", "nopcs_box_info"):
    getattr(_L, _name).restype = _i


def lib():
    return _L


def _check(ctx, st):
    if st != NOPCS_OK:
        msg = _L.nopcs_last_error(ctx)
        raise NopcsError(st, msg.decode() if msg else "")


def box_desc(p: dict) -> nopcs_box_desc:
    """Plain dict of box parameters -> nopcs_box_desc."""
    d = nopcs_box_desc()
    for k, v in p.items():
        if k in ("n", "sub_n"):
            getattr(d, k)[:] = [int(x) for x in v]
        elif k == "len":
            d.len[:] = [float(x) for x in v]
        elif hasattr(d, k):
            setattr(d, k, v)
    return d


def nopcs_init(boxes, prec: int = NOPCS_FP64, form: int = NOPCS_FORM_AUTO, stream: int = 0):
    """boxes: list of dicts (or nopcs_box_desc); returns an opaque context handle."""
    arr = (nopcs_box_desc * len(boxes))(*[b if isinstance(b, nopcs_box_desc) else box_desc(b) for b in boxes])
    out = _vp()
    _check(None, _L.nopcs_init(arr, len(boxes), prec, form, _vp(stream or None), C.byref(out)))
    return out.value


def nopcs_destroy(ctx) -> None:
    _L.nopcs_destroy(ctx)


def nopcs_last_error(ctx) -> str:
    m = _L.nopcs_last_error(ctx)
    return m.decode() if m else ""


def nopcs_set_state(ctx, box: int, q_ptr: int) -> None:
    _check(ctx, _L.nopcs_set_state(ctx, box, q_ptr))


def nopcs_get_state(ctx, box: int, q_ptr: int) -> None:
    _check(ctx, _L.nopcs_get_state(ctx, box, q_ptr))


def nopcs_stage_state(ctx, box: int, q_ptr: int) -> None:
    _check(ctx, _L.nopcs_stage_state(ctx, box, q_ptr))


def nopcs_commit_state(ctx, box: int) -> None:
    _check(ctx, _L.nopcs_commit_state(ctx, box))


def nopcs_reset_state(ctx, box: int) -> None:
    _check(ctx, _L.nopcs_reset_state(ctx, box))


def nopcs_set_step(ctx, box: int, step: int) -> None:
    _check(ctx, _L.nopcs_set_step(ctx, box, step))


def nopcs_set_memory_limit(nbytes: int) -> None:
    """Process-wide cap on the device bytes of each context created
    afterwards (0: no cap)."""
    _check(None, _L.nopcs_set_memory_limit(nbytes))


NOPCS_LAUNCH_GRAPH, NOPCS_LAUNCH_PERSISTENT, NOPCS_LAUNCH_PERSISTENT_WITHHOLD = 0, 1, 2


def nopcs_set_launch(ctx, mode: int, wait_limit_s: float = 2.0) -> None:
    """CUDA graph per step (default) or one persistent kernel per step."""
    _check(ctx, _L.nopcs_set_launch(ctx, mode, float(wait_limit_s)))


def nopcs_derivative(ctx, box: int, axis: int, order: int, dtype: int, f_ptr: int, df_ptr: int,
                     stream: int = 0) -> None:
    _check(ctx, _L.nopcs_derivative(ctx, box, axis, order, dtype, f_ptr, df_ptr, _vp(stream or None)))


def nopcs_derivative2_noalloc(ctx, box: int, axis: int, dtype: int, f_ptr: int, df_ptr: int,
                              stream: int = 0) -> None:
    """Second derivative without any device allocation in the call (fixed
    16 MiB library scratch; see include/nopcs.h for the limits)."""
    _check(ctx, _L.nopcs_derivative2_noalloc(ctx, box, axis, dtype, f_ptr, df_ptr, _vp(stream or None)))


def nopcs_rk_step(ctx, nsteps: int) -> None:
    _check(ctx, _L.nopcs_rk_step(ctx, nsteps))


def nopcs_rhs(ctx, box: int, q_ptr: int, r_ptr: int) -> None:
    _check(ctx, _L.nopcs_rhs(ctx, box, q_ptr, r_ptr))


def nopcs_filter(ctx, box: int) -> None:
    _check(ctx, _L.nopcs_filter(ctx, box))


def nopcs_diagnostics(ctx, box: int, allow_unstable: bool = False) -> dict:
    d = nopcs_diag()
    st = _L.nopcs_diagnostics(ctx, box, C.byref(d))
    if not (allow_unstable and st == NOPCS_EUNSTABLE):
        _check(ctx, st)
    return dict(mass=d.mass, momentum=list(d.momentum), energy_total=d.energy_total, max_speed=d.max_speed,
                max_dp=d.max_dp, max_mach=d.max_mach, step=d.step, nonfinite=d.nonfinite)


def nopcs_box_info(ctx, box: int) -> dict:
    """Sub-domain length, FP32-derivative form and flux-sweep tile width in
    force per axis."""
    sub = (_i * 3)()
    form = (_i * 3)()
    lines = (_i * 3)()
    _check(ctx, _L.nopcs_box_info(ctx, box, sub, form, lines))
    return {"sub_n": list(sub), "deriv_form": list(form), "tile_lines": list(lines)}


NOPCS_PLANE_DP, NOPCS_PLANE_VORTICITY_TERMS = 0, 1
NOPCS_ORDER_D2_COMPACT = 3


def nopcs_plane_fields(ctx, box: int, axis: int, index: int, what: int, out_ptr: int) -> None:
    """Plane diagnostics (disturbance pressure or the nine vorticity-transport
    terms) into a caller-owned device buffer; enqueued on the context stream."""
    _check(ctx, _L.nopcs_plane_fields(ctx, box, axis, index, what, out_ptr))


def nopcs_synchronize(ctx) -> None:
    _check(ctx, _L.nopcs_synchronize(ctx))


def nopcs_set_profiling(ctx, on: bool) -> None:
    _check(ctx, _L.nopcs_set_profiling(ctx, int(on)))


def nopcs_profile_read(ctx, reset: bool = False) -> dict:
    ms = (C.c_double * NOPCS_NUM_KERNELS)()
    n = (C.c_longlong * NOPCS_NUM_KERNELS)()
    _check(ctx, _L.nopcs_profile_read(ctx, ms, n, int(reset)))
    return {nopcs_kernel_name(k): (ms[k], n[k]) for k in range(NOPCS_NUM_KERNELS)}


def nopcs_kernel_name(kind: int):
    m = _L.nopcs_kernel_name(kind)
    return m.decode() if m else None


def nopcs_operator_rows(N: int, sub_n: int, kind: int = 0, alpha_f: float = 0.135, thresh: float = 1e-16):
    """Host tables of a line operator: (starts, end_j0, end_len, coef list per end row)."""
    cap = 4 * (N + 8) * (N + 2)
    nsub = _i()
    starts = (_i * (N + 2))()
    j0 = (_i * (2 * N + 4))()
    ln = (_i * (2 * N + 4))()
    coef = (_d * cap)()
    st = _L.nopcs_operator_rows(N, sub_n, kind, alpha_f, thresh, C.byref(nsub), starts, j0, ln, coef, cap)
    if st != NOPCS_OK:
        raise NopcsError(st, "bad operator request")
    nb = nsub.value
    rows = []
    off = 0
    for k in range(2 * nb):
        L = ln[k]
        rows.append((j0[k], [coef[off + t] for t in range(L)]))
        off += L
    return list(starts[: nb + 1]), rows


def nopcs_band_apply(N: int, f, kind: int = 0, alpha_f: float = 0.135, thresh: float = 1e-16):
    """Host FP64 evaluation of the banded explicit form on a numpy line f;
    returns (g, half_width, interior_lo, interior_hi)."""
    import numpy as np
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.zeros_like(f)
    h, lo, hi = _i(), _i(), _i()
    st = _L.nopcs_band_apply(N, kind, alpha_f, thresh, f.ctypes.data, g.ctypes.data, C.byref(h), C.byref(lo),
                             C.byref(hi))
    if st != NOPCS_OK:
        raise NopcsError(st, "bad operator request")
    return g, h.value, lo.value, hi.value


def nopcs_operator_apply(N: int, sub_n: int, f, kind: int = 0, alpha_f: float = 0.135, thresh: float = 1e-16):
    """Host FP64 evaluation of the library's line operator on a numpy line f."""
    import numpy as np
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.zeros_like(f)
    st = _L.nopcs_operator_apply(N, sub_n, kind, alpha_f, thresh, f.ctypes.data, g.ctypes.data)
    if st != NOPCS_OK:
        raise NopcsError(st, "bad operator request")
    return g


def _slab_check(slab, st):
    if st != NOPCS_OK:
        msg = _L.nopcs_slab_last_error(slab)
        raise NopcsError(st, msg.decode() if msg else "")


def nopcs_slab_create(box, z0: int, z1: int):
    """A z-slab [z0, z1) of the box (dict or nopcs_box_desc); returns a handle."""
    d = box if isinstance(box, nopcs_box_desc) else box_desc(box)
    out = _vp()
    _slab_check(None, _L.nopcs_slab_create(C.byref(d), z0, z1, C.byref(out)))
    return out.value


def nopcs_slab_destroy(slab) -> None:
    _L.nopcs_slab_destroy(slab)


def nopcs_slab_extent(slab, dtype: int):
    lo, hi = _i(), _i()
    _slab_check(slab, _L.nopcs_slab_extent(slab, dtype, C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def nopcs_slab_derivative(slab, axis: int, dtype: int, f_ptr: int, df_ptr: int, stream: int = 0) -> None:
    _slab_check(slab, _L.nopcs_slab_derivative(slab, axis, dtype, f_ptr, df_ptr, _vp(stream or None)))


def nopcs_slab_line_apply(N: int, sub_n: int, thresh: float, z0: int, z1: int, f=None):
    """Host FP64 evaluation of the slab-restricted line operator: with f = None
    returns (lo, hi); else f holds points [lo, hi) and the result (points
    [z0, z1), times h) is returned."""
    import numpy as np
    lo, hi = _i(), _i()
    if f is None:
        st = _L.nopcs_slab_line_apply(N, sub_n, thresh, z0, z1, None, None, C.byref(lo), C.byref(hi))
        if st != NOPCS_OK:
            raise NopcsError(st, "bad slab request")
        return lo.value, hi.value
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.zeros(z1 - z0)
    st = _L.nopcs_slab_line_apply(N, sub_n, thresh, z0, z1, f.ctypes.data, g.ctypes.data, C.byref(lo),
                                  C.byref(hi))
    if st != NOPCS_OK:
        raise NopcsError(st, "bad slab request")
    return g



def nopcs_slab_last_error(slab) -> str:
    m = _L.nopcs_slab_last_error(slab)
    return m.decode() if m else ""
