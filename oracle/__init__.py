"""FP64 CPU oracle for the NOHAP/OUCS3 compressible Navier-Stokes hot path.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may use this package; the product library never does.  It is a
ctypes front end over ``nopcs_oracle.c`` (plain C, FP64, OpenMP over lines) and
shares no code with the CUDA library.  See the header of ``nopcs_oracle.c`` for
the paper passages each function follows and the readings taken where the
paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nopcs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_FMA = os.path.join(_HERE, "liboracle_fma.so")

OUCS3 = (0.3793894912, 0.7877868952, 0.045801298, -0.025)  # alpha, b1, b2, beta
DERIV, FILTER, D2 = 0, 1, 2
LELE_D2 = (2.0 / 11.0, 12.0 / 11.0, 3.0 / 11.0)  # alpha, a, b of the sixth-order compact second derivative
THRESH_FP64 = 1e-16


def build(force: bool = False, contracted: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP) next to its source.  contracted:
    the same source with multiply-adds fused into FMAs wherever the compiler
    likes (-ffp-contract=fast; FMA instructions are native on aarch64), a
    second rounding of the same arithmetic, used only to size round-off
    differences."""
    path = _LIB_FMA if contracted else _LIB
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + ".tmp%d" % os.getpid()
        extra = []
        if contracted:
            extra = ["-ffp-contract=fast"]
            import platform
            if platform.machine() in ("x86_64", "AMD64"):
                extra.append("-mfma")
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", *extra, "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, path)
    return path


class _Box(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("len", C.c_double * 3), ("gravity_axis", C.c_int),
                ("sub_n", C.c_int * 3), ("Re", C.c_double), ("M", C.c_double), ("Pr", C.c_double),
                ("gamma", C.c_double), ("suth_S", C.c_double), ("mub_scale", C.c_double),
                ("mu_s_si", C.c_double), ("Ts_kelvin", C.c_double), ("T_upper", C.c_double),
                ("T_lower", C.c_double), ("g", C.c_double), ("dt", C.c_double),
                ("filter_every", C.c_int), ("filter_alpha", C.c_double), ("base_subtract", C.c_int),
                ("seed", C.c_ulonglong), ("perturb_amp", C.c_double), ("visc_compact", C.c_int)]


_lib = None
_lib_fma = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def lib_contracted():
    """The oracle built with FMA contraction (see build); for round-off studies."""
    global _lib_fma
    if _lib_fma is None:
        _lib_fma = _bind(C.CDLL(build(contracted=True)))
    return _lib_fma


def _bind(L):
    if True:
        L.orc_partition.argtypes = [C.c_int, C.c_int, _ip]
        L.orc_partition.restype = C.c_int
        L.orc_op_new.argtypes = [C.c_int, C.c_int, _dp, C.c_int, C.c_double]
        L.orc_op_new.restype = C.c_void_p
        L.orc_op_free.argtypes = [C.c_void_p]
        L.orc_op_get.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_op_nsub.argtypes = [C.c_void_p]
        L.orc_op_nsub.restype = C.c_int
        L.orc_op_apply_dense.argtypes = [C.c_void_p, _dp, _dp, C.c_double]
        L.orc_op_apply_nopcs.argtypes = [C.c_void_p, _dp, _dp, C.c_double]
        L.orc_apply_axis.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp,
                                     C.c_double, C.c_int]
        L.orc_d2_axis.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, _dp, _dp]
        L.orc_base_profile.argtypes = [C.POINTER(_Box), _dp, _dp]
        L.orc_solver_new.argtypes = [C.POINTER(_Box), C.c_double]
        L.orc_solver_new.restype = C.c_void_p
        L.orc_solver_free.argtypes = [C.c_void_p]
        L.orc_initial_state.argtypes = [C.c_void_p, _dp]
        L.orc_rhs.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_apply_wall_bc.argtypes = [C.c_void_p, _dp]
        L.orc_set_wall_extrapolation.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_filter.argtypes = [C.c_void_p, _dp]
        L.orc_rk_steps.argtypes = [C.c_void_p, _dp, C.c_int]
        L.orc_solver_step.argtypes = [C.c_void_p]
        L.orc_solver_step.restype = C.c_longlong
        L.orc_solver_set_step.argtypes = [C.c_void_p, C.c_longlong]
        L.orc_diagnostics.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_plane_fields.argtypes = [C.c_void_p, _dp, C.c_int, C.c_int, C.c_int, _dp]
        L.orc_plane_fields.restype = C.c_int
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
    return L


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on (for timing)."""
    lib().orc_set_num_threads(int(n))


def partition(N: int, sub_n: int) -> np.ndarray:
    """Sub-domain start indices (plus N) under the remainder rule."""
    st = np.zeros(N + 2, dtype=np.int32)
    nb = lib().orc_partition(N, sub_n, st)
    return st[: nb + 1].copy()


class Op:
    """One-dimensional compact operator on N points: derivative or filter."""

    def __init__(self, N: int, kind: int = DERIV, sub_n: int = 0, thresh: float = THRESH_FP64,
                 coef=None):
        if coef is None:
            coef = {DERIV: OUCS3, FILTER: (0.135,), D2: LELE_D2}[kind]
        self._coef = np.ascontiguousarray(coef, dtype=np.float64)
        self.N = N
        self._p = lib().orc_op_new(N, kind, self._coef, sub_n, thresh)
        if not self._p:
            raise ValueError("line too short for this operator")

    def __del__(self):
        if getattr(self, "_p", None):
            lib().orc_op_free(self._p)
            self._p = None

    def matrices(self):
        B = np.zeros((self.N, self.N))
        Cm = np.zeros((self.N, self.N))
        lib().orc_op_get(self._p, B.ctypes.data, Cm.ctypes.data, None)
        return B, Cm

    def starts(self):
        nb = lib().orc_op_nsub(self._p)
        st = np.zeros(nb + 1, dtype=np.int32)
        lib().orc_op_get(self._p, None, None, st.ctypes.data)
        return st

    def nopcs(self, f, scale=1.0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty_like(f)
        lib().orc_op_apply_nopcs(self._p, f, out, scale)
        return out

    def dense(self, f, scale=1.0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty_like(f)
        lib().orc_op_apply_dense(self._p, f, out, scale)
        return out


def deriv3d(f, axis: int, h: float, sub_n: int, thresh: float = THRESH_FP64, dense: bool = False,
            kind: int = DERIV):
    """Compact operator along `axis` (0 = x, fastest) of an (nz, ny, nx) array."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    N = (nx, ny, nz)[axis]
    op = Op(N, kind, sub_n, thresh)
    out = np.empty_like(f)
    scale = {DERIV: 1.0 / h, FILTER: 1.0, D2: 1.0 / (h * h)}[kind]
    lib().orc_apply_axis(op._p, nx, ny, nz, axis, f, out, scale, int(dense))
    return out


def explicit2(f, axis: int, h: float):
    """Second-order explicit first derivative along `axis`."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    out = np.empty_like(f)
    lib().orc_d2_axis(nx, ny, nz, axis, h, f, out)
    return out


def _box(p: dict) -> _Box:
    b = _Box()
    for k, v in p.items():
        if k in ("n", "sub_n"):
            getattr(b, k)[:] = [int(x) for x in v]
        elif k == "len":
            b.len[:] = [float(x) for x in v]
        else:
            setattr(b, k, v)
    return b


def base_profile(p: dict):
    b = _box(p)
    Ng = p["n"][p["gravity_axis"]]
    rho = np.zeros(Ng)
    pr = np.zeros(Ng)
    lib().orc_base_profile(C.byref(b), rho, pr)
    return rho, pr


class Solver:
    """FP64 reference solver for one box.  State arrays have shape (5, nz, ny, nx)."""

    def __init__(self, p: dict, thresh: float = THRESH_FP64, contracted: bool = False):
        self.p = dict(p)
        self._b = _box(p)
        self.shape = (5, p["n"][2], p["n"][1], p["n"][0])
        self._L = lib_contracted() if contracted else lib()
        self._s = self._L.orc_solver_new(C.byref(self._b), thresh)
        if not self._s:
            raise ValueError("box too small")

    def __del__(self):
        if getattr(self, "_s", None):
            self._L.orc_solver_free(self._s)
            self._s = None

    def initial_state(self):
        Q = np.zeros(self.shape)
        self._L.orc_initial_state(self._s, Q)
        return Q

    def rhs(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        R = np.zeros_like(Q)
        self._L.orc_rhs(self._s, Q, R)
        return R

    def wall_bc(self, Q):
        Q = np.array(Q, dtype=np.float64, order="C")
        self._L.orc_apply_wall_bc(self._s, Q)
        return Q

    @staticmethod
    def set_wall_extrapolation(w1: float = 4.0, w2: float = 1.0, w3: float = 3.0):
        """Weights of T_w = (w1 T_1 - w2 T_2) / w3 for every solver (default: the
        adiabatic rule).  For tests that plant a wrong rule; restore afterwards."""
        lib().orc_set_wall_extrapolation(float(w1), float(w2), float(w3))

    def filter(self, Q):
        Q = np.array(Q, dtype=np.float64, order="C")
        self._L.orc_filter(self._s, Q)
        return Q

    def step(self, Q, nsteps: int = 1):
        """Advance a copy of Q by nsteps RK4 steps (filter on its cadence)."""
        Q = np.array(Q, dtype=np.float64, order="C")
        self._L.orc_rk_steps(self._s, Q, int(nsteps))
        return Q

    @property
    def step_count(self) -> int:
        return self._L.orc_solver_step(self._s)

    @step_count.setter
    def step_count(self, v: int):
        self._L.orc_solver_set_step(self._s, int(v))

    def diagnostics(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.zeros(9)
        self._L.orc_diagnostics(self._s, Q, out)
        return dict(mass=out[0], momentum=out[1:4].copy(), energy_total=out[4], max_speed=out[5],
                    max_dp=out[6], max_mach=out[7], nonfinite=int(out[8]))

    def plane_fields(self, Q, axis: int, index: int, what: int):
        """Disturbance pressure (what = 0, shape (nb, na)) or the nine
        vorticity-transport terms of Eq. eqn12_1 (what = 1, shape (9, nb, na))
        on the plane normal to `axis` at node `index`."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        n = self.p["n"]
        a, b = [d for d in range(3) if d != axis]
        out = np.zeros((9 if what else 1, n[b], n[a]))
        k = self._L.orc_plane_fields(self._s, Q, axis, index, what, out)
        if k < 0:
            raise ValueError("bad plane request")
        return out[0] if what == 0 else out
