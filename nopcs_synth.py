"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds no arithmetic of the method: only workload parameters (the
numbers printed in arXiv 2203.00879, Sec. 2) and seeded random fields.  Random
numbers the solvers draw themselves (the initial velocity perturbation) are not
made here: each side implements SplitMix64 (Steele, Lea & Flood, OOPSLA 2014)
as a counter-based generator from its published definition.
"""
from __future__ import annotations

import math

import numpy as np

# --- physical scales of Sec. 2 ------------------------------------------------
L_SI = 0.15            # box edge, m
G_SI = 9.81            # gravity, m/s^2
TS_KELVIN = 300.0      # reference temperature T_s
RE = 12080.6           # printed Reynolds number
MACH = 0.0034939       # printed Mach number
PR = 0.712             # Prandtl number
GAMMA = 1.4
SUTH_S_KELVIN = 110.4  # Sutherland constant (standard air value; not printed)
# dimensional viscosity at T_s from Sutherland's law with mu = 1.716e-5 Pa s at
# 273.15 K (standard air constants; the paper prints only the resulting Re)
MU_S_SI = 1.8459162511975804e-05
T_S_SECONDS = math.sqrt(L_SI / G_SI)
DT_SI = 7.69e-8        # time step of the paper's run, s
DT_ND = DT_SI / T_S_SECONDS

# SplitMix64 constants (published definition)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def box_params(n=(48, 48, 48), *, sub_n=(24, 24, 24), length=None, gravity_axis=2,
               T_upper=1.0, T_lower=500.0 / 300.0, dt=DT_ND, filter_every=50,
               filter_alpha=0.135, base_subtract=0, seed=1, perturb_amp=1e-6,
               Re=RE, M=MACH, Pr=PR, gamma=GAMMA, mub_scale=1.0, g=1.0, visc_compact=0):
    """One box of the two-temperature Rayleigh-Taylor setup (plain dict).

    Nodes sit on the walls with a uniform spacing h = 1/(n_x - 1) unless
    `length` is given; the default is the unit cube.
    """
    n = tuple(int(v) for v in n)
    if length is None:
        h = 1.0 / (n[0] - 1)
        length = tuple(h * (v - 1) for v in n)
    return dict(n=n, len=tuple(float(v) for v in length), gravity_axis=int(gravity_axis),
                sub_n=tuple(int(v) for v in sub_n), Re=float(Re), M=float(M), Pr=float(Pr),
                gamma=float(gamma), suth_S=SUTH_S_KELVIN / TS_KELVIN, mub_scale=float(mub_scale),
                mu_s_si=MU_S_SI, Ts_kelvin=TS_KELVIN, T_upper=float(T_upper),
                T_lower=float(T_lower), g=float(g), dt=float(dt), filter_every=int(filter_every),
                filter_alpha=float(filter_alpha), base_subtract=int(base_subtract),
                seed=int(seed), perturb_amp=float(perturb_amp), visc_compact=int(visc_compact))


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Value number `counters` of the SplitMix64 stream seeded with `seed`."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (1.0 / 2.0 ** 53)


def normal(seed: int, count: int) -> np.ndarray:
    """Box-Muller normals on the SplitMix64 stream."""
    m = (count + 1) // 2
    c = np.arange(2 * m, dtype=np.uint64)
    u = uniform01(seed, c)
    u1 = np.maximum(u[0::2], 1e-300)
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:count]


def sine_profiles(n, kmax=64, seed=7, length=(1.0, 1.0, 1.0)):
    """Per-axis profiles sum_k (1/k) sin(2 pi k x + phi_k) on nodes x = i h."""
    prof = []
    for d in range(3):
        ph = 2 * np.pi * uniform01(seed, np.arange(kmax, dtype=np.uint64) + np.uint64(1000 * d))
        x = np.linspace(0.0, length[d], n[d])
        k = np.arange(1, kmax + 1)
        prof.append(np.sum(np.sin(2 * np.pi * k[:, None] * x[None, :] + ph[:, None]) / k[:, None], axis=0))
    return prof


def sine_field(n, kmax=64, seed=7, noise=1e-3, dtype=np.float64):
    """Derivative-benchmark field of shape (nz, ny, nx): random-phase sines along
    each axis plus N(0, noise^2) point noise (x fastest)."""
    nx, ny, nz = n
    px, py, pz = sine_profiles(n, kmax, seed, length=(1.0, 1.0, 1.0))
    f = pz[:, None, None] + py[None, :, None] + px[None, None, :]
    if noise:
        f = f + noise * normal(seed + 1, nx * ny * nz).reshape(nz, ny, nx)
    return np.ascontiguousarray(f, dtype=dtype)


def uneven_boxes(count=64, seed=11, edges=(32, 48, 64, 96, 128)):
    """Batch of independent boxes: edge from `edges`, height 1-2x edge (even),
    temperature contrast 50-250 K, upper half at T_s."""
    u = uniform01(seed, np.arange(3 * count, dtype=np.uint64)).reshape(count, 3)
    out = []
    for b in range(count):
        e = edges[min(int(u[b, 0] * len(edges)), len(edges) - 1)]
        hgt = int(round(e * (1.0 + u[b, 1]) / 2.0)) * 2
        dT = 50.0 + 200.0 * u[b, 2]
        out.append(box_params((e, e, hgt), sub_n=(64, 64, 64), T_upper=1.0,
                              T_lower=(TS_KELVIN + dT) / TS_KELVIN, seed=seed * 1000 + b))
    return out
