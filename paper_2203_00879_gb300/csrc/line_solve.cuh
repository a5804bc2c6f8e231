// NOHAP solve of one staged column (arXiv 2203.00879, Sec. 3).
//
// A column holds (at least) the solve window win_lo .. win_hi of one (line,
// field) pair in shared memory, row r at col[(r - org) * LP].  Given the sub-domain's
// two end values (the equivalent explicit rows g_i = sum_j C_ij f_j of
// Eq. CS:fpCf_i, evaluated by the caller) the solve
//   1. evaluates any explicit wall-closure row inside the sub-domain,
//   2. runs the Thomas forward sweep over the implicit rows (tabulated factors,
//      the end values moved to the right-hand side), keeping the last 2W+1
//      inputs in registers and writing the forward values in place,
//   3. back-substitutes in place,
// leaving the derivative (or filtered value) of rows s .. e in place, times
// osc when SCALED.
#pragma once

#include "nopcs_internal.cuh"

namespace nopcs {

template <typename T>
__device__ __forceinline__ const T *coef_ptr(const LineOpDev &op);
template <>
__device__ __forceinline__ const double *coef_ptr<double>(const LineOpDev &op) { return op.coef64; }
template <>
__device__ __forceinline__ const float *coef_ptr<float>(const LineOpDev &op) { return op.coef32; }
template <typename T>
__device__ __forceinline__ const T *cp_ptr(const LineOpDev &op);
template <>
__device__ __forceinline__ const double *cp_ptr<double>(const LineOpDev &op) { return op.cp64; }
template <>
__device__ __forceinline__ const float *cp_ptr<float>(const LineOpDev &op) { return op.cp32; }
template <typename T>
__device__ __forceinline__ const T *inv_ptr(const LineOpDev &op);
template <>
__device__ __forceinline__ const double *inv_ptr<double>(const LineOpDev &op) { return op.inv64; }
template <>
__device__ __forceinline__ const float *inv_ptr<float>(const LineOpDev &op) { return op.inv32; }

// dot product of `len` taps with a column (stride LP), four partial sums
template <typename T>
__device__ __forceinline__ T dot_col(const T *c, const T *f, int len, int LP)
{
    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    int k = 0;
    for (; k + 4 <= len; k += 4) {
        s0 += c[k] * f[(size_t)k * LP];
        s1 += c[k + 1] * f[(size_t)(k + 1) * LP];
        s2 += c[k + 2] * f[(size_t)(k + 2) * LP];
        s3 += c[k + 3] * f[(size_t)(k + 3) * LP];
    }
    for (; k < len; ++k) s0 += c[k] * f[(size_t)k * LP];
    return (s0 + s1) + (s2 + s3);
}

// org: the row at col[0]; gs / ge: the end values at rows s and e (ge unused
// when e == s); tcp / tiv: the first KC Thomas factors (the rest equal their
// limits cpL / invL).
template <typename T, int MODE, bool SCALED>
__device__ __forceinline__ void nohap_solve_column(const LineOpDev &op, T *col, int LP, int org, T gs, T ge,
                                                   const T *tcp, const T *tiv, int KC, const int *rec, T osc)
{
    constexpr int W = MODE == MODE_FILTER ? 3 : 2;     // right-hand-side half-width
    constexpr int NEXP = MODE == MODE_FILTER ? 3 : 2;  // explicit rows at each wall
    const int s = rec[0], e = rec[1], tlo = org;
    const int lene = rec[8];
    const int lo = rec[10], hi = rec[11];
    const int N = op.N;
    auto out = [&](T v) { return SCALED ? v * osc : v; };
    // explicit wall-closure rows strictly inside the sub-domain
    T exL[NEXP], exH[NEXP];
#pragma unroll
    for (int r = 0; r < NEXP; ++r) {
        exL[r] = 0;
        exH[r] = 0;
        if (r > s && r < e) {
            T acc = 0;
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (op.ex[r][j] != 0.0) acc += (T)op.ex[r][j] * col[(size_t)(j - tlo) * LP];
            exL[r] = acc;
        }
        const int rh = N - 1 - r;
        if (rh > s && rh < e) {
            T acc = 0;
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (op.ex[r][j] != 0.0) acc += (T)op.ex[r][j] * col[(size_t)(N - 1 - j - tlo) * LP];
            exH[r] = (T)op.ex_sign * acc;
        }
    }
    // 2./3. Thomas over the implicit rows lo..hi; forward values overwrite
    // the staged inputs, which a register window of 2W+1 keeps
    if (lo <= hi) {
        const int m = hi - lo + 1;
        const T al = (T)op.alpha;
        const T gL = lo == s + 1 ? gs : exL[NEXP - 1];
        const T gR = hi == e - 1 ? ge : exH[NEXP - 1];
        const T r0 = (T)op.rb[0], r1 = (T)op.rb[1], r2 = (T)op.rb[2], r3 = (T)op.rb[3];
        const T cL = (T)op.cpL, iL = (T)op.invL;
        T win[2 * W + 1];
        const T *pin = col + (size_t)(lo - W - tlo) * LP;
#pragma unroll
        for (int j = 0; j < 2 * W; ++j) win[j] = pin[(size_t)j * LP];
        pin += (size_t)(2 * W) * LP;                // row lo + W
        T *pout = col + (size_t)(lo - tlo) * LP;   // row lo
        T dprev = 0;
        // one forward row: right-hand side from the window, minus the
        // coupling `adj` to a known end value, then the elimination
        auto fwd = [&](T iv, T adj) {
            win[2 * W] = *pin;
            pin += LP;
            T rhs;
            if constexpr (MODE == MODE_FILTER)
                rhs = r0 * win[3] + r1 * (win[4] + win[2]) + r2 * (win[5] + win[1]) + r3 * (win[6] + win[0]);
            else if constexpr (MODE == MODE_FIELD2)
                rhs = r0 * win[2] + r1 * (win[3] + win[1]) + r2 * (win[4] + win[0]);
            else
                rhs = r0 * (win[3] - win[1]) + r1 * (win[4] - win[0]);
            const T dp = (rhs - adj - al * dprev) * iv;
            *pout = dp;
            pout += LP;
            dprev = dp;
#pragma unroll
            for (int j = 0; j < 2 * W; ++j) win[j] = win[j + 1];
        };
        // first row carries the left end value (and the right one if m == 1)
        fwd(tiv[0], al * gL + (m == 1 ? al * gR : T(0)));
        const int kmid = min(KC, m - 1);
        int r = 1;
#pragma unroll 4
        for (; r < kmid; ++r) fwd(tiv[r], T(0));
#pragma unroll 4
        for (; r < m - 1; ++r) fwd(iL, T(0));
        if (m > 1) fwd(m - 1 < KC ? tiv[m - 1] : iL, al * gR);
        // back substitution from row hi - 1 down to lo
        T x = dprev;
        if (SCALED) pout[-(ptrdiff_t)LP] = out(x);  // row hi
        pout -= 2 * (size_t)LP;                      // row hi - 1
        r = m - 2;
#pragma unroll 4
        for (; r >= KC; --r) {
            x = *pout - cL * x;
            *pout = out(x);
            pout -= LP;
        }
#pragma unroll 4
        for (; r >= 0; --r) {
            x = *pout - tcp[r] * x;
            *pout = out(x);
            pout -= LP;
        }
    }
    // explicit values into their rows
    col[(size_t)(s - tlo) * LP] = out(gs);
    if (lene > 0) col[(size_t)(e - tlo) * LP] = out(ge);
#pragma unroll
    for (int r = 0; r < NEXP; ++r) {
        if (r > s && r < e) col[(size_t)(r - tlo) * LP] = out(exL[r]);
        const int rh = N - 1 - r;
        if (rh > s && rh < e) col[(size_t)(rh - tlo) * LP] = out(exH[r]);
    }
}

}  // namespace nopcs
