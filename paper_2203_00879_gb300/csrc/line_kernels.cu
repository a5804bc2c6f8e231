// NOHAP line sweeps on sm_103a (arXiv 2203.00879, Sec. 3).
//
// One CUDA block owns one sub-domain [s, e] of LINES neighbouring grid lines.
// It streams in the rows the sub-domain needs: its own points, the +-2 (+-3
// for the filter) right-hand-side stencil, and the end-row supports of up to
// 48 (FP64) / 24 (FP32) points into the neighbouring sub-domains.  As rows
// pass, the two end values g_i = sum_j C_ij f_j (Eq. CS:fpCf_i) are summed
// from them; only the solve window (the own rows plus the stencil) is kept in
// shared memory, laid out [field][row][line] with an odd line pitch, so that
//   - a line along the contiguous x axis is read row-contiguous (coalesced,
//     a warp per line, its lanes' partial sums reduced with shuffles) and
//     transposed on the fly into the [row][line] layout, and
//   - lines along y or z are read line-contiguous (coalesced along x).
// Each thread then owns one (line, field) column and solves it
// (line_solve.cuh): explicit wall-closure rows, a Thomas forward sweep over
// the implicit rows with the end values moved to the right-hand side, and
// back substitution, in place.  The block finally writes its own rows back
// (transposed again for x).  Sub-domains are independent, so no block waits
// for another.  (The single-field derivative along x keeps its whole staged
// tile and takes the end values from it.)
//
// Modes: FIELD / FIELD2 one field; FLUX the five inviscid fluxes along the
// axis from the stage primitives, into R; FILTER five state fields; VGRAD and
// VDIV the compact viscous terms -- the derivatives of u, v, w, T, and those
// of the four viscous-flux components along the axis, added into R[1..4].
#include "line_body.cuh"

namespace nopcs {

template <typename T, int MODE, int AXIS>
__global__ void line_kernel(const LineOpDev op, const LineArgs<T> a)
{
    line_body<T, MODE, AXIS, true>(op, a, blockIdx.x, 0);
}

namespace {

template <typename T, int MODE, int AXIS>
cudaError_t launch_axis(const LineOpDev &op, LineArgs<T> a, int pref_lines, cudaStream_t st)
{
    LineGrid g;
    if (!line_grid<T, MODE, AXIS>(op, a, pref_lines, 0, XLINE_MAX_LINES, g)) return cudaErrorInvalidConfiguration;
    if (g.nblk <= 0) return cudaSuccess;
    if constexpr (AXIS == 0 && MODE == MODE_FLUX) {
        if (g.xline) return launch_xline_flux<T>(op, a, g.nblk, g.threads, g.smem, st);
    }
    line_kernel<T, MODE, AXIS><<<(unsigned)g.nblk, g.threads, g.smem, st>>>(op, a);
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_any(const LineOpDev &op, int axis, LineArgs<T> a, int pref, cudaStream_t st)
{
    switch (axis) {
    case 0: return launch_axis<T, MODE, 0>(op, a, pref, st);
    case 1: return launch_axis<T, MODE, 1>(op, a, pref, st);
    case 2: return launch_axis<T, MODE, 2>(op, a, pref, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int MODE, int AXIS>
cudaError_t allow_smem()
{
    cudaError_t e = cudaFuncSetAttribute(line_kernel<T, MODE, AXIS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    if constexpr (AXIS == 0 && MODE == MODE_FLUX) {
        if (e == cudaSuccess) e = init_xline_flux<T>();
    }
    return e;
}

}  // namespace

cudaError_t init_line_kernels()
{
    cudaError_t e = cudaSuccess;
    cudaError_t r[] = {
        allow_smem<float, MODE_FIELD, 0>(),  allow_smem<float, MODE_FIELD, 1>(),  allow_smem<float, MODE_FIELD, 2>(),
        allow_smem<double, MODE_FIELD, 0>(), allow_smem<double, MODE_FIELD, 1>(), allow_smem<double, MODE_FIELD, 2>(),
        allow_smem<float, MODE_FLUX, 0>(),   allow_smem<float, MODE_FLUX, 1>(),   allow_smem<float, MODE_FLUX, 2>(),
        allow_smem<double, MODE_FLUX, 0>(),  allow_smem<double, MODE_FLUX, 1>(),  allow_smem<double, MODE_FLUX, 2>(),
        allow_smem<double, MODE_FILTER, 0>(), allow_smem<double, MODE_FILTER, 1>(),
        allow_smem<double, MODE_FILTER, 2>(),  allow_smem<float, MODE_FILTER, 0>(),
        allow_smem<float, MODE_FILTER, 1>(),   allow_smem<float, MODE_FILTER, 2>(),
        allow_smem<float, MODE_FIELD2, 0>(),   allow_smem<float, MODE_FIELD2, 1>(),
        allow_smem<float, MODE_FIELD2, 2>(),   allow_smem<double, MODE_FIELD2, 0>(),
        allow_smem<double, MODE_FIELD2, 1>(),  allow_smem<double, MODE_FIELD2, 2>(),
        allow_smem<float, MODE_VGRAD, 0>(),    allow_smem<float, MODE_VGRAD, 1>(),
        allow_smem<float, MODE_VGRAD, 2>(),    allow_smem<double, MODE_VGRAD, 0>(),
        allow_smem<double, MODE_VGRAD, 1>(),   allow_smem<double, MODE_VGRAD, 2>(),
        allow_smem<float, MODE_VDIV, 0>(),     allow_smem<float, MODE_VDIV, 1>(),
        allow_smem<float, MODE_VDIV, 2>(),     allow_smem<double, MODE_VDIV, 0>(),
        allow_smem<double, MODE_VDIV, 1>(),    allow_smem<double, MODE_VDIV, 2>()};
    for (cudaError_t x : r)
        if (x != cudaSuccess) e = x;
    return e;
}

template <typename T>
cudaError_t launch_line_field(const LineOpDev &op, int axis, const int n[3], const T *f, T *out,
                              double scale, cudaStream_t st)
{
    LineArgs<T> a{};
    for (int d = 0; d < 3; ++d) a.n[d] = n[d];
    a.in[0] = f;
    a.out[0] = out;
    a.scale = (T)scale;
    return launch_any<T, MODE_FIELD>(op, axis, a, sizeof(T) == 4 ? 64 : 32, st);
}

template <typename T>
cudaError_t launch_line_flux(const LineOpDev &op, int axis, const BoxDev &bx, const T *W, T *R,
                             int first, cudaStream_t st, int lines)
{
    LineArgs<T> a{};
    for (int d = 0; d < 3; ++d) a.n[d] = bx.n[d];
    for (int k = 0; k < 6; ++k) a.in[k] = W + (size_t)k * bx.np;
    for (int k = 0; k < 5; ++k) a.out[k] = R + (size_t)k * bx.np;
    a.scale = (T)bx.inv_h[axis];
    a.first = first;
    a.ga = bx.ga;
    if (sizeof(T) == 8) {
        a.b0 = (const T *)bx.rho_b64;
        a.b1 = (const T *)bx.H_b64;
    } else {
        a.b0 = (const T *)bx.rho_b32;
        a.b1 = (const T *)bx.H_b32;
    }
    return launch_any<T, MODE_FLUX>(op, axis, a, lines > 0 ? lines : (sizeof(T) == 4 ? 32 : 16), st);
}

cudaError_t launch_line_filter(const LineOpDev &op, int axis, const BoxDev &bx, int base_subtract,
                               const double *Qin, double *Qout, cudaStream_t st)
{
    LineArgs<double> a{};
    for (int d = 0; d < 3; ++d) a.n[d] = bx.n[d];
    for (int k = 0; k < 5; ++k) {
        a.in[k] = Qin + (size_t)k * bx.np;
        a.out[k] = Qout + (size_t)k * bx.np;
    }
    a.ga = bx.ga;
    // the base tables hold the hydrostatic state in the base-subtracted form
    // and zeros in the plain form
    (void)base_subtract;
    a.b0 = bx.rho_b64;
    a.b1 = bx.E_b64;
    return launch_any<double, MODE_FILTER>(op, axis, a, 16, st);
}

cudaError_t launch_line_filter32(const LineOpDev &op, int axis, const BoxDev &bx, const float *in, float *out,
                                 cudaStream_t st)
{
    LineArgs<float> a{};
    for (int d = 0; d < 3; ++d) a.n[d] = bx.n[d];
    for (int k = 0; k < 5; ++k) {
        a.in[k] = in + (size_t)k * bx.np;
        a.out[k] = out + (size_t)k * bx.np;
    }
    a.ga = bx.ga;
    a.b0 = nullptr;  // the input is the deviation from the base already
    a.b1 = nullptr;
    return launch_any<float, MODE_FILTER>(op, axis, a, 32, st);
}

template <typename T>
cudaError_t launch_line_field2(const LineOpDev &op, int axis, const int n[3], const T *f, T *out, double scale,
                               cudaStream_t st)
{
    LineArgs<T> a{};
    for (int d = 0; d < 3; ++d) a.n[d] = n[d];
    a.in[0] = f;
    a.out[0] = out;
    a.scale = (T)scale;
    return launch_any<T, MODE_FIELD2>(op, axis, a, sizeof(T) == 4 ? 64 : 32, st);
}

template <typename T>
cudaError_t launch_line_vgrad(const LineOpDev &op, int axis, const BoxDev &bx, const T *W, T *G, cudaStream_t st)
{
    LineArgs<T> a{};
    for (int d = 0; d < 3; ++d) a.n[d] = bx.n[d];
    for (int k = 0; k < 5; ++k) a.in[k] = W + (size_t)k * bx.np;
    for (int k = 0; k < 4; ++k) a.out[k] = G + (size_t)k * bx.np;
    a.scale = (T)bx.inv_h[axis];
    a.ga = bx.ga;
    if constexpr (sizeof(T) == 8) {
        a.b0 = (const T *)bx.rho_b64;
        a.b1 = (const T *)bx.p_b64;
        a.gm2 = (T)bx.gm2;
    } else {
        a.b0 = (const T *)bx.T_b32;
        a.b1 = (const T *)bx.ip_b32;
        a.b2 = (const T *)bx.ir_b32;
    }
    return launch_any<T, MODE_VGRAD>(op, axis, a, sizeof(T) == 4 ? 32 : 16, st);
}

template <typename T>
cudaError_t launch_line_vdiv(const LineOpDev &op, int axis, const BoxDev &bx, const T *F, T *R, cudaStream_t st)
{
    LineArgs<T> a{};
    for (int d = 0; d < 3; ++d) a.n[d] = bx.n[d];
    for (int k = 0; k < 4; ++k) {
        a.in[k] = F + (size_t)k * bx.np;
        a.out[k] = R + (size_t)(1 + k) * bx.np;
    }
    a.scale = (T)bx.inv_h[axis];
    a.ga = bx.ga;
    return launch_any<T, MODE_VDIV>(op, axis, a, sizeof(T) == 4 ? 32 : 16, st);
}

template cudaError_t launch_line_vgrad<float>(const LineOpDev &, int, const BoxDev &, const float *, float *,
                                              cudaStream_t);
template cudaError_t launch_line_vgrad<double>(const LineOpDev &, int, const BoxDev &, const double *, double *,
                                               cudaStream_t);
template cudaError_t launch_line_vdiv<float>(const LineOpDev &, int, const BoxDev &, const float *, float *,
                                             cudaStream_t);
template cudaError_t launch_line_vdiv<double>(const LineOpDev &, int, const BoxDev &, const double *, double *,
                                              cudaStream_t);
template cudaError_t launch_line_field2<float>(const LineOpDev &, int, const int *, const float *, float *, double,
                                               cudaStream_t);
template cudaError_t launch_line_field2<double>(const LineOpDev &, int, const int *, const double *, double *,
                                                double, cudaStream_t);
template cudaError_t launch_line_field<float>(const LineOpDev &, int, const int *, const float *, float *,
                                              double, cudaStream_t);
template cudaError_t launch_line_field<double>(const LineOpDev &, int, const int *, const double *,
                                               double *, double, cudaStream_t);
template cudaError_t launch_line_flux<float>(const LineOpDev &, int, const BoxDev &, const float *, float *,
                                             int, cudaStream_t, int);
template cudaError_t launch_line_flux<double>(const LineOpDev &, int, const BoxDev &, const double *,
                                              double *, int, cudaStream_t, int);

}  // namespace nopcs
