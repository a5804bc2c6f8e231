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
#include "line_solve.cuh"

namespace nopcs {

template <typename T>
struct LineArgs {
    int n[3];
    int lines;      // lines per block (LINES)
    int ntile_a;    // tiles along the line-tile axis
    int rt;         // staged-row capacity (op.max_tile): tile rows along x
    int rw;         // solve-window capacity (op.max_win): tile rows along y, z
    // one base pointer per field, so a node is one 32-bit index away from a
    // kernel parameter (fields hold < 2^31 points)
    const T *in[6]; // FIELD: f; FLUX: W (6 fields); FILTER: Q (5 fields);
                    // VGRAD: W (first 5 fields); VDIV: 4 flux fields
    T *out[5];      // FIELD: df; FLUX: R (5 fields); FILTER: Qout (5 fields);
                    // VGRAD: 4 gradient fields; VDIV: R[1..4]
    T scale;        // 1/h for FIELD, FLUX, VGRAD and VDIV
    int first;      // FLUX: store (1) or subtract (0)
    int ga;         // gravity axis
    const T *b0;    // FLUX: rho_b, FILTER: rho_b, VGRAD: T_b (FP32) / rho_b (FP64)
    const T *b1;    // FLUX: H_b,   FILTER: E_b,   VGRAD: 1/p_b (FP32) / p_b (FP64)
    const T *b2;    // VGRAD: 1/rho_b (FP32)
    T gm2;          // VGRAD: gamma M^2 (FP64)
};

template <typename T, int MODE, int AXIS>
__global__ void line_kernel(const LineOpDev op, const LineArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr bool SINGLE = MODE == MODE_FIELD || MODE == MODE_FIELD2;  // one field in, one out
    constexpr bool VISC = MODE == MODE_VGRAD || MODE == MODE_VDIV;      // four fields out
    constexpr int NF = SINGLE ? 1 : (VISC ? 4 : 5);
    constexpr int NIN = SINGLE ? 1 : (MODE == MODE_FLUX ? 6 : (MODE == MODE_VDIV ? 4 : 5));
    // rows in flight per thread and staging pass: four along x, three along y
    // and z (the y and z flux sweeps ran 3% and 1% faster with three than
    // with four; x 4% slower; more rows than four cost occupancy)
    constexpr int U = AXIS == 0 ? 4 : 3;
    // STREAM: the end-row dot products are summed while staging and only the
    // solve window is kept (four blocks per SM instead of three for the flux
    // sweeps); along x a warp walks one line and reduces its lanes' sums with
    // shuffles.  The single-field derivative along x keeps the whole staged
    // tile and takes the dot products in the solve (faster there).
    constexpr bool STREAM = AXIS != 0 || !SINGLE;
    const int LINES = a.lines, LP = a.lines + 1, RW = STREAM ? a.rw : a.rt;
    const int KC = sizeof(T) == 8 ? op.kconv64 : op.kconv32;
    // row groups sharing a line while staging along y, z (one warp along x)
    const int RG = STREAM ? (AXIS == 0 ? 1 : (int)blockDim.x / LINES) : 0;
    // shared memory: end-row taps (2 x max_taps), Thomas factors (2 x KC),
    // end-row partial sums [RG][2][NF][LINES], tile [NF][RW][LP]
    T *cs = reinterpret_cast<T *>(smraw);
    T *ce = cs + op.max_taps;
    T *tcp = ce + op.max_taps;
    T *tiv = tcp + KC;
    T *part = tiv + KC;
    T *sm = part + (size_t)RG * 2 * NF * LINES;
    const int nx = a.n[0], ny = a.n[1];

    const int b = blockIdx.x % op.nsub;
    const int tile = blockIdx.x / op.nsub;
    const int ta = tile % a.ntile_a;
    const int cc = tile / a.ntile_a;
    const int a0 = ta * LINES;
    const int Na = AXIS == 0 ? ny : nx;
    const int nl = min(LINES, Na - a0);

    const int *rec = op.sub + b * SUB_REC;
    const int s = rec[0], e = rec[1], tlo = rec[2], thi = rec[3];
    const int j0s = rec[4], lens = rec[5], j0e = rec[7], lene = rec[8];
    const int org = STREAM ? rec[12] : tlo, last = STREAM ? rec[13] : thi;  // tile rows
    const int nrows = thi - tlo + 1;
    const int srow = AXIS == 0 ? 1 : (AXIS == 1 ? nx : nx * ny);
    const int sa = AXIS == 0 ? nx : 1;
    const int sc = AXIS == 2 ? nx : nx * ny;
    const int gbase = cc * sc + a0 * sa + tlo * srow;
    // which of (row, line, cc) is the coordinate along the gravity axis
    const int gsel = a.ga == AXIS ? 0 : (a.ga == (AXIS == 0 ? 1 : 0) ? 1 : 2);
    const size_t fs = (size_t)RW * LP;

    // ---- block constants: end-row taps and the unconverged Thomas factors ----
    // (STREAM reads the taps from the global table while staging: no barrier
    // between these loads and the staging loads)
    const T *coef = coef_ptr<T>(op);
    {
        if (!STREAM) {
            for (int k = threadIdx.x; k < lens; k += blockDim.x) cs[k] = coef[rec[6] + k];
            for (int k = threadIdx.x; k < lene; k += blockDim.x) ce[k] = coef[rec[9] + k];
        }
        const T *cpp = cp_ptr<T>(op), *ivp = inv_ptr<T>(op);
        for (int k = threadIdx.x; k < KC; k += blockDim.x) {
            tcp[k] = cpp[k];
            tiv[k] = ivp[k];
        }
    }

    // ---- stage rows [tlo, thi] of nl lines --------------------------------------
    // Rows [org, last] go to the tile [field][row][line].  STREAM: every
    // staged row also feeds the two end-row dot products
    // g_i = sum_j C_ij f_j (Eq. CS:fpCf_i) as it passes, so the end-row
    // supports outside the solve window need no shared memory.
    // x: a warp walks the rows of one line (coalesced along x, transposed into
    // the odd line pitch); y, z: consecutive threads take consecutive lines.
    {
        int r0, rstep, l0, lstep;
        if (AXIS == 0) {
            r0 = threadIdx.x & 31;
            rstep = 32;
            l0 = threadIdx.x >> 5;
            lstep = blockDim.x >> 5;
        } else {
            l0 = threadIdx.x % LINES;
            lstep = LINES;  // one line per thread
            r0 = threadIdx.x / LINES;
            rstep = RG;
            if (r0 >= RG) l0 = LINES;  // threads beyond RG x LINES do not stage
        }
        for (int l = l0; l < (AXIS == 0 ? nl : LINES); l += lstep) {
            const int src = gbase + l * sa;
            const int gl = gsel == 1 ? a0 + l : cc;
            T ps[NF], pe[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) ps[f] = pe[f] = T(0);
            for (int r = r0; l < nl && r < nrows; r += U * rstep) {
                T v[U][NIN];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int rr = r + u * rstep;
                    if (rr < nrows) {
                        const int p = src + rr * srow;
#pragma unroll
                        for (int k = 0; k < NIN; ++k) v[u][k] = a.in[k][p];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int rr = r + u * rstep;
                    if (rr >= nrows) continue;
                    const int g = tlo + rr;
                    T val[NF];
                    if constexpr (SINGLE) {
                        val[0] = v[u][0];
                    } else if constexpr (MODE == MODE_FLUX) {
                        const int gk = gsel == 0 ? g : gl;
                        const T rho = a.b0[gk] + v[u][0];
                        const T uu = v[u][1], vv = v[u][2], ww = v[u][3], pp = v[u][4];
                        const T H = a.b1[gk] + v[u][5];
                        const T ud = AXIS == 0 ? uu : (AXIS == 1 ? vv : ww);
                        const T m = rho * ud;
                        val[0] = m;
                        val[1] = m * uu + (AXIS == 0 ? pp : T(0));
                        val[2] = m * vv + (AXIS == 1 ? pp : T(0));
                        val[3] = m * ww + (AXIS == 2 ? pp : T(0));
                        val[4] = H * ud;
                    } else if constexpr (MODE == MODE_VGRAD) {
                        // u, v, w and T = gamma M^2 p / rho of the stage state
                        const int gk = gsel == 0 ? g : gl;
                        val[0] = v[u][1];
                        val[1] = v[u][2];
                        val[2] = v[u][3];
                        if constexpr (sizeof(T) == 4) {
                            // T_b (1 + p'/p_b) / (1 + rho'/rho_b) on the deviations
                            const T rr = v[u][0] * a.b2[gk];
                            val[3] = a.b0[gk] + __fdividef(a.b0[gk] * (v[u][4] * a.b1[gk] - rr), 1.0f + rr);
                        } else {
                            val[3] = a.gm2 * (a.b1[gk] + v[u][4]) / (a.b0[gk] + v[u][0]);
                        }
                    } else if constexpr (MODE == MODE_VDIV) {
#pragma unroll
                        for (int f = 0; f < 4; ++f) val[f] = v[u][f];
                    } else {  // FILTER on Q - base (no base tables: the input is a deviation already)
                        const int gk = gsel == 0 ? g : gl;
                        val[0] = a.b0 ? v[u][0] - a.b0[gk] : v[u][0];
                        val[1] = v[u][1];
                        val[2] = v[u][2];
                        val[3] = v[u][3];
                        val[4] = a.b1 ? v[u][4] - a.b1[gk] : v[u][4];
                    }
                    if (!STREAM || (g >= org && g <= last)) {
                        T *d = sm + (size_t)(g - org) * LP + l;
#pragma unroll
                        for (int f = 0; f < NF; ++f) d[f * fs] = val[f];
                    }
                    if constexpr (STREAM) {
                        const unsigned ks = (unsigned)(g - j0s), ke = (unsigned)(g - j0e);
                        if (ks < (unsigned)lens) {
                            const T c = __ldg(coef + rec[6] + ks);
#pragma unroll
                            for (int f = 0; f < NF; ++f) ps[f] += c * val[f];
                        }
                        if (ke < (unsigned)lene) {
                            const T c = __ldg(coef + rec[9] + ke);
#pragma unroll
                            for (int f = 0; f < NF; ++f) pe[f] += c * val[f];
                        }
                    }
                }
            }
            if constexpr (STREAM) {
                if constexpr (AXIS == 0) {
                    __syncwarp();
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            ps[f] += __shfl_xor_sync(0xffffffffu, ps[f], o);
                            pe[f] += __shfl_xor_sync(0xffffffffu, pe[f], o);
                        }
                    }
                    if (r0 == 0) {
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            part[(size_t)f * LINES + l] = ps[f];
                            part[(size_t)(NF + f) * LINES + l] = pe[f];
                        }
                    }
                } else {
                    T *pp = part + l + (size_t)r0 * 2 * NF * LINES;  // [k][which][f][line]
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        pp[(size_t)f * LINES] = ps[f];
                        pp[(size_t)(NF + f) * LINES] = pe[f];
                    }
                }
            }
        }
    }
    __syncthreads();

    // ---- per-(line, field) NOHAP solve ----------------------------------------
    {
        const int l = threadIdx.x % LINES;
        const int fld = threadIdx.x / LINES;
        if (l < nl && fld < NF) {
            T *col = sm + (size_t)fld * fs + l;
            T gs = 0, ge = 0;
            if constexpr (STREAM) {
                for (int k = 0; k < RG; ++k) {
                    gs += part[((size_t)k * 2 * NF + fld) * LINES + l];
                    ge += part[((size_t)k * 2 * NF + NF + fld) * LINES + l];
                }
            } else {
                gs = dot_col(cs, col + (size_t)(j0s - org) * LP, lens, LP);
                if (lene > 0) ge = dot_col(ce, col + (size_t)(j0e - org) * LP, lene, LP);
            }
            nohap_solve_column<T, MODE, false>(op, col, LP, org, gs, ge, tcp, tiv, KC, rec, T(1));
        }
    }
    __syncthreads();

    // ---- write the sub-domain's own rows ---------------------------------------
    {
        const int nown = e - s + 1;
        int r0, rstep, l0, lstep;
        if (AXIS == 0) {
            r0 = threadIdx.x & 31;
            rstep = 32;
            l0 = threadIdx.x >> 5;
            lstep = blockDim.x >> 5;
        } else {
            l0 = threadIdx.x % LINES;
            lstep = LINES;
            r0 = threadIdx.x / LINES;
            rstep = blockDim.x / LINES;
        }
        const int obase = gbase + (s - tlo) * srow;
        for (int ll = l0; ll < nl; ll += lstep) {
            const int dstg = obase + ll * sa;
            const T *srcs = sm + (size_t)(s - org) * LP + ll;
            const int gl = gsel == 1 ? a0 + ll : cc;
            for (int r = r0; r < nown; r += U * rstep) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int rr = r + u * rstep;
                    if (rr >= nown) continue;
                    const T *src = srcs + (size_t)rr * LP;
                    const int o = dstg + rr * srow;
                    if constexpr (SINGLE) {
                        a.out[0][o] = src[0] * a.scale;
                    } else if constexpr (MODE == MODE_FLUX) {
#pragma unroll
                        for (int f = 0; f < 5; ++f) {
                            const T v = -src[f * fs] * a.scale;
                            // later sweeps add through a reduction performed
                            // in L2 (the old value never travels to the SM,
                            // so the store phase waits on no load); every
                            // element takes exactly one addition per sweep,
                            // the same rounding as load + add + store
                            if (a.first)
                                a.out[f][o] = v;
                            else
                                atomicAdd(&a.out[f][o], v);
                        }
                    } else if constexpr (MODE == MODE_VGRAD) {
#pragma unroll
                        for (int f = 0; f < 4; ++f) a.out[f][o] = src[f * fs] * a.scale;
                    } else if constexpr (MODE == MODE_VDIV) {
                        // one addition per element and sweep, as for the flux
#pragma unroll
                        for (int f = 0; f < 4; ++f) atomicAdd(&a.out[f][o], src[f * fs] * a.scale);
                    } else {
                        const int gk = gsel == 0 ? s + rr : gl;
                        a.out[0][o] = a.b0 ? src[0] + a.b0[gk] : src[0];
                        a.out[1][o] = src[fs];
                        a.out[2][o] = src[2 * fs];
                        a.out[3][o] = src[3 * fs];
                        a.out[4][o] = a.b1 ? src[4 * fs] + a.b1[gk] : src[4 * fs];
                    }
                }
            }
        }
    }
}

namespace {

constexpr size_t SMEM_BUDGET = 200 * 1024;

int pick_lines(int pref, int rw, int nf, size_t esz)
{
    int L = pref;
    while (L > 1 && (size_t)nf * rw * (L + 1) * esz > SMEM_BUDGET) L /= 2;
    return L;
}

template <typename T, int MODE, int AXIS>
cudaError_t launch_axis(const LineOpDev &op, LineArgs<T> a, int pref_lines, cudaStream_t st)
{
    constexpr bool SINGLE = MODE == MODE_FIELD || MODE == MODE_FIELD2;
    constexpr int NF = SINGLE ? 1 : (MODE == MODE_VGRAD || MODE == MODE_VDIV ? 4 : 5);
    a.rt = op.max_tile;
    a.rw = op.max_win;
    const int rows = (AXIS != 0 || !SINGLE) ? a.rw : a.rt;
    a.lines = pick_lines(pref_lines, rows, NF, sizeof(T));
    const int kc = sizeof(T) == 8 ? op.kconv64 : op.kconv32;
    const int Na = AXIS == 0 ? a.n[1] : a.n[0];
    const int Nc = AXIS == 2 ? a.n[1] : a.n[2];
    a.ntile_a = (Na + a.lines - 1) / a.lines;
    long long nblk = (long long)op.nsub * a.ntile_a * Nc;
    if (nblk <= 0) return cudaSuccess;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    // extra threads beyond the lines x fields of the solve only stage and
    // store, which keeps more loads in flight per SM (8 per line for the five
    // flux fields, 4 per line for one field: the fastest on GB300)
    int threads = a.lines * NF;
    threads = (threads + 31) / 32 * 32;
    const int per_line = NF == 1 ? 4 : 8;
    if (threads < per_line * a.lines) threads = per_line * a.lines;
    if (threads < 128) threads = 128;
    if (threads > 1024) threads = (a.lines * NF + 31) / 32 * 32;
    if (threads > 1024) return cudaErrorInvalidConfiguration;
    const int rg = (AXIS != 0 || !SINGLE) ? (AXIS == 0 ? 1 : threads / a.lines) : 0;
    const size_t smem = ((size_t)NF * rows * (a.lines + 1) + 2 * (size_t)op.max_taps + 2 * (size_t)kc +
                         (size_t)rg * 2 * NF * a.lines) *
                        sizeof(T);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    line_kernel<T, MODE, AXIS><<<(unsigned)nblk, threads, smem, st>>>(op, a);
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
    return cudaFuncSetAttribute(line_kernel<T, MODE, AXIS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                227 * 1024);
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
