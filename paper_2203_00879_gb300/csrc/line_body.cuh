// Device bodies of the NOHAP line sweeps (arXiv 2203.00879, Sec. 3): the
// sub-domain sweep (line_body) and the whole-line x sweep (xline_body), each
// for one block given as a block index of its launch grid, so that the
// stand-alone kernels (line_kernels.cu) and the batched persistent kernel
// (batch_kernel.cu) run the same code.  The header comment of line_kernels.cu
// describes the algorithm.
#pragma once

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

// One block of the sub-domain sweep: block `vblock` of the launch grid
// (sub-domain vblock % nsub of line tile vblock / nsub), in the block's
// dynamic shared memory, threads 0 .. NT-1 working (a larger block's other
// threads only take part in the barriers, so the arithmetic, and its
// rounding, is that of an NT-thread launch).  The shared array is declared
// here rather than passed in.
template <typename T, int MODE, int AXIS, bool ALL = false>
__device__ __forceinline__ void line_body(const LineOpDev &op, const LineArgs<T> &a, const unsigned vblock,
                                          const int nt_req)
{
    extern __shared__ __align__(32) unsigned char smraw[];
    // ALL: every thread of the block works (the stand-alone launch)
    const int NT = ALL ? (int)blockDim.x : nt_req;
    const bool worker = ALL || (int)threadIdx.x < NT;
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
    const int RG = STREAM ? (AXIS == 0 ? 1 : NT / LINES) : 0;
    // shared memory: end-row taps (2 x max_taps), Thomas factors (2 x KC),
    // end-row partial sums [RG][2][NF][LINES], tile [NF][RW][LP]
    T *cs = reinterpret_cast<T *>(smraw);
    T *ce = cs + op.max_taps;
    T *tcp = ce + op.max_taps;
    T *tiv = tcp + KC;
    T *part = tiv + KC;
    T *sm = part + (size_t)RG * 2 * NF * LINES;
    const int nx = a.n[0], ny = a.n[1];

    // unsigned block index: the compiler then knows the tile coordinates are
    // non-negative (with a signed index the z sweep ran 5% slower)
    const int b = vblock % (unsigned)op.nsub;
    const int tile = vblock / (unsigned)op.nsub;
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
            for (int k = worker ? threadIdx.x : lens; k < lens; k += NT) cs[k] = coef[rec[6] + k];
            for (int k = worker ? threadIdx.x : lene; k < lene; k += NT) ce[k] = coef[rec[9] + k];
        }
        const T *cpp = cp_ptr<T>(op), *ivp = inv_ptr<T>(op);
        for (int k = worker ? threadIdx.x : KC; k < KC; k += NT) {
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
            l0 = worker ? (int)threadIdx.x >> 5 : nl;
            lstep = NT >> 5;
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
            l0 = worker ? (int)threadIdx.x >> 5 : nl;
            lstep = NT >> 5;
        } else {
            l0 = worker ? (int)threadIdx.x % LINES : nl;
            lstep = LINES;
            r0 = threadIdx.x / LINES;
            rstep = NT / LINES;
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

// ---- whole-line sweep along x -------------------------------------------------
// Along x a grid line is contiguous in memory and short enough (N x 5 fields
// x 4 B = 20 KB at N = 1024) for a block to stage LINES whole lines at once.
// Every point is then loaded once -- a sub-domain tile also stages the 2 x 24
// end-row support points of its neighbours, 1.75 times its own points at
// sub-domains of 64 -- and the end rows read their supports from the staged
// lines instead of summing partial products across a warp.  Each thread
// solves one (line, field, sub-domain) column in three phases separated by
// barriers, so that no column reads a row another column has overwritten:
//   A. the two end values g_i = sum_j C_ij f_j (Eq. CS:fpCf_i) and any
//      explicit wall row, from the staged inputs;
//   B. the Thomas solve of the implicit rows in place: it reads rows s-1 ..
//      e+1, and the only rows of other columns among them (s-1 and e+1) are
//      their end rows, which phase B never writes;
//   C. the end and wall values into their rows.
// The layout is [field][line][row] with one pad word per 32 rows and a line
// pitch chosen on the host (LineOpDev::xpitch) so that the columns a warp's
// threads take (neighbouring sub-domains, then the next line) fall in
// different banks.  The line's end-row taps (a few KB) are copied to shared
// memory once per block: the threads of a warp read the taps of different
// sub-domains, which from global memory would touch a cache line each.
__host__ __device__ __forceinline__ int xrow(int g) { return g + (g >> 5); }

// Inviscid flux along x (Eq. ge3) of one point's stage primitives
// v = (rho - rho_b, u, v, w, p, H - H_b) into the tile rows d[k FS], k = 0..4;
// gk is the point's coordinate along gravity.
template <typename T>
__device__ __forceinline__ void xline_flux_point(const LineArgs<T> &a, T *d, const size_t FS, const T v[6],
                                                 const int gk)
{
    const T rho = a.b0[gk] + v[0];
    const T uu = v[1], vv = v[2], ww = v[3], pp = v[4];
    const T H = a.b1[gk] + v[5];
    const T m = rho * uu;
    d[0] = m;
    d[FS] = m * uu + pp;
    d[2 * FS] = m * vv;
    d[3 * FS] = m * ww;
    d[4 * FS] = H * uu;
}

template <typename T, int MODE>
__device__ __forceinline__ void xline_solve_store(const LineOpDev &op, const LineArgs<T> &a, T *sm,
                                                  const T *ctab, const T *tcp, const T *tiv, const int line0,
                                                  const int nl);

// One block of the whole-line x sweep: lines vblock * LINES .. + LINES - 1,
// in the block's dynamic shared memory.
template <typename T, int MODE>
__device__ __forceinline__ void xline_body(const LineOpDev &op, const LineArgs<T> &a, const int vblock)
{
    extern __shared__ __align__(32) unsigned char smraw[];
    constexpr bool SINGLE = MODE == MODE_FIELD;
    constexpr int NF = SINGLE ? 1 : 5;
    constexpr int NIN = SINGLE ? 1 : 6;
    constexpr int U = 4;     // staged points in flight per thread and field
    const int N = op.N;      // = nx
    const int nx = a.n[0], ny = a.n[1];
    const int LINES = a.lines, LS = a.rt;  // lines per block, line pitch (padded)
    const size_t FS = (size_t)LINES * LS;
    const int KC = sizeof(T) == 8 ? op.kconv64 : op.kconv32;
    T *sm = reinterpret_cast<T *>(smraw);
    T *ctab = sm + NF * FS;  // end-row taps
    T *tcp = ctab + op.ncoef;
    T *tiv = tcp + KC;
    const int line0 = vblock * LINES;
    const int nl = min(LINES, ny * a.n[2] - line0);
    {
        const T *cpp = cp_ptr<T>(op), *ivp = inv_ptr<T>(op), *cf = coef_ptr<T>(op);
        for (int k = threadIdx.x; k < KC; k += blockDim.x) {
            tcp[k] = cpp[k];
            tiv[k] = ivp[k];
        }
        for (int k = threadIdx.x; k < op.ncoef; k += blockDim.x) ctab[k] = cf[k];
    }
    // ---- stage the lines: consecutive threads take consecutive points ----
    for (int l = 0; l < nl; ++l) {
        const int line = line0 + l;  // = y + ny z
        const int gl = a.ga == 1 ? line % ny : line / ny;  // coordinate along gravity (y or z)
        const int base = line * nx;
        for (int g0 = threadIdx.x; g0 < N; g0 += U * blockDim.x) {
            T v[U][NIN];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int g = g0 + u * (int)blockDim.x;
                if (g < N) {
#pragma unroll
                    for (int k = 0; k < NIN; ++k) v[u][k] = a.in[k][base + g];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int g = g0 + u * (int)blockDim.x;
                if (g >= N) continue;
                T *d = sm + (size_t)l * LS + xrow(g);
                if constexpr (SINGLE) {
                    d[0] = v[u][0];
                } else {
                    xline_flux_point(a, d, FS, v[u], a.ga == 0 ? g : gl);
                }
            }
        }
    }
    __syncthreads();
    xline_solve_store<T, MODE>(op, a, sm, ctab, tcp, tiv, line0, nl);
}

// The solve and the store of the whole-line x sweep, once lines line0 ..
// line0 + nl - 1 are staged in the tile sm (and a barrier has passed): the
// columns, thread c solving sub-domain c % nsub of line (c / nsub) % nl, field
// c / (nsub nl), in phases A-C, then the rows scaled by 1/h into the outputs.
template <typename T, int MODE>
__device__ __forceinline__ void xline_solve_store(const LineOpDev &op, const LineArgs<T> &a, T *sm,
                                                  const T *ctab, const T *tcp, const T *tiv, const int line0,
                                                  const int nl)
{
    constexpr bool SINGLE = MODE == MODE_FIELD;
    constexpr int NF = SINGLE ? 1 : 5;
    constexpr int NEXP = 2;  // explicit rows at each wall (derivative)
    const int N = op.N;      // = nx
    const int nx = a.n[0];
    const int LINES = a.lines, LS = a.rt;
    const size_t FS = (size_t)LINES * LS;
    const int KC = sizeof(T) == 8 ? op.kconv64 : op.kconv32;
    const int nsub = op.nsub;
    const int c = threadIdx.x;
    const bool active = c < nsub * NF * nl;
    const int b = c % nsub, l = (c / nsub) % max(nl, 1), f = c / (nsub * max(nl, 1));
    const int *rec = op.sub + b * SUB_REC;
    T *col = sm + (size_t)f * FS + (size_t)l * LS;
    const int s = rec[0], e = rec[1], lo = rec[10], hi = rec[11];
    T gs = 0, ge = 0;
    T exL[NEXP], exH[NEXP];
#pragma unroll
    for (int r = 0; r < NEXP; ++r) exL[r] = exH[r] = T(0);
    // A. end values and explicit wall rows from the staged inputs
    if (active) {
        const T *coef = ctab;
        auto dot = [&](const T *cf, int j0, int len) {
            T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
            int k = 0;
            for (; k + 4 <= len; k += 4) {
                s0 += cf[k] * col[xrow(j0 + k)];
                s1 += cf[k + 1] * col[xrow(j0 + k + 1)];
                s2 += cf[k + 2] * col[xrow(j0 + k + 2)];
                s3 += cf[k + 3] * col[xrow(j0 + k + 3)];
            }
            for (; k < len; ++k) s0 += cf[k] * col[xrow(j0 + k)];
            return (s0 + s1) + (s2 + s3);
        };
        gs = dot(coef + rec[6], rec[4], rec[5]);
        if (rec[8] > 0) ge = dot(coef + rec[9], rec[7], rec[8]);
#pragma unroll
        for (int r = 0; r < NEXP; ++r) {
            if (r > s && r < e) {
                T acc = 0;
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    if (op.ex[r][j] != 0.0) acc += (T)op.ex[r][j] * col[xrow(j)];
                exL[r] = acc;
            }
            const int rh = N - 1 - r;
            if (rh > s && rh < e) {
                T acc = 0;
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    if (op.ex[r][j] != 0.0) acc += (T)op.ex[r][j] * col[xrow(N - 1 - j)];
                exH[r] = (T)op.ex_sign * acc;
            }
        }
    }
    __syncthreads();
    // B. Thomas over the implicit rows lo..hi, forward values in place; a
    // register window keeps the inputs rows i-2 .. i+2 that row i reads
    if (active && lo <= hi) {
        const int m = hi - lo + 1;
        const T al = (T)op.alpha;
        const T gL = lo == s + 1 ? gs : exL[NEXP - 1];
        const T gR = hi == e - 1 ? ge : exH[NEXP - 1];
        const T r0 = (T)op.rb[0], r1 = (T)op.rb[1];
        const T cL = (T)op.cpL, iL = (T)op.invL;
        T win[5];
#pragma unroll
        for (int j = 0; j < 4; ++j) win[j] = col[xrow(lo - 2 + j)];
        int gin = lo + 2, gout = lo;
        T dprev = 0;
        auto fwd = [&](T iv, T adj) {
            win[4] = col[xrow(gin)];
            ++gin;
            const T rhs = r0 * (win[3] - win[1]) + r1 * (win[4] - win[0]);
            const T dp = (rhs - adj - al * dprev) * iv;
            col[xrow(gout)] = dp;
            ++gout;
            dprev = dp;
#pragma unroll
            for (int j = 0; j < 4; ++j) win[j] = win[j + 1];
        };
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
        int g = hi - 1;
        r = m - 2;
#pragma unroll 4
        for (; r >= KC; --r, --g) {
            x = col[xrow(g)] - cL * x;
            col[xrow(g)] = x;
        }
#pragma unroll 4
        for (; r >= 0; --r, --g) {
            x = col[xrow(g)] - tcp[r] * x;
            col[xrow(g)] = x;
        }
    }
    __syncthreads();
    // C. end values and wall rows into their rows
    if (active) {
        col[xrow(s)] = gs;
        if (rec[8] > 0) col[xrow(e)] = ge;
#pragma unroll
        for (int r = 0; r < NEXP; ++r) {
            if (r > s && r < e) col[xrow(r)] = exL[r];
            const int rh = N - 1 - r;
            if (rh > s && rh < e) col[xrow(rh)] = exH[r];
        }
    }
    __syncthreads();
    // ---- store (scaled by 1/h; the flux sweep stores -dF/dx into R) ----
    for (int ll = 0; ll < nl; ++ll) {
        const int base = (line0 + ll) * nx;
        const T *src = sm + (size_t)ll * LS;
        for (int g = threadIdx.x; g < N; g += blockDim.x) {
            const int o = base + g;
            const int q = xrow(g);
            if constexpr (SINGLE) {
                a.out[0][o] = src[q] * a.scale;
            } else {
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const T v = -src[(size_t)k * FS + q] * a.scale;
                    if (a.first)
                        a.out[k][o] = v;
                    else
                        atomicAdd(&a.out[k][o], v);
                }
            }
        }
    }
}


// ---- launch geometry (host) ----------------------------------------------------
constexpr size_t SMEM_BUDGET = 200 * 1024;
// whole-line x sweep: at most this much shared memory per block, and several
// lines per block only while a block stays below the second figure.  One line
// per block measured fastest for the five-field flux sweep at 1024^3 (14.73 ms
// against 16.02 with two lines and 15.62 for the sub-domain tiles); for a
// single field the sub-domain tiles stay faster (0.46 ms at 512^3 against 0.50
// with four lines and 1.42 with one), so FIELD keeps them.
constexpr size_t XLINE_SMEM = 100 * 1024, XLINE_SMEM_MULTI = 48 * 1024;
#ifndef XLINE_MAX_LINES
#define XLINE_MAX_LINES 1
#endif

inline int pick_lines(int pref, int rw, int nf, size_t esz)
{
    int L = pref;
    while (L > 1 && (size_t)nf * rw * (L + 1) * esz > SMEM_BUDGET) L /= 2;
    return L;
}

struct LineGrid {
    long long nblk = 0;  // blocks
    int threads = 0;
    size_t smem = 0;     // dynamic shared memory per block
    bool xline = false;  // the whole-line x kernel runs
};

// Geometry of one sweep along AXIS: fills a.lines, a.ntile_a, a.rt, a.rw.
// threads_req > 0 fixes the block size (the batched kernel's); max_xlines
// bounds the lines per block of the whole-line x kernel (FLUX along x only),
// which needs one thread per (line, field, sub-domain) column.  False if no
// configuration fits.
template <typename T, int MODE, int AXIS>
bool line_grid(const LineOpDev &op, LineArgs<T> &a, int pref_lines, int threads_req, int max_xlines, LineGrid &g)
{
    constexpr bool SINGLE = MODE == MODE_FIELD || MODE == MODE_FIELD2;
    constexpr int NF = SINGLE ? 1 : (MODE == MODE_VGRAD || MODE == MODE_VDIV ? 4 : 5);
    const int kc = sizeof(T) == 8 ? op.kconv64 : op.kconv32;
    g = LineGrid();
    // the whole-line kernel needs enough (field, sub-domain) columns per line
    // to keep a block busy in its solve: at 256^3 (20 columns) it was 1.7 times
    // slower than the sub-domain tiles, at 1024^3 (80 columns) 6% faster
    if (AXIS == 0 && MODE == MODE_FLUX && op.nsub * NF >= 64) {
        for (int L = max_xlines < 4 ? max_xlines : 4; L >= 1; --L) {
            const int pitch = op.xpitch[1][L - 1];
            const size_t bytes = ((size_t)NF * L * pitch + (size_t)op.ncoef + 2 * (size_t)kc) * sizeof(T);
            const int cols = op.nsub * NF * L;
            const int cap = threads_req > 0 ? threads_req : 1024;
            if (bytes > XLINE_SMEM || cols > cap) continue;
            if (L > 1 && bytes > XLINE_SMEM_MULTI) continue;
            a.lines = L;
            a.rt = pitch;
            int threads = (cols + 31) / 32 * 32;
            if (threads < 128) threads = 128;
            g.threads = threads_req > 0 ? threads_req : threads;
            g.smem = bytes;
            g.xline = true;
            g.nblk = ((long long)a.n[1] * a.n[2] + L - 1) / L;
            return g.nblk <= 0x7fffffffLL;
        }
    }
    a.rt = op.max_tile;
    a.rw = op.max_win;
    const int rows = (AXIS != 0 || !SINGLE) ? a.rw : a.rt;
    a.lines = pick_lines(pref_lines, rows, NF, sizeof(T));
    if (threads_req > 0)
        while (a.lines > 1 && a.lines * NF > threads_req) a.lines /= 2;
    const int Na = AXIS == 0 ? a.n[1] : a.n[0];
    const int Nc = AXIS == 2 ? a.n[1] : a.n[2];
    a.ntile_a = (Na + a.lines - 1) / a.lines;
    g.nblk = (long long)op.nsub * a.ntile_a * Nc;
    if (g.nblk > 0x7fffffffLL) return false;
    // extra threads beyond the lines x fields of the solve only stage and
    // store, which keeps more loads in flight per SM (8 per line for the five
    // flux fields, 4 per line for one field: the fastest on GB300)
    int threads = a.lines * NF;
    threads = (threads + 31) / 32 * 32;
    const int per_line = NF == 1 ? 4 : 8;
    if (threads < per_line * a.lines) threads = per_line * a.lines;
    if (threads < 128) threads = 128;
    if (threads > 1024) threads = (a.lines * NF + 31) / 32 * 32;
    if (threads > 1024) return false;
    if (threads_req > 0) threads = threads_req;
    const int rg = (AXIS != 0 || !SINGLE) ? (AXIS == 0 ? 1 : threads / a.lines) : 0;
    g.threads = threads;
    g.smem = ((size_t)NF * rows * (a.lines + 1) + 2 * (size_t)op.max_taps + 2 * (size_t)kc +
              (size_t)rg * 2 * NF * a.lines) *
             sizeof(T);
    return g.smem <= 227 * 1024;
}

// The whole-line x flux kernel lives in its own translation unit
// (xline_kernels.cu).
template <typename T>
cudaError_t launch_xline_flux(const LineOpDev &op, const LineArgs<T> &a, long long nblk, int threads, size_t smem,
                              cudaStream_t st);
template <typename T>
cudaError_t init_xline_flux();

}  // namespace nopcs
