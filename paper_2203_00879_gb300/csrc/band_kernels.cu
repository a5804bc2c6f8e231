// Banded explicit form of the NOHAP first derivative (arXiv 2203.00879, Sec. 3,
// Eqs. CS:fpCf, CS:fpCf_i).
//
// NOHAP takes the two end values of every sub-domain from the equivalent
// explicit scheme g_i = sum_j C_ij f_j, C = A^-1 B truncated where |C_ij| is
// below the working precision, and solves the compact system in between.  The
// banded form applies that explicit scheme at every row: far from the walls
// all rows of C are one translation-invariant stencil (49 taps at the FP32
// threshold, the row the paper tabulates in its appendix), and the rows near
// a wall have their own tabulated windows.  The result equals the NOHAP one
// to within the truncation; there is no recurrence, so every output is an
// independent dot product.
//
// A block stages TR + 2 BH rows of BL neighbouring lines ([row][line], an even
// line pitch so two lines form one 8-byte pair) and each thread computes RC
// consecutive rows of two lines.  Interior rows take their coefficients as
// kernel parameters (constant-bank operands of the FMA); rows near a wall
// read their window from the tabulated rows.  FP32 only: FP64 fields use the
// Thomas form (the 97-tap FP64 stencil is bound by the FP64 pipe).
#include "nopcs_internal.cuh"

namespace nopcs {

namespace {

constexpr int BH = 24;                          // interior half-width of the FP32 stencil
constexpr int BT = 2 * BH + 1;                  // interior taps
constexpr int TR = 64;                          // output rows per block
constexpr int RC = 8;                           // output rows per thread
constexpr int BL = 32;                          // lines per block
constexpr int BTHREADS = (BL / 2) * (TR / RC);  // 16 line pairs x 8 row chunks
constexpr int SR = TR + 2 * BH;                 // staged rows
constexpr int BP = BL + 2;                      // line pitch (even)

struct BandArgs {
    int n[3];
    int N;             // line length
    int ntile_a, nrt;  // line tiles, row tiles
    float scale;       // 1 / h
    const float *in;
    float *out;
    int in_lo, in_hi;  // interior rows
    int h;             // half-width of the stencil (<= BH)
    int W;             // tabulated window width
    const int *wj0;    // per tabulated row: first column of its window
    const int *wlen;   // per tabulated row: window length (<= W)
    const float *wtap; // per tabulated row: W taps
    const float *cg;   // interior stencil (global copy, for rows of mixed chunks)
    float c[BT];       // interior stencil
};

// one output row i near a wall (or next to the interior range), two lines:
// out of line so the unrolled interior loop keeps the instruction cache
__device__ __noinline__ float2 band_row(const BandArgs &a, const float2 *col, int i, int s0)
{
    float sx = 0.0f, sy = 0.0f;
    if (i >= a.in_lo && i <= a.in_hi) {
        for (int t = BH - a.h; t <= BH + a.h; ++t) {
            const float2 v = col[(i - BH + t - s0) * (BP / 2)];
            const float c = __ldg(a.cg + t);
            sx = fmaf(c, v.x, sx);
            sy = fmaf(c, v.y, sy);
        }
    } else {
        const int w = i < a.in_lo ? i : a.in_lo + (i - a.in_hi - 1);
        const int j0 = a.wj0[w], len = a.wlen[w];
        const float *tap = a.wtap + (size_t)w * a.W;
        for (int t = 0; t < len; ++t) {
            const float2 v = col[(j0 + t - s0) * (BP / 2)];
            const float c = __ldg(tap + t);
            sx = fmaf(c, v.x, sx);
            sy = fmaf(c, v.y, sy);
        }
    }
    return make_float2(sx, sy);
}

template <int AXIS>
__global__ void __launch_bounds__(BTHREADS) band_deriv_kernel(const BandArgs a)
{
    __shared__ __align__(16) float sm[SR * BP];
    const int nx = a.n[0], ny = a.n[1], N = a.N;
    const int rt = blockIdx.x % a.nrt;
    const int tile = blockIdx.x / a.nrt;
    const int ta = tile % a.ntile_a;
    const int cc = tile / a.ntile_a;
    const int a0 = ta * BL;
    const int Na = AXIS == 0 ? ny : nx;
    const int nl = min(BL, Na - a0);
    const int r0 = rt * TR;           // first output row
    const int s0 = r0 - BH;           // row of staged row 0
    const int srow = AXIS == 0 ? 1 : (AXIS == 1 ? nx : nx * ny);
    const int sa = AXIS == 0 ? nx : 1;
    const int sc = AXIS == 2 ? nx : nx * ny;
    const int lbase = cc * sc + a0 * sa;

    // ---- stage rows s0 .. s0 + SR - 1 (zeros outside the line) --------------
    // Every thread issues all of its loads before its first shared-memory
    // store, so the whole tile is in flight at once.
    {
        constexpr int NL = AXIS == 0 ? BL / (BTHREADS / 32) : 1;      // lines per thread
        constexpr int NQ = AXIS == 0 ? (SR + 31) / 32 : SR / (BTHREADS / BL);  // rows per line
        const int l0 = AXIS == 0 ? (int)(threadIdx.x >> 5) : (int)(threadIdx.x % BL);
        const int lstep = AXIS == 0 ? BTHREADS / 32 : BL;
        const int q0 = AXIS == 0 ? (int)(threadIdx.x & 31) : (int)(threadIdx.x / BL);
        const int qstep = AXIS == 0 ? 32 : BTHREADS / BL;
        float v[NL][NQ];
#pragma unroll
        for (int li = 0; li < NL; ++li) {
            const int l = l0 + li * lstep;
#pragma unroll
            for (int qi = 0; qi < NQ; ++qi) {
                const int q = q0 + qi * qstep, r = s0 + q;
                v[li][qi] = (q < SR && l < nl && r >= 0 && r < N) ? a.in[lbase + l * sa + r * srow] : 0.0f;
            }
        }
#pragma unroll
        for (int li = 0; li < NL; ++li) {
            const int l = l0 + li * lstep;
#pragma unroll
            for (int qi = 0; qi < NQ; ++qi) {
                const int q = q0 + qi * qstep;
                if (q < SR) sm[q * BP + l] = v[li][qi];
            }
        }
    }
    __syncthreads();

    // ---- RC rows x two lines per thread ---------------------------------------
    const int lp = threadIdx.x % (BL / 2), ch = threadIdx.x / (BL / 2);
    const int rb = r0 + ch * RC;  // first output row of this thread
    const bool live = rb < N && 2 * lp < nl;
    const float2 *col = reinterpret_cast<const float2 *>(sm) + lp;  // staged row q at col[q * BP / 2]
    float ax[RC], ay[RC];
#pragma unroll
    for (int j = 0; j < RC; ++j) ax[j] = ay[j] = 0.0f;
    if (live && rb >= a.in_lo && rb + RC - 1 <= a.in_hi) {
        // interior: output row rb + j sums staged rows (rb - s0) + j - BH + t,
        // t = 0 .. 2 BH, i.e. staged rows ch RC + j + t
#pragma unroll
        for (int k = 0; k < RC + 2 * BH; ++k) {
            const float2 v = col[(ch * RC + k) * (BP / 2)];
#pragma unroll
            for (int j = 0; j < RC; ++j) {
                const int t = k - j;
                if (t >= 0 && t < BT) {
                    ax[j] = fmaf(a.c[t], v.x, ax[j]);
                    ay[j] = fmaf(a.c[t], v.y, ay[j]);
                }
            }
        }
    } else if (live) {
        // rows near a wall (or a chunk straddling the interior edge)
#pragma unroll
        for (int j = 0; j < RC; ++j) {
            const float2 r = rb + j < N ? band_row(a, col, rb + j, s0) : make_float2(0.0f, 0.0f);
            ax[j] = r.x;
            ay[j] = r.y;
        }
    }
    // ---- results through shared memory, then stores coalesced along x ---------
    __syncthreads();  // every thread is done with the staged rows
    if (live) {
#pragma unroll
        for (int j = 0; j < RC; ++j) {
            sm[(ch * RC + j) * BP + 2 * lp] = ax[j] * a.scale;
            sm[(ch * RC + j) * BP + 2 * lp + 1] = ay[j] * a.scale;
        }
    }
    __syncthreads();
    const int nrow = min(TR, N - r0);
    if (AXIS == 0) {  // a warp writes the rows of one line
        for (int l = threadIdx.x >> 5; l < nl; l += BTHREADS / 32)
            for (int q = threadIdx.x & 31; q < nrow; q += 32) a.out[lbase + l * sa + (r0 + q) * srow] = sm[q * BP + l];
    } else {  // consecutive threads write consecutive lines
        const int l = threadIdx.x % BL;
        if (l < nl)
            for (int q = threadIdx.x / BL; q < nrow; q += BTHREADS / BL)
                a.out[lbase + l + (r0 + q) * srow] = sm[q * BP + l];
    }
}

}  // namespace

cudaError_t BandBuf::upload()
{
    release();
    const BandHost &h = host;
    const size_t nw = h.wrow.size();
    const size_t bytes = 2 * nw * sizeof(int) + nw * (size_t)h.W * sizeof(float) + (size_t)BT * sizeof(float) + 64;
    cudaError_t e = dev_alloc(&mem, bytes);
    if (e != cudaSuccess) {
        mem = nullptr;
        return e;
    }
    std::vector<unsigned char> stage(bytes, 0);
    float *cg = reinterpret_cast<float *>(stage.data());  // centred in BT taps
    for (int t = 0; t < BT; ++t) {
        const int k = t - BH + h.h;
        cg[t] = (k >= 0 && k < (int)h.stencil.size()) ? (float)h.stencil[k] : 0.0f;
    }
    int *j0 = reinterpret_cast<int *>(stage.data() + BT * sizeof(float));
    for (size_t i = 0; i < nw; ++i) {
        j0[i] = h.wj0[i];
        j0[nw + i] = h.wlen[i];
    }
    float *tap = reinterpret_cast<float *>(stage.data() + BT * sizeof(float) + 2 * nw * sizeof(int));
    for (size_t i = 0; i < nw * (size_t)h.W; ++i) tap[i] = (float)h.wtap[i];
    e = cudaMemcpy(mem, stage.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    dev.cg = reinterpret_cast<const float *>(mem);
    dev.wj0 = reinterpret_cast<const int *>((const char *)mem + BT * sizeof(float));
    dev.wlen = dev.wj0 + nw;
    dev.wtap = reinterpret_cast<const float *>((const char *)mem + BT * sizeof(float) + 2 * nw * sizeof(int));
    return cudaSuccess;
}

void BandBuf::release()
{
    if (mem) dev_free(mem);
    mem = nullptr;
}

// the kernel's window rules: the interior stencil fits BH, and every
// tabulated row's window lies inside the rows its block stages
bool band_supported(const BandHost &h)
{
    if (h.h > BH) return false;
    for (size_t t = 0; t < h.wrow.size(); ++t) {
        const int i = h.wrow[t], r0 = i / TR * TR;
        const int lo = r0 - BH > 0 ? r0 - BH : 0;
        const int hi = r0 + TR - 1 + BH < h.N - 1 ? r0 + TR - 1 + BH : h.N - 1;
        if (h.wj0[t] < lo || h.wj0[t] + h.wlen[t] - 1 > hi) return false;
    }
    return true;
}

cudaError_t launch_band_field(const BandBuf &op, int axis, const int n[3], const float *f, float *out, double scale,
                              cudaStream_t st)
{
    const BandHost &h = op.host;
    BandArgs a{};
    for (int d = 0; d < 3; ++d) a.n[d] = n[d];
    a.N = n[axis];
    a.nrt = (a.N + TR - 1) / TR;
    const int Na = axis == 0 ? n[1] : n[0];
    const int Nc = axis == 2 ? n[1] : n[2];
    a.ntile_a = (Na + BL - 1) / BL;
    a.scale = (float)scale;
    a.in = f;
    a.out = out;
    a.in_lo = h.in_lo;
    a.in_hi = h.in_hi;
    a.h = h.h;
    a.W = h.W;
    a.wj0 = op.dev.wj0;
    a.wlen = op.dev.wlen;
    a.wtap = op.dev.wtap;
    a.cg = op.dev.cg;
    // the stencil centred in BT taps (zeros beyond the table's half-width)
    for (int t = 0; t < BT; ++t) {
        const int k = t - BH + h.h;
        a.c[t] = (k >= 0 && k < (int)h.stencil.size()) ? (float)h.stencil[k] : 0.0f;
    }
    const long long nblk = (long long)a.nrt * a.ntile_a * Nc;
    if (nblk <= 0) return cudaSuccess;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    switch (axis) {
    case 0: band_deriv_kernel<0><<<(unsigned)nblk, BTHREADS, 0, st>>>(a); break;
    case 1: band_deriv_kernel<1><<<(unsigned)nblk, BTHREADS, 0, st>>>(a); break;
    default: band_deriv_kernel<2><<<(unsigned)nblk, BTHREADS, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace nopcs
