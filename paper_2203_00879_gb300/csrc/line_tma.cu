// NOHAP flux sweeps along y and z with TMA staging (arXiv 2203.00879, Sec. 3;
// fluxes of Eqs. ge6-ge8).
//
// Along y and z a grid line is strided in memory while x is contiguous, so a
// block's tile -- TL = 32 neighbouring x lines by the rt rows its sub-domain
// needs -- is a dense 4-D box (x, y, z, field) of the primitive array W.  One
// thread loads the whole box of all six W fields with a single tensor copy
// (cp.async.bulk.tensor) into shared memory laid out [field][row][line], which
// is the column layout the solve wants (consecutive threads, consecutive
// lines).  The block then
//   1. turns the six primitives of every staged node into the five fluxes of
//      this axis, in place,
//   2. solves each (line, field) column (the NOHAP solve shared with the
//      register-staged kernel), leaving -L(flux)/h in place, and
//   3. adds its own rows to R with tensor reduce-add copies
//      (cp.reduce.async.bulk.tensor .add), eight rows per copy; rows left
//      over when the sub-domain length is not a multiple of eight are added
//      by the threads.
// No thread holds a load in flight, so the copy engine keeps the whole tile's
// traffic outstanding at once.  Requirements (checked by the launcher, which
// otherwise uses the register-staged kernel): FP32, x extent a multiple of 4
// (16-byte strides), at most 256 staged rows.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "line_solve.cuh"

namespace nopcs {

namespace {

constexpr int TL = 32;               // lines per block: one 128-byte x segment
constexpr int TTHREADS = 256;
constexpr int RCHUNK = 8;            // rows per reduce-add copy
constexpr long long TMA_WAIT_ITERS = 1LL << 22;

struct TmaArgs {
    int n[3];
    int ntile_a;   // tiles along x
    int rt;        // staged rows per tile (box height)
    float nscale;  // -1/h
    int first;     // 1: store R, 0: add to R
    int ga;        // gravity axis
    const float *b0, *b1;  // rho_b, H_b
    float *R;              // 5 fields of np points: rows left over by the chunked copies
    long long np;
    int *err;
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// AXIS 1: rows along y, tiles (x, z); AXIS 2: rows along z, tiles (x, y)
template <int AXIS>
__global__ void __launch_bounds__(TTHREADS) flux_tma_kernel(const LineOpDev op, const TmaArgs a,
                                                            const __grid_constant__ CUtensorMap wmap,
                                                            const __grid_constant__ CUtensorMap rmap)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    float *sm = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~(uintptr_t)127);
    const int RT = a.rt, KC = op.kconv32;
    const int fs = RT * TL;  // field stride of the tile
    float *cs = sm + 6 * fs;
    float *ce = cs + op.max_taps;
    float *tcp = ce + op.max_taps;
    float *tiv = tcp + KC;
    uint64_t *bar = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(tiv + KC) + 7) & ~(uintptr_t)7);

    const int b = blockIdx.x % op.nsub;
    const int tile = blockIdx.x / op.nsub;
    const int ta = tile % a.ntile_a;
    const int cc = tile / a.ntile_a;  // z for AXIS 1, y for AXIS 2
    const int a0 = ta * TL;
    const int nl = min(TL, a.n[0] - a0);
    const int *rec = op.sub + b * SUB_REC;
    const int s = rec[0], e = rec[1], tlo = rec[2], thi = rec[3];
    const int lens = rec[5], lene = rec[8];
    const int nrows = thi - tlo + 1;

    // ---- 1. one tensor copy of the (TL x RT x 6) box of W --------------------
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)(6u * fs * sizeof(float));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes)
                     : "memory");
        const int c1 = AXIS == 1 ? tlo : cc, c2 = AXIS == 1 ? cc : tlo;
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(su32(sm)),
            "l"(reinterpret_cast<uint64_t>(&wmap)), "r"(a0), "r"(c1), "r"(c2), "r"(0), "r"(su32(bar))
            : "memory");
    }
    // block constants while the tile is in flight
    for (int k = threadIdx.x; k < lens; k += blockDim.x) cs[k] = op.coef32[rec[6] + k];
    for (int k = threadIdx.x; k < lene; k += blockDim.x) ce[k] = op.coef32[rec[9] + k];
    for (int k = threadIdx.x; k < KC; k += blockDim.x) {
        tcp[k] = op.cp32[k];
        tiv[k] = op.inv32[k];
    }
    bool ok = false;
    for (long long it = 0; it < TMA_WAIT_ITERS && !ok; ++it) ok = bar_try_wait(su32(bar), 0);
    if (!__syncthreads_and(ok)) {
        // the copy did not land: flag it, give it one more bounded wait, leave
        if (threadIdx.x == 0) {
            atomicExch(a.err, 1);
            bool done = false;
            for (long long it = 0; it < TMA_WAIT_ITERS && !done; ++it) done = bar_try_wait(su32(bar), 0);
        }
        __syncthreads();
        return;
    }

    // ---- 2. fluxes of this axis in place (Eqs. ge6-ge8, inviscid part) -------
    {
        const int gsel = a.ga == AXIS ? 0 : (a.ga == 0 ? 1 : 2);  // row, line (x) or cc
        for (int idx = threadIdx.x; idx < nrows * TL; idx += blockDim.x) {
            const int r = idx / TL, l = idx % TL;
            if (l >= nl) continue;
            float *d = sm + r * TL + l;
            const int gk = gsel == 0 ? tlo + r : (gsel == 1 ? a0 + l : cc);
            const float rho = a.b0[gk] + d[0];
            const float uu = d[fs], vv = d[2 * fs], ww = d[3 * fs], pp = d[4 * fs];
            const float H = a.b1[gk] + d[5 * fs];
            const float ud = AXIS == 1 ? vv : ww;
            const float m = rho * ud;
            d[0] = m;
            d[fs] = m * uu;
            d[2 * fs] = m * vv + (AXIS == 1 ? pp : 0.0f);
            d[3 * fs] = m * ww + (AXIS == 2 ? pp : 0.0f);
            d[4 * fs] = H * ud;
        }
    }
    __syncthreads();

    // ---- 3. per-(line, field) NOHAP solve, scaled by -1/h ----------------------
    {
        const int l = threadIdx.x % TL, fld = threadIdx.x / TL;
        if (l < nl && fld < 5)
            nohap_solve_column<float, MODE_FLUX, true>(op, sm + (size_t)fld * fs + l, TL, cs, ce, tcp, tiv, KC, rec,
                                                       a.nscale);
    }
    // generic-proxy writes of the tile become visible to the tensor copies
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();

    // ---- 4. own rows into R: reduce-add (or store) copies of 8 rows ------------
    const int nown = e - s + 1, nch = nown / RCHUNK;
    if (threadIdx.x < 5) {
        const int f = threadIdx.x;
        for (int j = 0; j < nch; ++j) {
            const int row = s + RCHUNK * j;
            const float *src = sm + (size_t)f * fs + (size_t)(row - tlo) * TL;
            const int c1 = AXIS == 1 ? row : cc, c2 = AXIS == 1 ? cc : row;
            if (a.first)
                asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                                 reinterpret_cast<uint64_t>(&rmap)),
                             "r"(a0), "r"(c1), "r"(c2), "r"(f), "r"(su32(src))
                             : "memory");
            else
                asm volatile(
                    "cp.reduce.async.bulk.tensor.4d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3, %4}], "
                    "[%5];" ::"l"(reinterpret_cast<uint64_t>(&rmap)),
                    "r"(a0), "r"(c1), "r"(c2), "r"(f), "r"(su32(src))
                    : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    // leftover rows (nown mod 8) by the threads
    {
        const int r0 = s + RCHUNK * nch, nrag = e - r0 + 1;
        const int nx = a.n[0], ny = a.n[1];
        for (int idx = threadIdx.x; idx < 5 * nrag * TL; idx += blockDim.x) {
            const int l = idx % TL, r = (idx / TL) % nrag, f = idx / (TL * nrag);
            if (l >= nl) continue;
            const int row = r0 + r;
            const int gi = AXIS == 1 ? (a0 + l) + nx * (row + ny * cc) : (a0 + l) + nx * (cc + ny * row);
            const float v = sm[(size_t)f * fs + (size_t)(row - tlo) * TL + l];
            float *o = a.R + (size_t)f * a.np + gi;
            *o = a.first ? v : *o + v;
        }
    }
    if (threadIdx.x < 5) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(su32(bar)) : "memory");
}

size_t tma_smem_bytes(const LineOpDev &op)
{
    return 128 + ((size_t)6 * op.max_tile * TL + 2 * (size_t)op.max_taps + 2 * (size_t)op.kconv32) * sizeof(float) +
           16;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 4-D FP32 map over (x, y, z, field) of an array of nf fields, box
// (TL, rows along AXIS, 1 along the other, bf fields)
bool encode_map(CUtensorMap *m, const BoxDev &bx, int axis, const float *base, int nf, int rows, int bf)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)bx.n[0], (cuuint64_t)bx.n[1], (cuuint64_t)bx.n[2], (cuuint64_t)nf};
    const cuuint64_t strides[3] = {(cuuint64_t)bx.n[0] * 4, (cuuint64_t)bx.n[0] * bx.n[1] * 4,
                                   (cuuint64_t)bx.np * 4};
    const cuuint32_t box[4] = {(cuuint32_t)TL, (cuuint32_t)(axis == 1 ? rows : 1), (cuuint32_t)(axis == 2 ? rows : 1),
                               (cuuint32_t)bf};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int AXIS>
cudaError_t launch_axis_tma(const LineOpDev &op, const BoxDev &bx, const float *W, float *R, int first,
                            cudaStream_t st)
{
    CUtensorMap wmap, rmap;
    if (!encode_map(&wmap, bx, AXIS, W, 6, op.max_tile, 6) || !encode_map(&rmap, bx, AXIS, R, 5, RCHUNK, 1))
        return cudaErrorNotSupported;
    TmaArgs a{};
    for (int d = 0; d < 3; ++d) a.n[d] = bx.n[d];
    a.ntile_a = (bx.n[0] + TL - 1) / TL;
    a.rt = op.max_tile;
    a.nscale = (float)(-bx.inv_h[AXIS]);
    a.first = first;
    a.ga = bx.ga;
    a.b0 = bx.rho_b32;
    a.b1 = bx.H_b32;
    a.R = R;
    a.np = bx.np;
    a.err = bx.err;
    const int Nc = AXIS == 2 ? bx.n[1] : bx.n[2];
    const long long nblk = (long long)op.nsub * a.ntile_a * Nc;
    if (nblk <= 0) return cudaSuccess;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    flux_tma_kernel<AXIS><<<(unsigned)nblk, TTHREADS, tma_smem_bytes(op), st>>>(op, a, wmap, rmap);
    return cudaGetLastError();
}

}  // namespace

bool flux_tma_usable(const LineOpDev &op, const BoxDev &bx, int axis, const void *W, const void *R)
{
    return (axis == 1 || axis == 2) && bx.n[0] % 4 == 0 && op.max_tile <= 256 && bx.err != nullptr &&
           (reinterpret_cast<uintptr_t>(W) % 16) == 0 && (reinterpret_cast<uintptr_t>(R) % 16) == 0 &&
           tma_smem_bytes(op) <= 227 * 1024 && encode_fn() != nullptr;
}

cudaError_t launch_flux_tma(const LineOpDev &op, int axis, const BoxDev &bx, const float *W, float *R, int first,
                            cudaStream_t st)
{
    return axis == 1 ? launch_axis_tma<1>(op, bx, W, R, first, st) : launch_axis_tma<2>(op, bx, W, R, first, st);
}

cudaError_t init_tma_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(flux_tma_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(flux_tma_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace nopcs
