// Tensor-core form of the NOHAP derivative (arXiv 2203.00879, Sec. 3).
//
// NOHAP makes every sub-domain's result a fixed linear map of the inputs in
// its staging window: the end rows are rows of C = A^-1 B and the interior is
// a Thomas solve, both linear.  So sub-domain b is g = D_b f_window with a
// small dense D_b (n_b outputs x Kpad window points, built on the host by
// applying the line algorithm to unit vectors), and the derivative of 128
// neighbouring lines is one dense contraction
//     OUT (128 lines x n_b) = F (128 lines x Kpad) . D_b^T (Kpad x n_b)
// on the 5th-generation tensor cores, FP32 accumulation in tensor memory, in
// one of two split precisions:
//   - "3xTF32" (tcgen05.mma kind::tf32, M = 128, N = Npad, K = 8 per
//     instruction): F = F_hi + F_lo and D = D_hi + D_lo with TF32 parts;
//     OUT = F_hi D_hi + F_hi D_lo + F_lo D_hi recovers ~21 bits;
//   - "BF16x3" (kind::f16 with BF16 operands, K = 16 per instruction):
//     F = F1 + F2 + F3 and D = D1 + D2 + D3 with BF16 parts (8 bits each);
//     OUT = sum of F_i D_j over i + j <= 4 (six products) keeps every term
//     down to 2^-16 of the leading one, FP32 level (~24 bits).
//
// Both operands sit in shared memory in the K-major, non-swizzled canonical
// layout of tcgen05: 8-row x 16-byte core matrices, contiguous along K
// (leading byte offset 128) and SBO bytes apart along M/N.  One thread issues
// the MMAs and commits them to an mbarrier; the block waits on it with an
// iteration bound, then each warp reads its 32 accumulator lanes with
// tcgen05.ld and stores them.
#include <cuda_bf16.h>
#include <stdint.h>

#include "nopcs_internal.cuh"

namespace nopcs {

namespace {

constexpr int GM = 128;       // lines per block (MMA M)
constexpr int KC = 32;        // window points per pipeline stage (4 MMA K-steps)
constexpr int A_PAD = 32;     // bytes added to A's 8-row stride (bank spread)
constexpr long long WAIT_ITERS = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for this architecture
    return d;                // base offset 0, relative LBO, layout type 0 (no swizzle)
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_tf32(int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(GM >> 4) << 24);
}

// instruction descriptor of kind::f16: D = F32, A = B = BF16 (format code 1;
// the two operands always share one type), both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(GM >> 4) << 24);
}

// the three BF16 parts of x (round to nearest even), packed in 16-bit words
__device__ __forceinline__ void bf16_parts(float x, uint16_t &p1, uint16_t &p2, uint16_t &p3)
{
    const __nv_bfloat16 a = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(a);
    const __nv_bfloat16 b = __float2bfloat16_rn(r1);
    const __nv_bfloat16 c = __float2bfloat16_rn(r1 - __bfloat162float(b));
    p1 = __bfloat16_as_ushort(a);
    p2 = __bfloat16_as_ushort(b);
    p3 = __bfloat16_as_ushort(c);
}

// nearest TF32 value (round to nearest, ties away), kept in an FP32 container
__device__ __forceinline__ float tf32_part(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_bf16(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// pack eight 16-bit words, element 0 at the lowest address
__device__ __forceinline__ uint4 pack8(const uint16_t w[8])
{
    return make_uint4((uint32_t)w[0] | ((uint32_t)w[1] << 16), (uint32_t)w[2] | ((uint32_t)w[3] << 16),
                      (uint32_t)w[4] | ((uint32_t)w[5] << 16), (uint32_t)w[6] | ((uint32_t)w[7] << 16));
}

// BF = false: 3xTF32; BF = true: BF16x3.  A core matrix row is 16 bytes: 4
// TF32 or 8 BF16 window points; one MMA spans two core matrices along K.
template <int AXIS, bool BF>
__global__ void __launch_bounds__(GM) gemm_deriv_kernel(const GemmOpDev op, int nx, int ny, int nz, int ntile_a,
                                                        const float *__restrict__ f, float *__restrict__ out,
                                                        float scale, int *err)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int NP = BF ? 3 : 2;     // operand parts
    constexpr int ESZ = BF ? 2 : 4;    // bytes per element
    constexpr int CME = 16 / ESZ;      // window points per core-matrix row
    constexpr int KMMA = 2 * CME;      // window points per MMA
    const int b = blockIdx.x % op.nsub;
    const int tile = blockIdx.x / op.nsub;
    const int ta = tile % ntile_a, cc = tile / ntile_a;
    const int a0 = ta * GM;
    const int Na = AXIS == 0 ? ny : nx;
    const int nl = min(GM, Na - a0);
    const int N = op.N;
    const int *rec = op.rec + b * DENSE_REC;
    const int s = rec[0], nb = rec[1], npad = rec[2], wlo = rec[4];
    const int kpad = BF ? rec[6] : rec[3], boff = BF ? rec[7] : rec[5];
    // per stage: NP parts of the A chunk (128 x KC) and of the B chunk (npad x KC)
    constexpr uint32_t SBO_A = (KC / CME) * 128u + A_PAD, SBO_B = (KC / CME) * 128u;
    constexpr uint32_t ABYTES = 16u * SBO_A;
    const uint32_t bbytes = (uint32_t)npad * KC * ESZ;
    const uint32_t stage_bytes = NP * ABYTES + NP * bbytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smraw + 2u * stage_bytes);  // one per stage
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5;
    int ncols = 32;
    while (ncols < npad) ncols <<= 1;
    const int nchunk = kpad / KC + (kpad % KC ? 1 : 0);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    const long long srow = AXIS == 0 ? 1 : (AXIS == 1 ? (long long)nx : (long long)nx * ny);
    const long long sa = AXIS == 0 ? (long long)nx : 1;
    const long long sc = AXIS == 2 ? (long long)nx : (long long)nx * ny;
    const long long gbase = (long long)cc * sc + (long long)a0 * sa;
    // Every row of D_b sums to zero (the operator annihilates constants), so
    // each line's window is shifted by its value at the sub-domain start before
    // the split: the same result, with less cancellation in the contraction.
    float c0 = 0.0f;
    if (AXIS != 0 && tid < nl) c0 = f[gbase + (long long)s * srow + tid];
    const uint32_t idesc = BF ? idesc_bf16(npad) : idesc_tf32(npad);
    // ok: every bounded wait of this thread so far succeeded; issued: the last
    // chunk whose MMAs were issued and committed (-1: none)
    bool ok = true;
    int issued = -1;
    for (int c = 0; c < nchunk; ++c) {
        const int st = c & 1;
        unsigned char *A0 = smraw + st * stage_bytes;  // part q at A0 + q ABYTES
        unsigned char *B0 = A0 + NP * ABYTES;          // part q at B0 + q bbytes
        // the MMAs of chunk c - 2 read this stage: wait for their commit
        if (c >= 2) {
            bool done = false;
            for (long long it = 0; it < WAIT_ITERS && !done; ++it)
                done = mbar_try_wait(smem_u32(mbar + st), (uint32_t)(((c - 2) >> 1) & 1));
            ok = ok && done;
        }
        const int k0 = c * KC;
        // B chunk: core matrices k0/CME .. k0/CME + KC/CME of every 8-row group
        {
            const int ncm = KC / CME;             // core matrices per group in a chunk
            const int nq = (npad / 8) * ncm * 8;  // 16-byte rows per part
            for (int i = tid; i < nq; i += GM) {
                const int g = i / (ncm * 8), rem = i % (ncm * 8), cm = rem / 8, row = rem % 8;
                const int kc = k0 / CME + cm;
                const uint32_t so = (uint32_t)g * SBO_B + (uint32_t)cm * 128u + row * 16u;
                if constexpr (BF) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        uint4 v = make_uint4(0u, 0u, 0u, 0u);
                        if (kc < kpad / 8) {
                            const size_t go = (size_t)boff + (size_t)g * (kpad / 8) * 64 + (size_t)kc * 64 + row * 8;
                            v = *reinterpret_cast<const uint4 *>(op.b16[q] + go);
                        }
                        *reinterpret_cast<uint4 *>(B0 + q * bbytes + so) = v;
                    }
                } else {
                    float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
                    if (kc < kpad / 4) {
                        const size_t go = (size_t)boff + (size_t)g * (kpad / 4) * 32 + (size_t)kc * 32 + row * 4;
                        h = *reinterpret_cast<const float4 *>(op.hi + go);
                        l = *reinterpret_cast<const float4 *>(op.lo + go);
                    }
                    *reinterpret_cast<float4 *>(B0 + so) = h;
                    *reinterpret_cast<float4 *>(B0 + bbytes + so) = l;
                }
            }
        }
        // A chunk: the lines' window points k0 .. k0 + KC - 1, split into parts
        if (AXIS == 0) {
            for (int q = tid; q < GM * KC; q += GM) {
                const int m = q / KC, k = q % KC;
                const int pos = wlo + k0 + k;
                float v = 0.0f;
                if (m < nl && pos < N && k0 + k < kpad)
                    v = f[gbase + (long long)m * sa + pos] - f[gbase + (long long)m * sa + s];
                const uint32_t o = (uint32_t)(m >> 3) * SBO_A + (uint32_t)(k / CME) * 128u + (m & 7) * 16u +
                                   (uint32_t)(k % CME) * ESZ;
                if constexpr (BF) {
                    uint16_t p1, p2, p3;
                    bf16_parts(v, p1, p2, p3);
                    *reinterpret_cast<uint16_t *>(A0 + o) = p1;
                    *reinterpret_cast<uint16_t *>(A0 + ABYTES + o) = p2;
                    *reinterpret_cast<uint16_t *>(A0 + 2 * ABYTES + o) = p3;
                } else {
                    const float h = tf32_part(v), l = tf32_part(v - h);
                    *reinterpret_cast<float *>(A0 + o) = h;
                    *reinterpret_cast<float *>(A0 + ABYTES + o) = l;
                }
            }
        } else {
            const int m = tid;
#pragma unroll 2
            for (int kr = 0; kr < KC; kr += CME) {  // one core-matrix row per pass
                float v[CME];
#pragma unroll
                for (int t = 0; t < CME; ++t) {
                    const int pos = wlo + k0 + kr + t;
                    v[t] = (m < nl && pos < N && k0 + kr + t < kpad) ? f[gbase + (long long)pos * srow + m] - c0 : 0.0f;
                }
                const uint32_t o = (uint32_t)(m >> 3) * SBO_A + (uint32_t)(kr / CME) * 128u + (m & 7) * 16u;
                if constexpr (BF) {
                    uint16_t w[3][8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) bf16_parts(v[t], w[0][t], w[1][t], w[2][t]);
#pragma unroll
                    for (int q = 0; q < 3; ++q) *reinterpret_cast<uint4 *>(A0 + q * ABYTES + o) = pack8(w[q]);
                } else {
                    float4 h, l;
                    h.x = tf32_part(v[0]);
                    h.y = tf32_part(v[1]);
                    h.z = tf32_part(v[2]);
                    h.w = tf32_part(v[3]);
                    l.x = tf32_part(v[0] - h.x);
                    l.y = tf32_part(v[1] - h.y);
                    l.z = tf32_part(v[2] - h.z);
                    l.w = tf32_part(v[3] - h.w);
                    *reinterpret_cast<float4 *>(A0 + o) = h;
                    *reinterpret_cast<float4 *>(A0 + ABYTES + o) = l;
                }
            }
        }
        // generic-proxy shared stores -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        // the block agrees whether every wait so far succeeded; after a wait
        // gave up, no further MMA is issued (the stores above may have hit a
        // stage still being read: shared memory only, and the result is
        // discarded)
        if (!__syncthreads_and(ok ? 1 : 0)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int ksteps = min(KC, kpad - k0) / KMMA;
            for (int kk = 0; kk < ksteps; ++kk) {
                const uint32_t ko = (uint32_t)kk * 256u;  // two 128-byte core matrices along K
                const uint32_t acc0 = (c > 0 || kk > 0) ? 1u : 0u;
                if constexpr (BF) {
                    uint64_t da[3], db[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        da[q] = smem_desc(smem_u32(A0 + q * ABYTES) + ko, 128u, SBO_A);
                        db[q] = smem_desc(smem_u32(B0 + q * bbytes) + ko, 128u, SBO_B);
                    }
                    // F_i D_j for i + j <= 4 (parts numbered from 1)
                    mma_bf16(tmem, da[0], db[0], idesc, acc0);
                    mma_bf16(tmem, da[0], db[1], idesc, 1u);
                    mma_bf16(tmem, da[1], db[0], idesc, 1u);
                    mma_bf16(tmem, da[0], db[2], idesc, 1u);
                    mma_bf16(tmem, da[1], db[1], idesc, 1u);
                    mma_bf16(tmem, da[2], db[0], idesc, 1u);
                } else {
                    const uint32_t ah = smem_u32(A0), al = smem_u32(A0 + ABYTES);
                    const uint32_t bh = smem_u32(B0), bl = smem_u32(B0 + bbytes);
                    const uint64_t dah = smem_desc(ah + ko, 128u, SBO_A), dal = smem_desc(al + ko, 128u, SBO_A);
                    const uint64_t dbh = smem_desc(bh + ko, 128u, SBO_B), dbl = smem_desc(bl + ko, 128u, SBO_B);
                    mma_tf32(tmem, dah, dbh, idesc, acc0);
                    mma_tf32(tmem, dah, dbl, idesc, 1u);
                    mma_tf32(tmem, dal, dbh, idesc, 1u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(mbar + st))
                         : "memory");
        }
        issued = c;
    }
    // The last commit covers every MMA issued before it.  On the normal path
    // this is the wait for the result; after a wait gave up it drains the
    // MMAs still in flight (again bounded) before the accumulator columns are
    // freed.  Chunk `issued`'s barrier had its previous phase (chunk
    // issued - 2) observed at the start of chunk `issued`, so its parity is
    // unambiguous.
    if (issued >= 0) {
        bool done = false;
        for (long long it = 0; it < WAIT_ITERS && !done; ++it)
            done = mbar_try_wait(smem_u32(mbar + (issued & 1)), (uint32_t)((issued >> 1) & 1));
        ok = ok && done;
    }
    const int all_ok = __syncthreads_and(ok ? 1 : 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (all_ok) {
        // accumulator lanes 32*warp .. +31 = lines; columns = outputs
        const long long obase = gbase + (long long)s * srow;
        const int m = tid;
        for (int cb = 0; cb < npad; cb += 16) {
            uint32_t r[16];
            const uint32_t ta_ = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(ta_));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < nl) {
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int n = cb + t;
                    if (n < nb) out[obase + (long long)n * srow + (long long)m * sa] = __uint_as_float(r[t]) * scale;
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// two pipeline stages of NP operand parts (the window length does not enter:
// it streams through in chunks of KC points), plus the mbarriers and TMEM slot
size_t gemm_smem_bytes(int npad, bool bf)
{
    const size_t np = bf ? 3 : 2, esz = bf ? 2 : 4, cme = 16 / esz;
    const size_t abytes = 16 * ((size_t)(KC / cme) * 128 + A_PAD);
    const size_t stage = np * abytes + np * (size_t)npad * KC * esz;
    return 2 * stage + 32;
}

template <int AXIS, bool BF>
cudaError_t launch_gemm_axis(const GemmOpDev &op, const int n[3], const float *f, float *out, double scale,
                             int *err, cudaStream_t st)
{
    const int Na = AXIS == 0 ? n[1] : n[0];
    const int Nc = AXIS == 2 ? n[1] : n[2];
    const int ntile = (Na + GM - 1) / GM;
    const long long nblk = (long long)op.nsub * ntile * Nc;
    const size_t smem = gemm_smem_bytes(op.max_npad, BF);
    if (smem > 227 * 1024 || op.max_npad > 256) return cudaErrorInvalidConfiguration;
    gemm_deriv_kernel<AXIS, BF><<<(unsigned)nblk, GM, smem, st>>>(op, n[0], n[1], n[2], ntile, f, out,
                                                                   (float)scale, err);
    return cudaGetLastError();
}

}  // namespace

bool gemm_smem_fits(const DenseHost &h)
{
    return h.max_npad <= 256 && gemm_smem_bytes(h.max_npad, false) <= 227 * 1024 &&
           gemm_smem_bytes(h.max_npad, true) <= 227 * 1024;
}

cudaError_t init_gemm_kernels()
{
    const void *k[6] = {(const void *)gemm_deriv_kernel<0, false>, (const void *)gemm_deriv_kernel<1, false>,
                        (const void *)gemm_deriv_kernel<2, false>, (const void *)gemm_deriv_kernel<0, true>,
                        (const void *)gemm_deriv_kernel<1, true>,  (const void *)gemm_deriv_kernel<2, true>};
    for (const void *fn : k) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_gemm_field(const GemmOpDev &op, bool bf16x3, int axis, const int n[3], const float *f, float *out,
                              double scale, int *err, cudaStream_t st)
{
    switch (axis * 2 + (bf16x3 ? 1 : 0)) {
    case 0: return launch_gemm_axis<0, false>(op, n, f, out, scale, err, st);
    case 1: return launch_gemm_axis<0, true>(op, n, f, out, scale, err, st);
    case 2: return launch_gemm_axis<1, false>(op, n, f, out, scale, err, st);
    case 3: return launch_gemm_axis<1, true>(op, n, f, out, scale, err, st);
    case 4: return launch_gemm_axis<2, false>(op, n, f, out, scale, err, st);
    case 5: return launch_gemm_axis<2, true>(op, n, f, out, scale, err, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t GemmOpBuf::upload()
{
    release();
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t nrec = host.rec.size() * sizeof(int), nf = host.hi.size() * sizeof(float);
    const size_t n16 = host.b16[0].size() * sizeof(uint16_t);
    const size_t o_hi = al(nrec), o_lo = o_hi + al(nf), o_b16 = o_lo + al(nf);
    cudaError_t e = dev_alloc(&mem, o_b16 + 3 * al(n16) + 16);
    if (e != cudaSuccess) {
        mem = nullptr;
        return e;
    }
    char *b = (char *)mem;
    e = cudaMemcpy(b, host.rec.data(), nrec, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_hi, host.hi.data(), nf, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_lo, host.lo.data(), nf, cudaMemcpyHostToDevice);
    for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        e = cudaMemcpy(b + o_b16 + q * al(n16), host.b16[q].data(), n16, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    dev.N = host.N;
    dev.nsub = host.nsub;
    dev.max_npad = host.max_npad;
    dev.max_kpad = host.max_kpad;
    dev.max_kpad16 = host.max_kpad16;
    dev.rec = (const int *)b;
    dev.hi = (const float *)(b + o_hi);
    dev.lo = (const float *)(b + o_lo);
    for (int q = 0; q < 3; ++q) dev.b16[q] = (const uint16_t *)(b + o_b16 + q * al(n16));
    return cudaSuccess;
}

void GemmOpBuf::release()
{
    if (mem) dev_free(mem);
    mem = nullptr;
}

}  // namespace nopcs
