// Tensor-core form of the NOHAP derivative (arXiv 2203.00879, Sec. 3).
//
// NOHAP makes every sub-domain's result a fixed linear map of the inputs in
// its staging window: the end rows are rows of C = A^-1 B and the interior is
// a Thomas solve, both linear.  So sub-domain b is g = D_b f_window with a
// small dense D_b (n_b outputs x Kpad window points, built on the host by
// applying the line algorithm to unit vectors), and the derivative of 128
// neighbouring lines is one dense contraction
//     OUT (128 lines x n_b) = F (128 lines x Kpad) . D_b^T (Kpad x n_b)
// on the 5th-generation tensor cores (tcgen05.mma, kind::tf32, M = 128,
// N = Npad, K = 8 per instruction), FP32 accumulation in tensor memory.
// Split precision ("3xTF32"): F = F_hi + F_lo and D = D_hi + D_lo with TF32
// parts; OUT = F_hi D_hi + F_hi D_lo + F_lo D_hi recovers ~21 bits.
//
// Both operands sit in shared memory in the K-major, non-swizzled canonical
// layout of tcgen05: 8-row x 16-byte core matrices, contiguous along K
// (leading byte offset 128) and SBO bytes apart along M/N.  One thread issues
// the MMAs and commits them to an mbarrier; the block waits on it with an
// iteration bound, then each warp reads its 32 accumulator lanes with
// tcgen05.ld and stores them.
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

template <int AXIS>
__global__ void __launch_bounds__(GM) gemm_deriv_kernel(const GemmOpDev op, int nx, int ny, int nz, int ntile_a,
                                                        const float *__restrict__ f, float *__restrict__ out,
                                                        float scale, int *err)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    const int b = blockIdx.x % op.nsub;
    const int tile = blockIdx.x / op.nsub;
    const int ta = tile % ntile_a, cc = tile / ntile_a;
    const int a0 = ta * GM;
    const int Na = AXIS == 0 ? ny : nx;
    const int nl = min(GM, Na - a0);
    const int N = op.N;
    const int *rec = op.rec + b * DENSE_REC;
    const int s = rec[0], nb = rec[1], npad = rec[2], kpad = rec[3], wlo = rec[4], boff = rec[5];
    // per stage: A chunk (128 x KC, hi and lo) and B chunk (npad x KC, hi and lo)
    constexpr uint32_t SBO_A = (KC / 4) * 128u + A_PAD, SBO_B = (KC / 4) * 128u;
    constexpr uint32_t ABYTES = 16u * SBO_A;
    const uint32_t bbytes = (uint32_t)npad * KC * 4u;
    const uint32_t stage_bytes = 2u * ABYTES + 2u * bbytes;
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
    const uint32_t idesc = idesc_tf32(npad);
    bool ok = true;
    for (int c = 0; c < nchunk; ++c) {
        const int st = c & 1;
        unsigned char *Ahi = smraw + st * stage_bytes, *Alo = Ahi + ABYTES;
        unsigned char *Bhi = Alo + ABYTES, *Blo = Bhi + bbytes;
        // the MMAs of chunk c - 2 read this stage: wait for their commit
        if (c >= 2) {
            bool done = false;
            for (long long it = 0; it < WAIT_ITERS && !done; ++it)
                done = mbar_try_wait(smem_u32(mbar + st), (uint32_t)(((c - 2) >> 1) & 1));
            ok = ok && done;
        }
        const int k0 = c * KC;
        // B chunk: core matrices k0/4 .. k0/4 + KC/4 of every 8-row group
        {
            const int ncm = KC / 4;  // core matrices per group in a chunk
            const int nq = (npad / 8) * ncm * 8;  // float4 per part
            for (int i = tid; i < nq; i += GM) {
                const int g = i / (ncm * 8), rem = i % (ncm * 8), cm = rem / 8, row = rem % 8;
                const int kc = k0 / 4 + cm;
                float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
                if (kc < kpad / 4) {
                    const size_t go = (size_t)boff + (size_t)g * (kpad / 4) * 32 + (size_t)kc * 32 + row * 4;
                    h = *reinterpret_cast<const float4 *>(op.hi + go);
                    l = *reinterpret_cast<const float4 *>(op.lo + go);
                }
                const uint32_t so = (uint32_t)g * SBO_B + (uint32_t)cm * 128u + row * 16u;
                *reinterpret_cast<float4 *>(Bhi + so) = h;
                *reinterpret_cast<float4 *>(Blo + so) = l;
            }
        }
        // A chunk: the lines' window points k0 .. k0 + KC - 1, split into TF32 hi/lo
        if (AXIS == 0) {
            for (int q = tid; q < GM * KC; q += GM) {
                const int m = q / KC, k = q % KC;
                const int pos = wlo + k0 + k;
                float v = 0.0f;
                if (m < nl && pos < N && k0 + k < kpad)
                    v = f[gbase + (long long)m * sa + pos] - f[gbase + (long long)m * sa + s];
                const float h = tf32_part(v), l = tf32_part(v - h);
                const uint32_t o = (uint32_t)(m >> 3) * SBO_A + (uint32_t)(k >> 2) * 128u + (m & 7) * 16u + (k & 3) * 4u;
                *reinterpret_cast<float *>(Ahi + o) = h;
                *reinterpret_cast<float *>(Alo + o) = l;
            }
        } else {
            const int m = tid;
#pragma unroll 2
            for (int k4 = 0; k4 < KC; k4 += 4) {
                float v[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int pos = wlo + k0 + k4 + t;
                    v[t] = (m < nl && pos < N && k0 + k4 + t < kpad) ? f[gbase + (long long)pos * srow + m] - c0 : 0.0f;
                }
                float4 h, l;
                h.x = tf32_part(v[0]);
                h.y = tf32_part(v[1]);
                h.z = tf32_part(v[2]);
                h.w = tf32_part(v[3]);
                l.x = tf32_part(v[0] - h.x);
                l.y = tf32_part(v[1] - h.y);
                l.z = tf32_part(v[2] - h.z);
                l.w = tf32_part(v[3] - h.w);
                const uint32_t o = (uint32_t)(m >> 3) * SBO_A + (uint32_t)(k4 >> 2) * 128u + (m & 7) * 16u;
                *reinterpret_cast<float4 *>(Ahi + o) = h;
                *reinterpret_cast<float4 *>(Alo + o) = l;
            }
        }
        // generic-proxy shared stores -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
            const int ksteps = min(KC, kpad - k0) / 8;
            for (int kk = 0; kk < ksteps; ++kk) {
                const uint32_t ko = (uint32_t)kk * 256u;  // two 128-byte core matrices along K
                const uint64_t dah = smem_desc(ah + ko, 128u, SBO_A), dal = smem_desc(al + ko, 128u, SBO_A);
                const uint64_t dbh = smem_desc(bh + ko, 128u, SBO_B), dbl = smem_desc(bl + ko, 128u, SBO_B);
                mma_tf32(tmem, dah, dbh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, dah, dbl, idesc, 1u);
                mma_tf32(tmem, dal, dbh, idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(mbar + st))
                         : "memory");
        }
    }
    // the last commit covers every MMA issued before it
    {
        const int c = nchunk - 1;
        bool done = false;
        for (long long it = 0; it < WAIT_ITERS && !done; ++it)
            done = mbar_try_wait(smem_u32(mbar + (c & 1)), (uint32_t)((c >> 1) & 1));
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

size_t gemm_smem_bytes(int npad, int kpad)
{
    (void)kpad;
    const size_t abytes = 16 * ((size_t)(KC / 4) * 128 + A_PAD);
    const size_t stage = 2 * abytes + 2 * (size_t)npad * KC * 4;
    return 2 * stage + 32;
}

template <int AXIS>
cudaError_t launch_gemm_axis(const GemmOpDev &op, const int n[3], const float *f, float *out, double scale,
                             int *err, cudaStream_t st)
{
    const int Na = AXIS == 0 ? n[1] : n[0];
    const int Nc = AXIS == 2 ? n[1] : n[2];
    const int ntile = (Na + GM - 1) / GM;
    const long long nblk = (long long)op.nsub * ntile * Nc;
    const size_t smem = gemm_smem_bytes(op.max_npad, op.max_kpad);
    if (smem > 227 * 1024 || op.max_npad > 256) return cudaErrorInvalidConfiguration;
    gemm_deriv_kernel<AXIS><<<(unsigned)nblk, GM, smem, st>>>(op, n[0], n[1], n[2], ntile, f, out, (float)scale,
                                                               err);
    return cudaGetLastError();
}

}  // namespace

bool gemm_smem_fits(const DenseHost &h)
{
    return h.max_npad <= 256 && gemm_smem_bytes(h.max_npad, h.max_kpad) <= 227 * 1024;
}

cudaError_t init_gemm_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(gemm_deriv_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_deriv_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gemm_deriv_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    return e;
}

cudaError_t launch_gemm_field(const GemmOpDev &op, int axis, const int n[3], const float *f, float *out,
                              double scale, int *err, cudaStream_t st)
{
    switch (axis) {
    case 0: return launch_gemm_axis<0>(op, n, f, out, scale, err, st);
    case 1: return launch_gemm_axis<1>(op, n, f, out, scale, err, st);
    case 2: return launch_gemm_axis<2>(op, n, f, out, scale, err, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t GemmOpBuf::upload()
{
    release();
    const size_t nrec = host.rec.size() * sizeof(int), nf = host.hi.size() * sizeof(float);
    const size_t o_hi = (nrec + 255) & ~(size_t)255, o_lo = o_hi + ((nf + 255) & ~(size_t)255);
    cudaError_t e = cudaMalloc(&mem, o_lo + nf + 16);
    if (e != cudaSuccess) {
        mem = nullptr;
        return e;
    }
    char *b = (char *)mem;
    e = cudaMemcpy(b, host.rec.data(), nrec, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_hi, host.hi.data(), nf, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_lo, host.lo.data(), nf, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    dev.N = host.N;
    dev.nsub = host.nsub;
    dev.max_npad = host.max_npad;
    dev.max_kpad = host.max_kpad;
    dev.rec = (const int *)b;
    dev.hi = (const float *)(b + o_hi);
    dev.lo = (const float *)(b + o_lo);
    return cudaSuccess;
}

void GemmOpBuf::release()
{
    if (mem) cudaFree(mem);
    mem = nullptr;
}

}  // namespace nopcs
