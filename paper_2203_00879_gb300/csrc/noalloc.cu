// Allocation-free second derivative: nopcs_derivative2_noalloc (include/nopcs.h).
//
// nopcs_derivative(order = 2) keeps the first derivative between its two
// passes in scratch that the library allocates with cudaMalloc on the first
// such call for a box.  Some callers cannot allow that: a host program whose
// device memory is owned by its own pool allocator (a framework or a serving
// process with a fixed memory budget), or a latency-critical loop where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
// This entry point does the same two passes but keeps the intermediate in the
// fixed array below, which is part of the library's device image: every GPU
// that loads the library holds it until the process exits, and this call
// allocates nothing.
//
// In host code `g_noalloc_scratch` only names a host-side stand-in for the
// array; its device address is obtained with cudaGetSymbolAddress, once per
// device, with that device current, and that address is what the kernels get.
// nopcs_init does that lookup on its device (noalloc_prepare), which also
// loads this file's module there: from then on the 16 MiB are resident on
// that device, and no call of the entry point loads a module or allocates.
#include <mutex>

#include "nopcs_internal.cuh"

namespace {

// 16 MiB: 2^21 FP64 values (a 128^3 field) or 2^22 FP32 values.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};

// device address of the scratch array on the current device (set up once)
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

namespace nopcs {

cudaError_t noalloc_prepare()
{
    void *p = nullptr;
    return scratch_address(&p);
}

}  // namespace nopcs

using namespace nopcs;

extern "C" nopcs_status nopcs_derivative2_noalloc(nopcs_ctx *ctx, int box, int axis, int dtype, const void *f,
                                                  void *df, void *stream)
{
    if (!ctx) return NOPCS_EINVAL;
    long long np = 0;
    nopcs_status s = ctx_derivative_check(ctx, box, axis, dtype, &np);
    if (s != NOPCS_OK) return s;
    if (!f || !df) return ctx_error(ctx, NOPCS_EINVAL, "null field pointer");
    const size_t es = dtype == 0 ? 8 : 4;
    const size_t bytes = (size_t)np * es;
    if (bytes > NOALLOC_SCRATCH_BYTES)
        return ctx_error(ctx, NOPCS_EINVAL,
                         "nopcs_derivative2_noalloc: the field needs more than the 16 MiB of static scratch "
                         "(at most 2^21 FP64 or 2^22 FP32 points); use nopcs_derivative with order 2");
    const char *fc = (const char *)f, *dc = (const char *)df;
    if (fc < dc + bytes && dc < fc + bytes) return ctx_error(ctx, NOPCS_EINVAL, "f and df overlap");
    void *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return ctx_error(ctx, NOPCS_ECUDA, "nopcs_derivative2_noalloc: scratch address");
    cudaStream_t st = (cudaStream_t)stream;
    // the two passes of nopcs_derivative(order = 2), in the same form per axis
    // (Thomas, banded or tensor-core); pass 1 writes every element of the
    // scratch that pass 2 reads, so nothing needs clearing
    e = ctx_first_derivative(ctx, box, axis, dtype, f, scratch, st);
    if (e == cudaSuccess) e = ctx_first_derivative(ctx, box, axis, dtype, scratch, df, st);
    if (e != cudaSuccess) return ctx_error(ctx, NOPCS_ECUDA, "nopcs_derivative2_noalloc: launch failed");
    return NOPCS_OK;
}
