// The whole-line x flux sweep as a stand-alone kernel (body: xline_body in
// line_body.cuh), in a translation unit of its own.
#include "line_body.cuh"

namespace nopcs {

namespace {

template <typename T>
__global__ void xline_kernel(const LineOpDev op, const LineArgs<T> a)
{
    xline_body<T, MODE_FLUX>(op, a, (int)blockIdx.x);
}

}  // namespace

template <typename T>
cudaError_t launch_xline_flux(const LineOpDev &op, const LineArgs<T> &a, long long nblk, int threads, size_t smem,
                              cudaStream_t st)
{
    xline_kernel<T><<<(unsigned)nblk, threads, smem, st>>>(op, a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t init_xline_flux()
{
    return cudaFuncSetAttribute(xline_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XLINE_SMEM);
}

template cudaError_t launch_xline_flux<float>(const LineOpDev &, const LineArgs<float> &, long long, int, size_t,
                                              cudaStream_t);
template cudaError_t launch_xline_flux<double>(const LineOpDev &, const LineArgs<double> &, long long, int, size_t,
                                               cudaStream_t);
template cudaError_t init_xline_flux<float>();
template cudaError_t init_xline_flux<double>();

}  // namespace nopcs
