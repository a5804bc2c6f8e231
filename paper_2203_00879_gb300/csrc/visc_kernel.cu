// Viscous terms, gravity source and the classical RK4 stage update, fused in
// one z-marching kernel (arXiv 2203.00879: Eqs. ge6-ge8a, ge19, ge20, bv1-bv3;
// Sec. 4: second-order explicit viscous terms, four-stage RK4).
//
// The viscous right-hand side at a node is the second-order explicit
// divergence of nodal viscous fluxes, and each nodal flux needs second-order
// explicit gradients of u, v, w, T at its node: a +-2 stencil (+-3 next to a
// wall, where both operators are one-sided).  A block owns a TX x TY column
// tile and marches along z, keeping the primitives (u, v, w, T) of the five
// planes o-2 .. o+2 around the output plane o, with a two-node x/y halo, in a
// shared-memory ring; every primitive is loaded from global memory once per
// block and plane.  For each plane the block then
//   1. evaluates every nodal viscous flux once: E_v on the plane's tile plus
//      a one-node x halo, F_v on the tile plus a one-node y halo, and G_v on
//      the tile of the planes the z divergence needs, kept in a ring of three
//      planes so each G_v plane is computed once and used twice;
//   2. takes the divergence at its tile nodes, adds the gravity source to the
//      convective right-hand side accumulated by the sweeps, holds momentum at
//      zero on wall nodes (no-slip) and applies the RK4 stage.
// The primitive loads of the next plane are issued during step 2.
//
// Tiles never start past n - TX, so every tile is at least min(n, TX) wide and
// the one-sided wall stencils stay inside it; a tile that had to be shifted
// back writes only the columns it owns.
#include "visc_body.cuh"

namespace nopcs {

namespace {

// FP32: three blocks (24 warps) per SM, with up to 85 registers per thread;
// a 64-register cap for four blocks was 1.4% slower once the L2 prefetches
// had taken the load latency off the update.  S fixes the stage and the
// gravity axis at compile time (Spec) or leaves them to the arguments.
template <typename T, class S>
__global__ void __launch_bounds__(TX *TY, (sizeof(T) == 4 ? 768 : 512) / (TX * TY)) visc_rk_kernel(const VArgs<T> a)
{
    extern __shared__ __align__(32) unsigned char smraw[];
    visc_rk_block<T, S>(a, blockIdx.x, blockIdx.y, blockIdx.z, smraw);
}

// Compact viscous terms, step 2 of 3: the nodal viscous fluxes from the
// gradients that the VGRAD sweeps left in G, written over them in place
// (field 4 d + q = d(prim q)/dx_d in, field 4 d + c = component c of the flux
// along d out; a node's twelve values are read before any is written).
template <typename T>
__global__ void __launch_bounds__(256) visc_flux_kernel(const VArgs<T> a, T *__restrict__ G)
{
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const size_t np = (size_t)a.np;
    for (long long q = blockIdx.x * blockDim.x + threadIdx.x; q < a.np; q += gridDim.x * blockDim.x) {
        const int p = (int)q;  // boxes hold < 2^31 points
        T g[3][4];  // g[d][q] = d(prim q)/dx_d, prim = u, v, w, T
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int q = 0; q < 4; ++q) g[d][q] = G[(4 * d + q) * np + p];
        const int x = p % nx, y = (p / nx) % ny, z = p / (nx * ny);
        const int kg = a.ga == 0 ? x : (a.ga == 1 ? y : z);
        const T u = a.W[1][p], v = a.W[2][p], w = a.W[3][p];
        T mu, mub;
        visc_coeffs(a, node_temperature(a, kg, a.W[0][p], a.W[4][p]), mu, mub);
        const T k43 = (T(4) / T(3) * mu + mub) * a.iRe, k23 = (T(-2) / T(3) * mu + mub) * a.iRe, ks = mu * a.iRe;
        // stress tensor, Eqs. ge19, bv1-bv3 (d u_i / d x_j = g[j][i])
        const T txx = k43 * g[0][0] + k23 * (g[1][1] + g[2][2]);
        const T tyy = k43 * g[1][1] + k23 * (g[0][0] + g[2][2]);
        const T tzz = k43 * g[2][2] + k23 * (g[0][0] + g[1][1]);
        const T txy = ks * (g[1][0] + g[0][1]);
        const T txz = ks * (g[2][0] + g[0][2]);
        const T tyz = ks * (g[2][1] + g[1][2]);
        // heat flux, Eq. ge20; its normal component is zero on an adiabatic wall
        const T mk = -mu * a.kq;
        const T qx = (x == 0 || x == nx - 1) ? T(0) : mk * g[0][3];
        const T qy = (y == 0 || y == ny - 1) ? T(0) : mk * g[1][3];
        const T qz = (z == 0 || z == nz - 1) ? T(0) : mk * g[2][3];
        const T f[12] = {txx, txy, txz, u * txx + v * txy + w * txz - qx,
                         txy, tyy, tyz, u * txy + v * tyy + w * tyz - qy,
                         txz, tyz, tzz, u * txz + v * tyz + w * tzz - qz};
#pragma unroll
        for (int k = 0; k < 12; ++k) G[k * np + p] = f[k];
    }
}

// Compact viscous terms, step 3 of 3 (after the VDIV sweeps added the
// divergence into R): gravity source, no-slip walls and the RK stage.
template <typename T>
__global__ void __launch_bounds__(256) source_rk_kernel(const VArgs<T> a)
{
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    for (long long q = blockIdx.x * blockDim.x + threadIdx.x; q < a.np; q += gridDim.x * blockDim.x) {
        const int p = (int)q;  // boxes hold < 2^31 points
        T r[5];
        float kd[5], dn[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) r[k] = a.R[k][p];
        if constexpr (sizeof(T) == 4) {
            if (a.stage >= 2) {
#pragma unroll
                for (int k = 0; k < 5; ++k) kd[k] = a.Kacc[k][p];
            }
            if (a.stage >= 1 && a.stage <= 3) {
#pragma unroll
                for (int k = 0; k < 5; ++k) dn[k] = a.Dn[k][p];
            }
        }
        const int x = p % nx, y = (p / nx) % ny, z = p / (nx * ny);
        const int kg = a.ga == 0 ? x : (a.ga == 1 ? y : z);
        const bool wall = x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || z == 0 || z == nz - 1;
        source_and_stage(a, p, kg, wall, a.W[0][p], a.W[1 + a.ga][p], r, kd, dn);
    }
}

// pointwise kernels: a grid of 8 blocks of 256 per SM striding over the box
unsigned pointwise_blocks(long long np)
{
    long long b = (np + 255) / 256;
    if (b > 152LL * 8) b = 152LL * 8;
    return (unsigned)(b < 1 ? 1 : b);
}

// The stage kernel for (stage, gravity axis): FP32 with gravity along z, the
// benchmark's case, specialised per stage; everything else generic.
template <typename T>
const void *visc_kernel_for(int stage, int ga)
{
    if constexpr (sizeof(T) == 4) {
        if (ga == 2) {
            switch (stage) {
            case 0: return (const void *)visc_rk_kernel<float, Spec<0, 2>>;
            case 1: return (const void *)visc_rk_kernel<float, Spec<1, 2>>;
            case 2: return (const void *)visc_rk_kernel<float, Spec<2, 2>>;
            case 3: return (const void *)visc_rk_kernel<float, Spec<3, 2>>;
            case 4: return (const void *)visc_rk_kernel<float, Spec<4, 2>>;
            }
        }
    }
    return (const void *)visc_rk_kernel<T, RunSpec>;
}

}  // namespace

cudaError_t init_visc_kernels()
{
    for (int ga = 0; ga < 3; ga += 2)
        for (int s = 0; s <= 4; ++s) {
            cudaError_t e = cudaFuncSetAttribute(visc_kernel_for<float>(s, ga),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_bytes<float>());
            if (e != cudaSuccess) return e;
        }
    return cudaFuncSetAttribute(visc_kernel_for<double>(0, 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ring_bytes<double>());
}

template <typename T>
cudaError_t launch_visc_update(const BoxDev &bx, const T *W, const T *R, int stage, const StageRegs<T> &g,
                               cudaStream_t st)
{
    VArgs<T> a = make_vargs(bx, W, R, stage, g);
    const int gx = (bx.n[0] + TX - 1) / TX, gy = (bx.n[1] + TY - 1) / TY;
    // z chunk: enough blocks for the whole GPU, 8 to 32 planes per block (at
    // 1024^3, 32 planes ran 1% faster than 64, a finer last wave; 16 paid
    // more for the ring's start-up planes than it gained)
    const long long want = 152LL * 8;
    int nzc = (int)((want + (long long)gx * gy - 1) / ((long long)gx * gy));
    int zc = (bx.n[2] + nzc - 1) / nzc;
    if (zc < 8) zc = 8;
    if (zc > 32) zc = 32;
    a.zc = zc;
    dim3 grid(gx, gy, (bx.n[2] + zc - 1) / zc);
    void *args[] = {&a};
    return cudaLaunchKernel(visc_kernel_for<T>(stage, bx.ga), grid, dim3(TX * TY), args, ring_bytes<T>(), st);
}

template <typename T>
cudaError_t launch_visc_flux(const BoxDev &bx, const T *W, T *G, cudaStream_t st)
{
    const VArgs<T> a = make_vargs(bx, W, (const T *)nullptr, 0, StageRegs<T>{});
    visc_flux_kernel<T><<<pointwise_blocks(bx.np), 256, 0, st>>>(a, G);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_source_update(const BoxDev &bx, const T *W, const T *R, int stage, const StageRegs<T> &g,
                                 cudaStream_t st)
{
    const VArgs<T> a = make_vargs(bx, W, R, stage, g);
    source_rk_kernel<T><<<pointwise_blocks(bx.np), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_visc_flux<float>(const BoxDev &, const float *, float *, cudaStream_t);
template cudaError_t launch_visc_flux<double>(const BoxDev &, const double *, double *, cudaStream_t);
template cudaError_t launch_source_update<float>(const BoxDev &, const float *, const float *, int,
                                                 const StageRegs<float> &, cudaStream_t);
template cudaError_t launch_source_update<double>(const BoxDev &, const double *, const double *, int,
                                                  const StageRegs<double> &, cudaStream_t);
template cudaError_t launch_visc_update<float>(const BoxDev &, const float *, const float *, int,
                                              const StageRegs<float> &, cudaStream_t);
template cudaError_t launch_visc_update<double>(const BoxDev &, const double *, const double *, int,
                                               const StageRegs<double> &, cudaStream_t);

}  // namespace nopcs
