// Viscous terms, gravity source and the classical RK4 stage update, fused in
// one z-marching kernel (arXiv 2203.00879: Eqs. ge6-ge8a, ge19, ge20, bv1-bv3;
// Sec. 4: second-order explicit viscous terms, four-stage RK4).
//
// The viscous right-hand side at a node is the second-order explicit
// divergence of nodal viscous fluxes, and each nodal flux needs second-order
// explicit gradients of u, v, w, T at its node: a +-2 stencil (+-3 next to a
// wall, where both operators are one-sided).  A block owns a TX x TY column
// tile and marches along z; it keeps the primitives (u, v, w, T) of the seven
// planes o-3 .. o+3 around the output plane o, with a two-node x/y halo, in a
// shared-memory ring, so every primitive is loaded from global memory once per
// block and plane.  Each thread evaluates the six nodal fluxes its divergence
// needs from shared memory, adds the gravity source to the convective
// right-hand side accumulated by the sweeps, holds the momentum at zero on
// wall nodes (no-slip) and applies the RK4 stage to the FP64 registers.
//
// Tiles never start past n - TX, so every tile is at least min(n, TX) wide and
// the one-sided wall stencils stay inside its halo; a tile that had to be
// shifted back writes only the columns it owns.
#include <math.h>

#include "nopcs_internal.cuh"

namespace nopcs {

namespace {

constexpr int TX = 32, TY = 8, HALO = 2;
constexpr int PX = TX + 2 * HALO, PY = TY + 2 * HALO, PLANE = PX * PY;
constexpr int RING = 7;   // planes o-3 .. o+3
constexpr int NPF = 4;    // u, v, w, T

template <typename T>
struct VArgs {
    int n[3];
    long long np;
    T ih2[3];             // 1 / (2 h)
    int ga, zc;           // gravity axis, planes per block
    T gm2, iRe, kq, S1, S, c0, c1, g;
    const T *W;
    const T *rho_b, *p_b;                 // base tables (zeros in the plain form)
    const float *T_b, *ip_b, *ir_b;       // mixed form: T_b, 1/p_b, 1/rho_b
    const T *R;
    int stage;
    double dt;
    StageRegs<T> rg_out;
    const double *rho_b64, *E_b64;        // mixed form: base state for the deviation of Q_n
    float gm1;                            // gamma - 1
};

template <typename T>
struct Ring {
    T *s;
    int x0, y0;
    __device__ __forceinline__ T &at(int f, int x, int y, int z) const
    {
        return s[((z % RING) * NPF + f) * PLANE + (y - y0 + HALO) * PX + (x - x0 + HALO)];
    }
};

// temperature from W at (global index i, gravity coordinate kg)
template <typename T>
__device__ __forceinline__ T temp_of(const VArgs<T> &a, long long i, int kg)
{
    const T w0 = a.W[i], w4 = a.W[4 * a.np + i];
    if constexpr (sizeof(T) == 4) {
        // T = T_b (1 + p'/p_b) / (1 + rho'/rho_b): exact at rest, where p' = rho' = 0
        const float rr = w0 * a.ir_b[kg];
        return a.T_b[kg] + a.T_b[kg] * (w4 * a.ip_b[kg] - rr) / (1.0f + rr);
    } else {
        return a.gm2 * (a.p_b[kg] + w4) / (a.rho_b[kg] + w0);
    }
}

template <typename T>
__device__ void load_plane(const VArgs<T> &a, const Ring<T> &rg, int z)
{
    const int nx = a.n[0], ny = a.n[1];
    for (int idx = threadIdx.x; idx < PLANE; idx += blockDim.x) {
        const int lx = idx % PX, ly = idx / PX;
        const int gx = rg.x0 - HALO + lx, gy = rg.y0 - HALO + ly;
        T u = 0, v = 0, w = 0, t = 0;
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
            const long long i = gx + (long long)nx * (gy + (long long)ny * z);
            u = a.W[a.np + i];
            v = a.W[2 * a.np + i];
            w = a.W[3 * a.np + i];
            t = temp_of(a, i, a.ga == 0 ? gx : (a.ga == 1 ? gy : z));
        }
        T *p = rg.s + (size_t)(z % RING) * NPF * PLANE + idx;
        p[0] = u;
        p[PLANE] = v;
        p[2 * PLANE] = w;
        p[3 * PLANE] = t;
    }
}

// second-order explicit derivative of primitive f along axis AX at node (x, y, z)
template <int AX, typename T>
__device__ __forceinline__ T grad(const VArgs<T> &a, const Ring<T> &rg, int f, int x, int y, int z)
{
    const int c = AX == 0 ? x : (AX == 1 ? y : z);
    const int N = a.n[AX];
    auto at = [&](int off) -> T {
        return rg.at(f, x + (AX == 0 ? off : 0), y + (AX == 1 ? off : 0), z + (AX == 2 ? off : 0));
    };
    if (c == 0) return (T(-3) * at(0) + T(4) * at(1) - at(2)) * a.ih2[AX];
    if (c == N - 1) return (T(3) * at(0) - T(4) * at(-1) + at(-2)) * a.ih2[AX];
    return (at(1) - at(-1)) * a.ih2[AX];
}

// nodal viscous flux along axis D at node (x, y, z): (tau_D0, tau_D1, tau_D2, u_k tau_Dk - q_D)
template <int D, typename T>
__device__ __forceinline__ void nodal_flux(const VArgs<T> &a, const Ring<T> &rg, int x, int y, int z, T out[4])
{
    constexpr int E1 = (D + 1) % 3, E2 = (D + 2) % 3;  // the two other axes
    const T Tn = rg.at(3, x, y, z);
    const T mu = Tn * sqrt(Tn) * a.S1 / (Tn + a.S);   // Sutherland
    const T mub = a.c0 * Tn + a.c1;                    // Eq. reg over mu_s
    const T gD = grad<D>(a, rg, D, x, y, z);            // d u_D / d x_D
    const T g1D = grad<D>(a, rg, E1, x, y, z);          // d u_E1 / d x_D
    const T g2D = grad<D>(a, rg, E2, x, y, z);          // d u_E2 / d x_D
    const T g11 = grad<E1>(a, rg, E1, x, y, z);         // d u_E1 / d x_E1
    const T g22 = grad<E2>(a, rg, E2, x, y, z);         // d u_E2 / d x_E2
    const T gD1 = grad<E1>(a, rg, D, x, y, z);          // d u_D / d x_E1
    const T gD2 = grad<E2>(a, rg, D, x, y, z);          // d u_D / d x_E2
    T tau[3];
    // Eq. ge19 off the diagonal; Eqs. bv1-bv3 on it:
    // (4/3 mu + mu_b/mu_s) on the normal strain, (-2/3 mu + mu_b/mu_s) on the other two
    tau[E1] = mu * a.iRe * (g1D + gD1);
    tau[E2] = mu * a.iRe * (g2D + gD2);
    tau[D] = ((T(4) / T(3) * mu + mub) * gD + (T(-2) / T(3) * mu + mub) * (g11 + g22)) * a.iRe;
    const int cD = D == 0 ? x : (D == 1 ? y : z);
    T q = 0;
    if (cD != 0 && cD != a.n[D] - 1) q = -mu * a.kq * grad<D>(a, rg, 3, x, y, z);  // Eq. ge20; adiabatic walls
    out[0] = tau[0];
    out[1] = tau[1];
    out[2] = tau[2];
    out[3] = rg.at(0, x, y, z) * tau[0] + rg.at(1, x, y, z) * tau[1] + rg.at(2, x, y, z) * tau[2] - q;
}

// adds d(nodal viscous flux along D)/dx_D at (x, y, z) to r[1..4]
template <int D, typename T>
__device__ __forceinline__ void add_div(const VArgs<T> &a, const Ring<T> &rg, int x, int y, int z, T r[5])
{
    const int c = D == 0 ? x : (D == 1 ? y : z);
    const int N = a.n[D];
    const T ih = a.ih2[D];
    const int dx = D == 0, dy = D == 1, dz = D == 2;
    T fa[4], fb[4], fc[4];
    if (c == 0) {
        nodal_flux<D>(a, rg, x, y, z, fa);
        nodal_flux<D>(a, rg, x + dx, y + dy, z + dz, fb);
        nodal_flux<D>(a, rg, x + 2 * dx, y + 2 * dy, z + 2 * dz, fc);
#pragma unroll
        for (int k = 0; k < 4; ++k) r[1 + k] += (T(-3) * fa[k] + T(4) * fb[k] - fc[k]) * ih;
    } else if (c == N - 1) {
        nodal_flux<D>(a, rg, x, y, z, fa);
        nodal_flux<D>(a, rg, x - dx, y - dy, z - dz, fb);
        nodal_flux<D>(a, rg, x - 2 * dx, y - 2 * dy, z - 2 * dz, fc);
#pragma unroll
        for (int k = 0; k < 4; ++k) r[1 + k] += (T(3) * fa[k] - T(4) * fb[k] + fc[k]) * ih;
    } else {
        nodal_flux<D>(a, rg, x + dx, y + dy, z + dz, fa);
        nodal_flux<D>(a, rg, x - dx, y - dy, z - dz, fb);
#pragma unroll
        for (int k = 0; k < 4; ++k) r[1 + k] += (fa[k] - fb[k]) * ih;
    }
}

// primitives of a stage state from its FP32 deviation D = (rho', m_x, m_y, m_z, E')
__device__ __forceinline__ void prim_from_dev(const VArgs<float> &a, long long p, int kg, const float D[5])
{
    const long long np = a.np;
    const float rho = a.rho_b[kg] + D[0];
    const float ir = 1.0f / rho;
    const float u = D[1] * ir, v = D[2] * ir, w = D[3] * ir;
    const float ke = 0.5f * (D[1] * u + D[2] * v + D[3] * w);
    const float pd = a.gm1 * (D[4] - ke);
    float *Wn = a.rg_out.Wn;
    Wn[p] = D[0];
    Wn[np + p] = u;
    Wn[2 * np + p] = v;
    Wn[3 * np + p] = w;
    Wn[4 * np + p] = pd;
    Wn[5 * np + p] = D[4] + pd;
}

// Mixed form of the classical RK4 stage.  The slopes are FP32 (they are FP32
// right-hand sides); K = k1 + 2 k2 + 2 k3 + k4 is accumulated in FP32 and added
// to the FP64 state once, Q_n += dt/6 K, in FP64.  The stage states
// Q_n + c dt k are formed as FP32 deviations from the hydrostatic base, the
// same quantities the primitive recovery of the FP64 form rounds to FP32.
__device__ __forceinline__ void mixed_update(const VArgs<float> &a, long long p, int kg, const float r[5])
{
    const long long np = a.np;
    const int s = a.stage;
    float K[5];
    if (s == 1) {
#pragma unroll
        for (int k = 0; k < 5; ++k) K[k] = r[k];
    } else {
        const float w = s == 4 ? 1.0f : 2.0f;
#pragma unroll
        for (int k = 0; k < 5; ++k) K[k] = a.rg_out.Kacc[k * np + p] + w * r[k];
    }
    float D[5];
    if (s < 4) {
#pragma unroll
        for (int k = 0; k < 5; ++k) a.rg_out.Kacc[k * np + p] = K[k];
        const float c = (float)(s == 3 ? a.dt : 0.5 * a.dt);
#pragma unroll
        for (int k = 0; k < 5; ++k) D[k] = a.rg_out.Dn[k * np + p] + c * r[k];
    } else {
        const double w6 = a.dt / 6.0;
        double q[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            q[k] = a.rg_out.Qn[k * np + p] + w6 * (double)K[k];
            a.rg_out.Qn[k * np + p] = q[k];
        }
        D[0] = (float)(q[0] - a.rho_b64[kg]);
        D[1] = (float)q[1];
        D[2] = (float)q[2];
        D[3] = (float)q[3];
        D[4] = (float)(q[4] - a.E_b64[kg]);
#pragma unroll
        for (int k = 0; k < 5; ++k) a.rg_out.Dn[k * np + p] = D[k];
    }
    prim_from_dev(a, p, kg, D);
}

template <typename T>
__global__ void __launch_bounds__(TX *TY) visc_rk_kernel(const VArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const int xs = blockIdx.x * TX, ys = blockIdx.y * TY;
    Ring<T> rg;
    rg.s = reinterpret_cast<T *>(smraw);
    rg.x0 = min(xs, max(nx - TX, 0));
    rg.y0 = min(ys, max(ny - TY, 0));
    const int z0 = blockIdx.z * a.zc, z1 = min(nz, z0 + a.zc);
    const int x = rg.x0 + (int)(threadIdx.x % TX), y = rg.y0 + (int)(threadIdx.x / TX);
    const bool own = x < nx && y < ny && x >= xs && y >= ys;
    const long long np = a.np;

    for (int z = max(0, z0 - 3); z <= min(nz - 1, z0 + 2); ++z) load_plane(a, rg, z);
    for (int o = z0; o < z1; ++o) {
        if (o + 3 < nz) load_plane(a, rg, o + 3);
        __syncthreads();
        if (own) {
            const long long p = x + (long long)nx * (y + (long long)ny * o);
            T r[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) r[k] = a.R[k * np + p];
            // divergence of the nodal viscous fluxes (same explicit operator)
            add_div<0>(a, rg, x, y, o, r);
            add_div<1>(a, rg, x, y, o, r);
            add_div<2>(a, rg, x, y, o, r);
            // gravity source, Eq. ge8a
            const int kg = a.ga == 0 ? x : (a.ga == 1 ? y : o);
            const T w0 = a.W[p];
            const T rho = a.rho_b[kg] + w0;
            const T ug = rg.at(a.ga, x, y, o);
            const T sg = w0 * a.g;
            if (a.ga == 0) r[1] -= sg;
            if (a.ga == 1) r[2] -= sg;
            if (a.ga == 2) r[3] -= sg;
            r[4] -= rho * ug * a.g;
            // no-slip walls
            if (x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || o == 0 || o == nz - 1) r[1] = r[2] = r[3] = 0;
            if (a.stage == 0) {
#pragma unroll
                for (int k = 0; k < 5; ++k) a.rg_out.Rout[k * np + p] = r[k];
            } else if constexpr (sizeof(T) == 4) {
                mixed_update(a, p, kg, r);
            } else {
                // classical RK4: acc collects Q_n + dt (k1 + 2 k2 + 2 k3 + k4) / 6
                const double bw = (a.stage == 1 || a.stage == 4) ? a.dt / 6.0 : a.dt / 3.0;
                const double cw = a.stage == 3 ? a.dt : 0.5 * a.dt;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const double rk = (double)r[k];
                    const long long i = k * np + p;
                    if (a.stage == 1) {
                        const double q = a.rg_out.Qn[i];
                        a.rg_out.acc[i] = q + bw * rk;
                        a.rg_out.Qout[i] = q + cw * rk;
                    } else if (a.stage < 4) {
                        a.rg_out.acc[i] = a.rg_out.acc[i] + bw * rk;
                        a.rg_out.Qout[i] = a.rg_out.Qn[i] + cw * rk;
                    } else {
                        a.rg_out.Qout[i] = a.rg_out.acc[i] + bw * rk;
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <typename T>
size_t ring_bytes()
{
    return (size_t)RING * NPF * PLANE * sizeof(T);
}

}  // namespace

cudaError_t init_visc_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(visc_rk_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ring_bytes<float>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(visc_rk_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ring_bytes<double>());
}

template <typename T>
cudaError_t launch_visc_update(const BoxDev &bx, const T *W, const T *R, int stage, const StageRegs<T> &g,
                               cudaStream_t st)
{
    VArgs<T> a{};
    for (int d = 0; d < 3; ++d) {
        a.n[d] = bx.n[d];
        a.ih2[d] = (T)(0.5 * bx.inv_h[d]);
    }
    a.np = bx.np;
    a.ga = bx.ga;
    a.gm2 = (T)bx.gm2;
    a.iRe = (T)(1.0 / bx.Re);
    a.kq = (T)bx.kq;
    a.S1 = (T)(1.0 + bx.suth_S);
    a.S = (T)bx.suth_S;
    a.c0 = (T)bx.mub_coef0;
    a.c1 = (T)bx.mub_coef1;
    a.g = (T)bx.g;
    a.W = W;
    if constexpr (sizeof(T) == 8) {
        a.rho_b = (const T *)bx.rho_b64;
        a.p_b = (const T *)bx.p_b64;
    } else {
        a.rho_b = (const T *)bx.rho_b32;
    }
    a.T_b = bx.T_b32;
    a.ip_b = bx.ip_b32;
    a.ir_b = bx.ir_b32;
    a.R = R;
    a.stage = stage;
    a.dt = bx.dt;
    a.rg_out = g;
    a.rho_b64 = bx.rho_b64;
    a.E_b64 = bx.E_b64;
    a.gm1 = (float)(bx.gamma - 1.0);
    const int gx = (bx.n[0] + TX - 1) / TX, gy = (bx.n[1] + TY - 1) / TY;
    // z chunk: enough blocks for the whole GPU, at least 8 planes per block
    const long long want = 152LL * 8;
    int nzc = (int)((want + (long long)gx * gy - 1) / ((long long)gx * gy));
    int zc = (bx.n[2] + nzc - 1) / nzc;
    if (zc < 8) zc = 8;
    if (zc > 64) zc = 64;
    a.zc = zc;
    dim3 grid(gx, gy, (bx.n[2] + zc - 1) / zc);
    visc_rk_kernel<T><<<grid, TX * TY, ring_bytes<T>(), st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_visc_update<float>(const BoxDev &, const float *, const float *, int,
                                              const StageRegs<float> &, cudaStream_t);
template cudaError_t launch_visc_update<double>(const BoxDev &, const double *, const double *, int,
                                               const StageRegs<double> &, cudaStream_t);

}  // namespace nopcs
