// Device body of the fused viscous / source / RK stage kernel (arXiv
// 2203.00879: Eqs. ge6-ge8a, ge19, ge20, bv1-bv3; Sec. 4), one block given as
// (bx, by, bz), with its argument block (VArgs, make_vargs) and shared-memory
// size, so that the stand-alone kernel (visc_kernel.cu) and the batched
// persistent kernel (batch_kernel.cu) run the same code.  The header comment of
// visc_kernel.cu describes the algorithm.
#pragma once

#include <math.h>

#include "fp_bits.cuh"
#include "nopcs_internal.cuh"

namespace nopcs {

namespace {

constexpr int TX = 32, TY = 8, HALO = 2;
constexpr int PX = TX + 2 * HALO, PY = TY + 2 * HALO, PLANE = PX * PY;
constexpr int RING = 5;   // planes o-2 .. o+2 (o-3 .. o+1 / o-1 .. o+3 at a wall)
constexpr int NPF = 4;    // u, v, w, T
constexpr int GSLOTS = 3; // planes of G_v kept
// FP32: E_v and F_v of plane o+1 are evaluated with its G_v, from one stencil,
// and kept for the next plane (two slots); FP64 evaluates them at plane o (one
// slot), which keeps its shared memory within two blocks per SM.
template <typename T>
__host__ __device__ constexpr bool flux_ahead() { return sizeof(T) == 4; }
template <typename T>
__host__ __device__ constexpr int ef_slots() { return flux_ahead<T>() ? 2 : 1; }

// Every field array is passed as its own base pointer, so a node's address is
// one 32-bit index away from a kernel parameter (boxes hold < 2^31 points).
template <typename T>
struct VArgs {
    int n[3];
    int np;
    T ih2[3];             // 1 / (2 h)
    int ga, zc;           // gravity axis, planes per block
    T gm2, iRe, kq, S1, S, c0, c1, g;
    const T *W[6];
    const T *rho_b, *p_b;                 // base tables (zeros in the plain form)
    const float *T_b, *ip_b, *ir_b;       // mixed form: T_b, 1/p_b, 1/rho_b
    const T *R[5];
    int stage;
    double dt;
    double dt6, dt3, dt2;                 // dt/6, dt/3, dt/2 (host-computed: no FP64 division per node)
    float cdt2, cdt1;                     // FP32 dt/2 and dt (mixed-form stage states)
    T *Rout[5];                           // stage 0: right-hand side out
    double *Qn[5], *acc[5], *Qout[5];     // FP64 stage registers
    float *Kacc[5], *Dn[5];               // mixed form: slope sum, deviation of Q_n
    T *Wn[6];                             // mixed form: next stage's W
    const double *rho_b64, *E_b64;        // mixed form: base state for the deviation of Q_n
    float gm1;                            // gamma - 1
};

// Compile-time specialisation of the stage kernel: the RK stage (0..4) and
// the gravity axis (0..2) fixed at compile time, or -1 to take them from the
// arguments at run time.  The benchmark's stages run specialised: no per-node
// tests of the stage or the gravity axis, and no dead code of other stages.
template <int STAGE, int GA>
struct Spec {
    static constexpr int stage_c = STAGE, ga_c = GA;
};
using RunSpec = Spec<-1, -1>;
template <class S, typename A>
__device__ __forceinline__ int st_of(const A &a)
{
    return S::stage_c >= 0 ? S::stage_c : a.stage;
}
template <class S, typename A>
__device__ __forceinline__ int ga_of(const A &a)
{
    return S::ga_c >= 0 ? S::ga_c : a.ga;
}

// T = gamma M^2 p / rho of a stage state from its primitives W0 = rho - rho_b
// and W4 = p - p_b at gravity coordinate kg (FP32: T_b (1 + p'/p_b) /
// (1 + rho'/rho_b), which keeps the deviations' digits)
template <typename T>
__device__ __forceinline__ T node_temperature(const VArgs<T> &a, int kg, T w0, T w4)
{
    if constexpr (sizeof(T) == 4) {
        // fixed-order arithmetic, like the fluxes: every kernel that forms a
        // node's temperature gets the same bits
        const float rr = __fmul_rn(w0, a.ir_b[kg]);
        return __fadd_rn(a.T_b[kg], __fdividef(__fmul_rn(a.T_b[kg], __fmaf_rn(w4, a.ip_b[kg], -rr)),
                                               __fadd_rn(1.0f, rr)));
    } else {
        return a.gm2 * (a.p_b[kg] + w4) / (a.rho_b[kg] + w0);
    }
}

// ---- four ring fields per node ------------------------------------------------
// A ring node holds (u, v, w, T) as one 16-byte (FP32) or 32-byte (FP64)
// vector, so the gradient of all four fields along an axis is two vector
// loads; the FP32 arithmetic on such vectors runs as packed FP32x2 operations.
struct alignas(32) dbl4 {
    double x, y, z, w;
};
template <typename T>
struct V4T;
template <>
struct V4T<float> {
    using type = float4;
};
template <>
struct V4T<double> {
    using type = dbl4;
};
template <typename T>
using V4 = typename V4T<T>::type;

// Scalar arithmetic in a fixed order (no contraction into FMAs the compiler
// might choose differently in different places): a flux evaluated at the same
// node from the same inputs gives the same bits in every block that needs it.
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ float2 lo2(const float4 &a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(const float4 &a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 cat4(float2 l, float2 h) { return make_float4(l.x, l.y, h.x, h.y); }

// a - b (as fma(b, -1, a): one rounding, the same as a subtraction)
__device__ __forceinline__ float4 v_sub(const float4 &a, const float4 &b)
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
    return cat4(__ffma2_rn(lo2(b), m1, lo2(a)), __ffma2_rn(hi2(b), m1, hi2(a)));
}
__device__ __forceinline__ float4 v_add(const float4 &a, const float4 &b)
{
    return cat4(__fadd2_rn(lo2(a), lo2(b)), __fadd2_rn(hi2(a), hi2(b)));
}
__device__ __forceinline__ float4 v_mul(const float4 &a, float s)
{
    const float2 s2 = make_float2(s, s);
    return cat4(__fmul2_rn(lo2(a), s2), __fmul2_rn(hi2(a), s2));
}
// a s + c
__device__ __forceinline__ float4 v_fma(const float4 &a, float s, const float4 &c)
{
    const float2 s2 = make_float2(s, s);
    return cat4(__ffma2_rn(lo2(a), s2, lo2(c)), __ffma2_rn(hi2(a), s2, hi2(c)));
}
__device__ __forceinline__ dbl4 v_sub(const dbl4 &a, const dbl4 &b)
{
    return dbl4{__dadd_rn(a.x, -b.x), __dadd_rn(a.y, -b.y), __dadd_rn(a.z, -b.z), __dadd_rn(a.w, -b.w)};
}
__device__ __forceinline__ dbl4 v_add(const dbl4 &a, const dbl4 &b)
{
    return dbl4{__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y), __dadd_rn(a.z, b.z), __dadd_rn(a.w, b.w)};
}
__device__ __forceinline__ dbl4 v_mul(const dbl4 &a, double s)
{
    return dbl4{__dmul_rn(a.x, s), __dmul_rn(a.y, s), __dmul_rn(a.z, s), __dmul_rn(a.w, s)};
}
__device__ __forceinline__ dbl4 v_fma(const dbl4 &a, double s, const dbl4 &c)
{
    return dbl4{__fma_rn(a.x, s, c.x), __fma_rn(a.y, s, c.y), __fma_rn(a.z, s, c.z), __fma_rn(a.w, s, c.w)};
}

// second-order differences of a ring vector: central (p+ - p-) / (2h) and the
// one-sided (-3 p0 + 4 p1 - p2) / (2h) at a low wall, (3 p0 - 4 p-1 + p-2) /
// (2h) at a high wall (ih = 1 / (2h))
template <typename V, typename T>
__device__ __forceinline__ V d_central(const V &pp, const V &pm, T ih)
{
    return v_mul(v_sub(pp, pm), ih);
}
template <typename V, typename T>
__device__ __forceinline__ V d_low(const V &p0, const V &p1, const V &p2, T ih)
{
    return v_mul(v_sub(v_fma(p1, T(4), v_mul(p0, T(-3))), p2), ih);
}
template <typename V, typename T>
__device__ __forceinline__ V d_high(const V &p0, const V &pm1, const V &pm2, T ih)
{
    return v_mul(v_add(v_fma(pm1, T(-4), v_mul(p0, T(3))), pm2), ih);
}

// Ask L2 for what the RK update of node p will load: its right-hand side and
// (mixed form) K, D_n and, in stage 4, Q_n.  Issued a plane ahead, these take
// the DRAM latency off the update, which runs after the plane's barrier; an L2
// prefetch holds no register.  (One bulk prefetch per tile row and field
// instead, from a few threads, was 18% slower for the whole kernel.)
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
template <typename T, class S>
__device__ __forceinline__ void prefetch_node(const VArgs<T> &a, int p)
{
    const int stage = st_of<S>(a);
#pragma unroll
    for (int k = 0; k < 5; ++k) prefetch_l2(a.R[k] + p);
    if constexpr (sizeof(T) == 4) {
        if (stage >= 2) {
#pragma unroll
            for (int k = 0; k < 5; ++k) prefetch_l2(a.Kacc[k] + p);
        }
        if (stage >= 1 && stage <= 3) {
#pragma unroll
            for (int k = 0; k < 5; ++k) prefetch_l2(a.Dn[k] + p);
        }
        if (stage == 4) {
#pragma unroll
            for (int k = 0; k < 5; ++k) prefetch_l2(a.Qn[k] + p);
        }
    }
}

template <typename T>
struct Ring {
    V4<T> *s;
    int x0, y0;
    __device__ __forceinline__ const V4<T> &at(int x, int y, int z) const
    {
        return s[(z % RING) * PLANE + (y - y0 + HALO) * PX + (x - x0 + HALO)];
    }
};

// A plane load split in two halves: issue() starts the global loads of this
// thread's ring nodes into registers, finish() computes T and writes the ring,
// so the loads are in flight while the thread does other work.  The in-plane
// part of each node's address is fixed per block and computed once.
constexpr int PL_PER_THREAD = (PLANE + TX * TY - 1) / (TX * TY);
template <typename T, class S>
struct PlaneLoad {
    int goff[PL_PER_THREAD];  // gx + nx * gy, or -1 outside the box / ring
    int kgxy[PL_PER_THREAD];  // gravity coordinate when gravity is along x or y
    T w0[PL_PER_THREAD], u[PL_PER_THREAD], v[PL_PER_THREAD], w[PL_PER_THREAD], w4[PL_PER_THREAD];
    int z;
    __device__ __forceinline__ void init(const VArgs<T> &a, const Ring<T> &rg)
    {
        const int nx = a.n[0], ny = a.n[1];
#pragma unroll
        for (int t = 0; t < PL_PER_THREAD; ++t) {
            const int idx = threadIdx.x + t * TX * TY;
            const int lx = idx % PX, ly = idx / PX;
            const int gx = rg.x0 - HALO + lx, gy = rg.y0 - HALO + ly;
            const bool ok = idx < PLANE && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
            goff[t] = ok ? gx + nx * gy : -1;
            kgxy[t] = ga_of<S>(a) == 0 ? gx : gy;
        }
    }
    __device__ __forceinline__ void issue(const VArgs<T> &a, int zz)
    {
        z = zz;
        const int zo = a.n[0] * a.n[1] * zz;
#pragma unroll
        for (int t = 0; t < PL_PER_THREAD; ++t) {
            if (goff[t] >= 0) {
                const int i = zo + goff[t];
                w0[t] = a.W[0][i];
                u[t] = a.W[1][i];
                v[t] = a.W[2][i];
                w[t] = a.W[3][i];
                w4[t] = a.W[4][i];
            }
        }
    }
    // ask L2 for plane zz's primitives of this thread's ring nodes (the plane
    // after the one being loaded, so its loads find them there)
    __device__ __forceinline__ void prefetch(const VArgs<T> &a, int zz) const
    {
        const int zo = a.n[0] * a.n[1] * zz;
#pragma unroll
        for (int t = 0; t < PL_PER_THREAD; ++t) {
            if (goff[t] >= 0) {
                const int i = zo + goff[t];
#pragma unroll
                for (int k = 0; k < 5; ++k) prefetch_l2(a.W[k] + i);
            }
        }
    }
    __device__ __forceinline__ void finish(const VArgs<T> &a, const Ring<T> &rg) const
    {
#pragma unroll
        for (int t = 0; t < PL_PER_THREAD; ++t) {
            const int idx = threadIdx.x + t * TX * TY;
            if (idx >= PLANE) continue;
            V4<T> q{};
            if (goff[t] >= 0) {
                const int kg = ga_of<S>(a) == 2 ? z : kgxy[t];
                q.x = u[t];
                q.y = v[t];
                q.z = w[t];
                q.w = node_temperature(a, kg, w0[t], w4[t]);
            }
            rg.s[(size_t)(z % RING) * PLANE + idx] = q;
        }
    }
};

// Second-order explicit derivatives of (u, v, w, T) at one node of the ring:
// central inside, one-sided (-3, 4, -1)/(2h) on a wall.  mode 0: central, 1:
// low wall (forward), 2: high wall (backward).  EDGE is false for blocks whose
// nodes are all at least one node away from the x and y walls, so only the z
// mode (uniform over a plane) is tested there.
template <typename T, bool EDGE>
struct Stencil {
    const V4<T> *b0, *bm1, *bp1, *bm2, *bp2;  // bases of planes j, j-1, j+1, j-2, j+2
    int off;                                  // ly * PX + lx
    int xm, ym, zm;
    T ihx, ihy, ihz;                          // 1 / (2 h)
    __device__ __forceinline__ V4<T> val() const { return b0[off]; }
    __device__ __forceinline__ V4<T> dx() const
    {
        const V4<T> *p = b0 + off;
        if (!EDGE || xm == 0) return d_central(p[1], p[-1], ihx);
        if (xm == 1) return d_low(p[0], p[1], p[2], ihx);
        return d_high(p[0], p[-1], p[-2], ihx);
    }
    __device__ __forceinline__ V4<T> dy() const
    {
        const V4<T> *p = b0 + off;
        if (!EDGE || ym == 0) return d_central(p[PX], p[-PX], ihy);
        if (ym == 1) return d_low(p[0], p[PX], p[2 * PX], ihy);
        return d_high(p[0], p[-PX], p[-2 * PX], ihy);
    }
    __device__ __forceinline__ V4<T> dz() const
    {
        if (zm == 0) return d_central(bp1[off], bm1[off], ihz);
        if (zm == 1) return d_low(b0[off], bp1[off], bp2[off], ihz);
        return d_high(b0[off], bm1[off], bm2[off], ihz);
    }
};

__device__ __forceinline__ int wall_mode(int c, int n) { return c == 0 ? 1 : (c == n - 1 ? 2 : 0); }

// Sutherland's law and Eq. reg (over mu_s), in a fixed order
template <typename T>
__device__ __forceinline__ void visc_coeffs(const VArgs<T> &a, T Tn, T &mu, T &mub)
{
    if constexpr (sizeof(T) == 4)
        mu = __fdividef(r_mul(r_mul(r_mul(Tn, Tn), rsqrtf(Tn)), a.S1), r_add(Tn, a.S));  // FP32 intrinsics
    else
        mu = r_mul(r_mul(Tn, sqrt(Tn)), a.S1) / r_add(Tn, a.S);
    mub = r_fma(a.c0, Tn, a.c1);
}

// the three viscosity factors of the stress (Eqs. ge19, bv1-bv3) divided by Re
template <typename T>
struct ViscK {
    T k43, k23, ks, mk;  // (4/3 mu + mu_b)/Re, (-2/3 mu + mu_b)/Re, mu/Re, -mu kq
    __device__ __forceinline__ ViscK(const VArgs<T> &a, T Tn)
    {
        T mu, mub;
        visc_coeffs(a, Tn, mu, mub);
        k43 = r_mul(r_fma(T(4) / T(3), mu, mub), a.iRe);
        k23 = r_mul(r_fma(T(-2) / T(3), mu, mub), a.iRe);
        ks = r_mul(mu, a.iRe);
        mk = r_mul(-mu, a.kq);
    }
};

// Viscous fluxes at a node from its values q = (u, v, w, T) and the
// gradients gx, gy, gz of (u, v, w, T) (Eqs. ge6-ge8, ge19, ge20, bv1-bv3).
// The heat flux normal to an adiabatic wall is zero on the wall node (wq = 0).
template <typename T>
__device__ __forceinline__ V4<T> flux_E(const ViscK<T> &k, const V4<T> &q, const V4<T> &gx, const V4<T> &gy,
                                        const V4<T> &gz, bool wq)
{
    const T txx = r_fma(k.k43, gx.x, r_mul(k.k23, r_add(gy.y, gz.z)));
    const T txy = r_mul(k.ks, r_add(gy.x, gx.y));
    const T txz = r_mul(k.ks, r_add(gz.x, gx.z));
    const T qx = wq ? r_mul(k.mk, gx.w) : T(0);
    return V4<T>{txx, txy, txz, r_add(r_fma(q.z, txz, r_fma(q.y, txy, r_mul(q.x, txx))), -qx)};
}
template <typename T>
__device__ __forceinline__ V4<T> flux_F(const ViscK<T> &k, const V4<T> &q, const V4<T> &gx, const V4<T> &gy,
                                        const V4<T> &gz, bool wq)
{
    const T tyy = r_fma(k.k43, gy.y, r_mul(k.k23, r_add(gx.x, gz.z)));
    const T txy = r_mul(k.ks, r_add(gy.x, gx.y));
    const T tyz = r_mul(k.ks, r_add(gz.y, gy.z));
    const T qy = wq ? r_mul(k.mk, gy.w) : T(0);
    return V4<T>{txy, tyy, tyz, r_add(r_fma(q.z, tyz, r_fma(q.y, tyy, r_mul(q.x, txy))), -qy)};
}
template <typename T>
__device__ __forceinline__ V4<T> flux_G(const ViscK<T> &k, const V4<T> &q, const V4<T> &gx, const V4<T> &gy,
                                        const V4<T> &gz, bool wq)
{
    const T tzz = r_fma(k.k43, gz.z, r_mul(k.k23, r_add(gx.x, gy.y)));
    const T txz = r_mul(k.ks, r_add(gz.x, gx.z));
    const T tyz = r_mul(k.ks, r_add(gz.y, gy.z));
    const T qz = wq ? r_mul(k.mk, gz.w) : T(0);
    return V4<T>{txz, tyz, tzz, r_add(r_fma(q.z, tzz, r_fma(q.y, tyz, r_mul(q.x, txz))), -qz)};
}



// primitives of a stage state from its FP32 deviation D = (rho', m_x, m_y, m_z, E')
__device__ __forceinline__ void prim_from_dev(const VArgs<float> &a, int p, int kg, const float D[5])
{
    float Wv[6];
    prim_from_deviation(a.rho_b[kg], a.gm1, D, Wv);
#pragma unroll
    for (int k = 0; k < 6; ++k) a.Wn[k][p] = Wv[k];
}

// Mixed form of the classical RK4 stage.  The slopes are FP32 (they are FP32
// right-hand sides); K = k1 + 2 k2 + 2 k3 + k4 is accumulated in FP32 and added
// to the FP64 state once, Q_n += dt/6 K, in FP64.  The stage states
// Q_n + c dt k are formed as FP32 deviations from the hydrostatic base, the
// same quantities the primitive recovery of the FP64 form rounds to FP32.
template <class S>
__device__ __forceinline__ void mixed_update(const VArgs<float> &a, int p, int kg, const float r[5],
                                             const float kold[5], const float dn[5])
{
    const int s = st_of<S>(a);
    float K[5];
    if (s == 1) {
#pragma unroll
        for (int k = 0; k < 5; ++k) K[k] = r[k];
    } else {
        const float w = s == 4 ? 1.0f : 2.0f;
#pragma unroll
        for (int k = 0; k < 5; ++k) K[k] = __fmaf_rn(w, r[k], kold[k]);
    }
    float D[5];
    if (s < 4) {
#pragma unroll
        for (int k = 0; k < 5; ++k) a.Kacc[k][p] = K[k];
        const float c = s == 3 ? a.cdt1 : a.cdt2;
#pragma unroll
        for (int k = 0; k < 5; ++k) D[k] = __fmaf_rn(c, r[k], dn[k]);
    } else {
        const double w6 = a.dt6;
        double q[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            q[k] = __fma_rn(w6, widen_f32(K[k]), a.Qn[k][p]);
            a.Qn[k][p] = q[k];
        }
        D[0] = narrow_f64(q[0] - a.rho_b64[kg]);
        D[1] = narrow_f64(q[1]);
        D[2] = narrow_f64(q[2]);
        D[3] = narrow_f64(q[3]);
        D[4] = narrow_f64(q[4] - a.E_b64[kg]);
#pragma unroll
        for (int k = 0; k < 5; ++k) a.Dn[k][p] = D[k];
    }
    prim_from_dev(a, p, kg, D);
}

// Gravity source (Eq. ge8a), no-slip walls and the RK4 stage at node p, whose
// right-hand side r holds every other term.  w0 = rho - rho_b, ug = the
// velocity along gravity; kd, dn (mixed form) = the node's K and D_n.
template <typename T, class S = RunSpec>
__device__ __forceinline__ void source_and_stage(const VArgs<T> &a, int p, int kg, bool wall, T w0, T ug, T r[5],
                                                 const float kd[5], const float dn[5])
{
    const int ga = ga_of<S>(a), stage = st_of<S>(a);
    // fixed-order arithmetic: the same bits whether the stage and the gravity
    // axis are compile-time constants (Spec) or not
    const T rho = r_add(a.rho_b[kg], w0);
    const T sg = r_mul(w0, a.g);
    if (ga == 0) r[1] = r_add(r[1], -sg);
    if (ga == 1) r[2] = r_add(r[2], -sg);
    if (ga == 2) r[3] = r_add(r[3], -sg);
    r[4] = r_add(r[4], -r_mul(r_mul(rho, ug), a.g));
    // no-slip walls
    if (wall) r[1] = r[2] = r[3] = 0;
    if (stage == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) a.Rout[k][p] = r[k];
    } else if constexpr (sizeof(T) == 4) {
        mixed_update<S>(a, p, kg, r, kd, dn);
    } else {
        // classical RK4: acc collects Q_n + dt (k1 + 2 k2 + 2 k3 + k4) / 6
        const double bw = (stage == 1 || stage == 4) ? a.dt6 : a.dt3;
        const double cw = stage == 3 ? a.dt : a.dt2;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const double rk = (double)r[k];
            if (stage == 1) {
                const double q = a.Qn[k][p];
                a.acc[k][p] = __fma_rn(bw, rk, q);
                a.Qout[k][p] = __fma_rn(cw, rk, q);
            } else if (stage < 4) {
                a.acc[k][p] = __fma_rn(bw, rk, a.acc[k][p]);
                a.Qout[k][p] = __fma_rn(cw, rk, a.Qn[k][p]);
            } else {
                a.Qout[k][p] = __fma_rn(bw, rk, a.acc[k][p]);
            }
        }
    }
}


template <typename T, bool EDGE, class S>
__device__ __forceinline__ void visc_rk_body(const VArgs<T> &a, const unsigned bx, const unsigned by,
                                             const unsigned bz, unsigned char *smraw)
{
    const int stage = st_of<S>(a), ga = ga_of<S>(a);
    using V = V4<T>;
    constexpr int EW = TX + 2, FH = TY + 2;  // E_v row width, F_v rows (one-node halos)
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
    const int xs = bx * TX, ys = by * TY;  // unsigned block coordinates, as blockIdx
    Ring<T> rg;
    rg.s = reinterpret_cast<V *>(smraw);
    rg.x0 = min(xs, max(nx - TX, 0));
    rg.y0 = min(ys, max(ny - TY, 0));
    constexpr bool AHEAD = flux_ahead<T>();
    constexpr int EFS = ef_slots<T>();
    V *EV = rg.s + (size_t)RING * PLANE;  // [EFS][TY][EW], local x + 1
    V *FV = EV + EFS * TY * EW;           // [EFS][FH][TX], local y + 1
    V *GV = FV + EFS * FH * TX;           // [GSLOTS][TY][TX]
    const int z0 = bz * a.zc, z1 = min(nz, z0 + a.zc);
    const int tx = (int)(threadIdx.x % TX), ty = (int)(threadIdx.x / TX);
    const int x = rg.x0 + tx, y = rg.y0 + ty;
    // a block off the x and y walls (EDGE false) is never shifted back and
    // owns all its nodes, halo nodes included, inside the box
    const bool in_dom = !EDGE || (x < nx && y < ny);
    const bool own = !EDGE || (in_dom && x >= xs && y >= ys);
    // G_v planes are computed in increasing order; ghi is the last one, and
    // the ring holds the GSLOTS planes up to it; efhi is the last plane whose
    // E_v and F_v are held (plane j in slot j mod EFS)
    int ghi = -1000, efhi = -1000;

    // ring bases of planes o-3 .. o+3, refreshed once per plane (plane o + d
    // sits in slot (o + d) mod RING; o+-3 share the slots of o-+2, and a
    // stencil reaches o+-3 only next to a wall, where o-+2 lies outside the box)
    const V *pb0, *pb1, *pb2, *pb3, *pb4, *pb5, *pb6;
    auto pbase = [&](int k) -> const V * {  // k = d + 3, 0..6
        switch (k) {
        case 0: return pb0;
        case 1: return pb1;
        case 2: return pb2;
        case 3: return pb3;
        case 4: return pb4;
        case 5: return pb5;
        default: return pb6;
        }
    };
    // stencil at local (lx, ly) of plane j = o + dz, |dz| <= 2 (planes outside
    // the box are never dereferenced: the z mode picks the one-sided form)
    auto stencil_at = [&](int lx, int ly, int dz, int j) {
        Stencil<T, EDGE> St;
        St.b0 = pbase(dz + 3);
        St.bm1 = pbase(dz + 2);
        St.bp1 = pbase(dz + 4);
        St.bm2 = pbase(dz >= -1 ? dz + 1 : dz + 3);
        St.bp2 = pbase(dz <= 1 ? dz + 5 : dz + 3);
        St.off = (ly + HALO) * PX + (lx + HALO);
        St.xm = EDGE ? wall_mode(rg.x0 + lx, nx) : 0;
        St.ym = EDGE ? wall_mode(rg.y0 + ly, ny) : 0;
        St.zm = wall_mode(j, nz);
        St.ihx = a.ih2[0];
        St.ihy = a.ih2[1];
        St.ihz = a.ih2[2];
        return St;
    };

    PlaneLoad<T, S> pl;
    pl.init(a, rg);
    // planes the first output plane needs: z0-2 .. z0+2, and up to z0+3
    // (down to z0-3) when it is the bottom (top) wall, for the G_v plane two
    // nodes in; later planes load one plane ahead, up to o+3, into the slot of
    // o-2, which no later plane reads
    int lhi = min(nz - 1, max(z0 + 2, 3));
    for (int z = max(0, min(z0 - 2, nz - 4)); z <= lhi; ++z) {
        pl.issue(a, z);
        pl.finish(a, rg);
    }
    __syncthreads();
    for (int o = z0; o < z1; ++o) {
        {
            const int so = o % RING;
            auto sb = [&](int d) {
                int t = so + d;
                t = t >= RING ? t - RING : (t < 0 ? t + RING : t);
                return (const V *)(rg.s + (size_t)t * PLANE);
            };
            pb0 = sb(-3);
            pb1 = sb(-2);
            pb2 = sb(-1);
            pb3 = sb(0);
            pb4 = sb(1);
            pb5 = sb(2);
            pb6 = sb(3);
        }
        // ---- 1. nodal viscous fluxes ------------------------------------------
        // fluxes_at(dz, wantEF, wantG): the requested fluxes of plane j = o + dz
        // at this thread's node from one stencil; with wantEF also F_v on the
        // y halo (warps 0-1) and E_v on the x halo (warp 2), with the same
        // arithmetic as in the tile that owns the node, so the same bits, and
        // no warp evaluating more than one halo flux per plane
        auto fluxes_at = [&](const int dz, const bool wantEF, const bool wantG) {
            const int j = o + dz;
            const int es = j & (EFS - 1);
            V *ev = EV + es * TY * EW, *fv = FV + es * FH * TX;
            if (in_dom) {
                const Stencil<T, EDGE> St = stencil_at(tx, ty, dz, j);
                const V q = St.val(), gx = St.dx(), gy = St.dy(), gz = St.dz();
                const ViscK<T> k(a, q.w);
                if (wantEF) {
                    ev[ty * EW + tx + 1] = flux_E(k, q, gx, gy, gz, St.xm == 0);
                    fv[(ty + 1) * TX + tx] = flux_F(k, q, gx, gy, gz, St.ym == 0);
                }
                if (wantG) GV[((j % GSLOTS) * TY + ty) * TX + tx] = flux_G(k, q, gx, gy, gz, St.zm == 0);
            }
            if (!wantEF) return;
            if (threadIdx.x < 2 * TX) {  // F_v on the y halo
                const int t = threadIdx.x;
                const int side = t / TX, hx = t % TX;
                const int ly = side ? TY : -1;
                const int gxx = rg.x0 + hx, gyy = rg.y0 + ly;
                if (!EDGE || (gyy >= 0 && gyy < ny && gxx < nx)) {
                    const Stencil<T, EDGE> St = stencil_at(hx, ly, dz, j);
                    const V q = St.val(), gx = St.dx(), gy = St.dy(), gz = St.dz();
                    fv[(ly + 1) * TX + hx] = flux_F(ViscK<T>(a, q.w), q, gx, gy, gz, St.ym == 0);
                }
            } else if (threadIdx.x < 2 * TX + 2 * TY) {  // E_v on the x halo
                const int t = threadIdx.x - 2 * TX;
                const int side = t / TY, hy = t % TY;
                const int lx = side ? TX : -1;
                const int gxx = rg.x0 + lx, gyy = rg.y0 + hy;
                if (!EDGE || (gxx >= 0 && gxx < nx && gyy < ny)) {
                    const Stencil<T, EDGE> St = stencil_at(lx, hy, dz, j);
                    const V q = St.val(), gx = St.dx(), gy = St.dy(), gz = St.dz();
                    ev[hy * EW + lx + 1] = flux_E(ViscK<T>(a, q.w), q, gx, gy, gz, St.xm == 0);
                }
            }
        };
        // the divergence of plane o needs E_v, F_v of plane o and G_v of o-1 and
        // o+1, or of o..o+2 / o-2..o on a z wall: all of jlo..jlo+2
        const int zw = wall_mode(o, nz);
        const int jlo = zw == 1 ? o : (zw == 2 ? o - 2 : o - 1);
        if (zw == 0 && ghi == o && (!AHEAD || efhi == o)) {
            // steady state away from the z walls, plane offsets known at compile
            // time: all three fluxes of plane o+1 (FP64: E_v, F_v of plane o and
            // G_v of plane o+1)
            if constexpr (AHEAD) {
                fluxes_at(1, true, true);
                efhi = o + 1;
            } else {
                fluxes_at(0, true, false);
                fluxes_at(1, false, true);
                efhi = o;
            }
            ghi = o + 1;
        } else {
            for (int j = jlo; j <= jlo + 2; ++j) {
                const bool wantG = j > ghi;
                const bool wantEF = j > efhi && (j == o || (AHEAD && j == o + 1));
                if (!wantG && !wantEF) continue;
                fluxes_at(j - o, wantEF, wantG);
                if (wantG) ghi = j;
                if (wantEF) efhi = j;
            }
        }
        // the node's own inputs of phase 2, loaded before the barrier so that
        // they are in flight while the block waits at it
        const int p = x + nx * (y + ny * o);
        T r[5], w0 = T(0);
        float kd[5], dn[5];
        if (own) {
#pragma unroll
            for (int k = 0; k < 5; ++k) r[k] = a.R[k][p];
            w0 = a.W[0][p];
            if constexpr (sizeof(T) == 4) {
                if (stage >= 2) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) kd[k] = a.Kacc[k][p];
                }
                if (stage >= 1 && stage <= 3) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) dn[k] = a.Dn[k][p];
                }
            }
        }
        __syncthreads();
        // ---- 2. divergence, source, RK stage; next plane's primitives ----------
        const int zn = lhi + 1;
        const bool next = o + 1 < z1 && zn < nz && zn <= o + 3;
        if (next) pl.issue(a, zn);
        if (next && zn + 1 < nz && zn + 1 <= o + 4 && o + 2 < z1) pl.prefetch(a, zn + 1);  // the next issue's plane
        if (own && o + 1 < z1) prefetch_node<T, S>(a, x + nx * (y + ny * (o + 1)));
        if (own) {
            const int xm = EDGE ? wall_mode(x, nx) : 0, ym = EDGE ? wall_mode(y, ny) : 0;
            const T ihx = a.ih2[0], ihy = a.ih2[1], ihz = a.ih2[2];
            const int es = o & (EFS - 1);
            const V *e = EV + es * TY * EW + ty * EW + tx + 1;
            const V *f = FV + es * FH * TX + (ty + 1) * TX + tx;
            V dvx, dvy, dvz;
            if (xm == 0)
                dvx = d_central(e[1], e[-1], ihx);
            else if (xm == 1)
                dvx = d_low(e[0], e[1], e[2], ihx);
            else
                dvx = d_high(e[0], e[-1], e[-2], ihx);
            if (ym == 0)
                dvy = d_central(f[TX], f[-TX], ihy);
            else if (ym == 1)
                dvy = d_low(f[0], f[TX], f[2 * TX], ihy);
            else
                dvy = d_high(f[0], f[-TX], f[-2 * TX], ihy);
            // G_v planes o-2 .. o+2 sit in slots (o + d) mod GSLOTS
            const V *g = GV + ty * TX + tx;
            const int sm1 = (o + 2) % GSLOTS, sp1 = (o + 1) % GSLOTS, s0 = o % GSLOTS;
            if (zw == 0)
                dvz = d_central(g[sp1 * TY * TX], g[sm1 * TY * TX], ihz);
            else if (zw == 1)  // planes o, o+1, o+2
                dvz = d_low(g[s0 * TY * TX], g[sp1 * TY * TX], g[sm1 * TY * TX], ihz);
            else  // planes o, o-1, o-2
                dvz = d_high(g[s0 * TY * TX], g[sm1 * TY * TX], g[sp1 * TY * TX], ihz);
            const V dv = v_add(v_add(dvx, dvy), dvz);
            r[1] = r_add(r[1], dv.x);
            r[2] = r_add(r[2], dv.y);
            r[3] = r_add(r[3], dv.z);
            r[4] = r_add(r[4], dv.w);
            const int kg = ga == 0 ? x : (ga == 1 ? y : o);
            const bool wall = (EDGE && (x == 0 || x == nx - 1 || y == 0 || y == ny - 1)) || o == 0 || o == nz - 1;
            const V qo = rg.at(x, y, o);
            source_and_stage<T, S>(a, p, kg, wall, w0, ga == 0 ? qo.x : (ga == 1 ? qo.y : qo.z), r, kd, dn);
        }
        if (next) {
            pl.finish(a, rg);
            lhi = zn;
        }
        __syncthreads();
    }
}

// One block (bx, by, bz) of the fused viscous / source / RK stage kernel:
// blocks whose x and y ranges (with the one-node flux halo) stay off the walls
// take the branch-free stencils.
template <typename T, class S = RunSpec>
__device__ __forceinline__ void visc_rk_block(const VArgs<T> &a, const unsigned bx, const unsigned by,
                                              const unsigned bz, unsigned char *smraw)
{
    const int nx = a.n[0], ny = a.n[1];
    const int x0 = min(bx * TX, max(nx - TX, 0)), y0 = min(by * TY, max(ny - TY, 0));
    const bool edge = x0 - 1 <= 0 || x0 + TX >= nx - 1 || y0 - 1 <= 0 || y0 + TY >= ny - 1;
    if (edge)
        visc_rk_body<T, true, S>(a, bx, by, bz, smraw);
    else
        visc_rk_body<T, false, S>(a, bx, by, bz, smraw);
}

template <typename T>
size_t ring_bytes()
{
    return ((size_t)RING * NPF * PLANE + ef_slots<T>() * (4 * TY * (TX + 2) + 4 * (TY + 2) * TX) +
            (size_t)GSLOTS * 4 * TY * TX) *
           sizeof(T);
}

template <typename T>
VArgs<T> make_vargs(const BoxDev &bx, const T *W, const T *R, int stage, const StageRegs<T> &g)
{
    VArgs<T> a{};
    for (int d = 0; d < 3; ++d) {
        a.n[d] = bx.n[d];
        a.ih2[d] = (T)(0.5 * bx.inv_h[d]);
    }
    a.np = (int)bx.np;
    a.ga = bx.ga;
    a.gm2 = (T)bx.gm2;
    a.iRe = (T)(1.0 / bx.Re);
    a.kq = (T)bx.kq;
    a.S1 = (T)(1.0 + bx.suth_S);
    a.S = (T)bx.suth_S;
    a.c0 = (T)bx.mub_coef0;
    a.c1 = (T)bx.mub_coef1;
    a.g = (T)bx.g;
    for (int k = 0; k < 6; ++k) a.W[k] = W + (size_t)k * bx.np;
    if constexpr (sizeof(T) == 8) {
        a.rho_b = (const T *)bx.rho_b64;
        a.p_b = (const T *)bx.p_b64;
    } else {
        a.rho_b = (const T *)bx.rho_b32;
    }
    a.T_b = bx.T_b32;
    a.ip_b = bx.ip_b32;
    a.ir_b = bx.ir_b32;
    for (int k = 0; k < 5; ++k) a.R[k] = R + (size_t)k * bx.np;
    a.stage = stage;
    a.dt = bx.dt;
    a.dt6 = bx.dt / 6.0;
    a.dt3 = bx.dt / 3.0;
    a.dt2 = 0.5 * bx.dt;
    a.cdt2 = (float)(0.5 * bx.dt);
    a.cdt1 = (float)bx.dt;
    auto fp = [&](auto *base, int k) { return base ? base + (size_t)k * bx.np : base; };
    for (int k = 0; k < 5; ++k) {
        a.Rout[k] = fp(g.Rout, k);
        a.Qn[k] = fp(g.Qn, k);
        a.acc[k] = fp(g.acc, k);
        a.Qout[k] = fp(g.Qout, k);
        a.Kacc[k] = fp(g.Kacc, k);
        a.Dn[k] = fp(g.Dn, k);
    }
    for (int k = 0; k < 6; ++k) a.Wn[k] = fp(g.Wn, k);
    a.rho_b64 = bx.rho_b64;
    a.E_b64 = bx.E_b64;
    a.gm1 = (float)(bx.gamma - 1.0);
    return a;
}

}  // namespace

}  // namespace nopcs
