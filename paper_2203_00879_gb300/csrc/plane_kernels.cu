// Plane diagnostics of Sec. 4 (arXiv 2203.00879): the disturbance pressure
// p - p_h on a plane (the field of the paper's pressure figures) and the three
// right-hand-side terms of the inviscid vorticity transport equation, Eq.
// eqn12_1 -- vortex stretching (omega . grad) V, dilatation -omega (div V) and
// the baroclinic term (grad rho x grad p) / rho^2 -- on a plane (the paper
// plots them on the interface plane).  omega = curl V.  Gradients are the
// second-order explicit differences of the viscous terms: central inside,
// one-sided (-3, 4, -1) / (2h) on a wall.  FP64 throughout, from the FP64
// state; one thread per plane node.
#include "nopcs_internal.cuh"

namespace nopcs {

namespace {

struct Prim {
    double r, u, v, w, p;
};

__device__ __forceinline__ Prim prim_at(const BoxDev &bx, const double *__restrict__ Q, long long i)
{
    const long long np = bx.np;
    Prim q;
    q.r = Q[i];
    q.u = Q[np + i] / q.r;
    q.v = Q[2 * np + i] / q.r;
    q.w = Q[3 * np + i] / q.r;
    q.p = (bx.gamma - 1.0) * (Q[4 * np + i] - 0.5 * q.r * (q.u * q.u + q.v * q.v + q.w * q.w));
    return q;
}

// d/dx_d of the five primitives at node i (coordinate c along d)
__device__ void grad_axis(const BoxDev &bx, const double *__restrict__ Q, long long i, int d, int c, double g[5])
{
    const long long st = d == 0 ? 1 : (d == 1 ? (long long)bx.n[0] : (long long)bx.n[0] * bx.n[1]);
    const int N = bx.n[d];
    const double i2h = 1.0 / (2.0 * bx.h[d]);
    if (c == 0) {
        const Prim a = prim_at(bx, Q, i), b = prim_at(bx, Q, i + st), e = prim_at(bx, Q, i + 2 * st);
        g[0] = (-3.0 * a.r + 4.0 * b.r - e.r) * i2h;
        g[1] = (-3.0 * a.u + 4.0 * b.u - e.u) * i2h;
        g[2] = (-3.0 * a.v + 4.0 * b.v - e.v) * i2h;
        g[3] = (-3.0 * a.w + 4.0 * b.w - e.w) * i2h;
        g[4] = (-3.0 * a.p + 4.0 * b.p - e.p) * i2h;
    } else if (c == N - 1) {
        const Prim a = prim_at(bx, Q, i), b = prim_at(bx, Q, i - st), e = prim_at(bx, Q, i - 2 * st);
        g[0] = (3.0 * a.r - 4.0 * b.r + e.r) * i2h;
        g[1] = (3.0 * a.u - 4.0 * b.u + e.u) * i2h;
        g[2] = (3.0 * a.v - 4.0 * b.v + e.v) * i2h;
        g[3] = (3.0 * a.w - 4.0 * b.w + e.w) * i2h;
        g[4] = (3.0 * a.p - 4.0 * b.p + e.p) * i2h;
    } else {
        const Prim b = prim_at(bx, Q, i + st), e = prim_at(bx, Q, i - st);
        g[0] = (b.r - e.r) * i2h;
        g[1] = (b.u - e.u) * i2h;
        g[2] = (b.v - e.v) * i2h;
        g[3] = (b.w - e.w) * i2h;
        g[4] = (b.p - e.p) * i2h;
    }
}

__global__ void plane_fields_kernel(const BoxDev bx, const double *__restrict__ Q, int axis, int index, int what,
                                    double *__restrict__ out)
{
    const int ia = axis == 0 ? 1 : 0, ib = axis == 2 ? 1 : 2;
    const int na = bx.n[ia], nb = bx.n[ib];
    const long long plane = (long long)na * nb;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < plane;
         o += (long long)gridDim.x * blockDim.x) {
        int c[3];
        c[axis] = index;
        c[ia] = (int)(o % na);
        c[ib] = (int)(o / na);
        const long long i = c[0] + (long long)bx.n[0] * (c[1] + (long long)bx.n[1] * c[2]);
        if (what == 0) {
            out[o] = prim_at(bx, Q, i).p - bx.p_h64[c[bx.ga]];
            continue;
        }
        double g[3][5];  // g[d][q]: d(prim q)/dx_d, q = rho, u, v, w, p
        for (int d = 0; d < 3; ++d) grad_axis(bx, Q, i, d, c[d], g[d]);
        // G[i][j] = dV_i / dx_j
        const double G00 = g[0][1], G01 = g[1][1], G02 = g[2][1];
        const double G10 = g[0][2], G11 = g[1][2], G12 = g[2][2];
        const double G20 = g[0][3], G21 = g[1][3], G22 = g[2][3];
        const double om0 = G21 - G12, om1 = G02 - G20, om2 = G10 - G01;
        const double divv = G00 + G11 + G22;
        const double r = prim_at(bx, Q, i).r, ir2 = 1.0 / (r * r);
        const double dr0 = g[0][0], dr1 = g[1][0], dr2 = g[2][0];
        const double dp0 = g[0][4], dp1 = g[1][4], dp2 = g[2][4];
        out[0 * plane + o] = om0 * G00 + om1 * G01 + om2 * G02;
        out[1 * plane + o] = om0 * G10 + om1 * G11 + om2 * G12;
        out[2 * plane + o] = om0 * G20 + om1 * G21 + om2 * G22;
        out[3 * plane + o] = -om0 * divv;
        out[4 * plane + o] = -om1 * divv;
        out[5 * plane + o] = -om2 * divv;
        out[6 * plane + o] = (dr1 * dp2 - dr2 * dp1) * ir2;
        out[7 * plane + o] = (dr2 * dp0 - dr0 * dp2) * ir2;
        out[8 * plane + o] = (dr0 * dp1 - dr1 * dp0) * ir2;
    }
}

}  // namespace

cudaError_t launch_plane_fields(const BoxDev &bx, const double *Q, int axis, int index, int what, double *out,
                                cudaStream_t st)
{
    const int ia = axis == 0 ? 1 : 0, ib = axis == 2 ? 1 : 2;
    const long long plane = (long long)bx.n[ia] * bx.n[ib];
    long long blocks = (plane + 255) / 256;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    if (blocks < 1) blocks = 1;
    plane_fields_kernel<<<(unsigned)blocks, 256, 0, st>>>(bx, Q, axis, index, what, out);
    return cudaGetLastError();
}

}  // namespace nopcs
