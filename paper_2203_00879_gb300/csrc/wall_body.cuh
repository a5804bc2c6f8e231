// Device side of the no-slip adiabatic wall conditions (a reading of Sec. 2,
// Fig. 1), shared by the stand-alone wall kernels (rk_kernels.cu) and the
// batched persistent kernel (batch_kernel.cu).
#pragma once

#include "nopcs_internal.cuh"

namespace nopcs {

namespace {

// ---------------------------------------------------------------------------
// No-slip adiabatic walls: momentum zero on every wall node (kept by the
// update), T_w = (4 T_1 - T_2) / 3 along the inward normal, averaged over the
// normals of edge and corner nodes; faces first, then edges from the faces,
// then corners from the edges.  E_w = rho_w T_w / (gamma (gamma-1) M^2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double temp_q(const BoxDev &bx, const double *Q, long long i)
{
    const long long np = bx.np;
    const double r = Q[i];
    const double ke = 0.5 * (Q[np + i] * Q[np + i] + Q[2 * np + i] * Q[2 * np + i] + Q[3 * np + i] * Q[3 * np + i]) / r;
    return bx.gm2 * (bx.gamma - 1.0) * (Q[4 * np + i] - ke) / r;
}

__device__ void set_wall_node(const BoxDev &bx, double *Q, const int c[3], float *Dn, float *Wf)
{
    const long long st[3] = {1, bx.n[0], (long long)bx.n[0] * bx.n[1]};
    const long long i = c[0] + st[1] * c[1] + st[2] * c[2];
    double Tw = 0.0;
    int nw = 0;
    for (int d = 0; d < 3; ++d) {
        long long s;
        if (c[d] == 0)
            s = st[d];
        else if (c[d] == bx.n[d] - 1)
            s = -st[d];
        else
            continue;
        Tw += (4.0 * temp_q(bx, Q, i + s) - temp_q(bx, Q, i + 2 * s)) / 3.0;
        ++nw;
    }
    Tw /= nw;
    const long long np = bx.np;
    Q[np + i] = Q[2 * np + i] = Q[3 * np + i] = 0.0;
    Q[4 * np + i] = Q[i] * Tw * bx.cE;
    if (Dn) {
        const int kg = c[bx.ga];
        const float D[5] = {(float)(Q[i] - bx.rho_b64[kg]), 0.0f, 0.0f, 0.0f, (float)(Q[4 * np + i] - bx.E_b64[kg])};
        float Wv[6];
        prim_from_deviation(bx.rho_b32[kg], (float)(bx.gamma - 1.0), D, Wv);
#pragma unroll
        for (int k = 0; k < 5; ++k) Dn[k * np + i] = D[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) Wf[k * np + i] = Wv[k];
    }
}

// ---------------------------------------------------------------------------
// The same wall conditions on an FP32 stage state held as W (mixed form):
// T = T_b + T' with T' = T_b (p'/p_b - rho'/rho_b) / (1 + rho'/rho_b), the
// extrapolated wall temperature kept as its difference dT from T_b at the
// node, and E_w - E_b = cE (rho' T_w + rho_b dT) (E_b = cE rho_b T_b).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float temp_dev_w(const BoxDev &bx, const float *W, long long i, int kg)
{
    const long long np = bx.np;
    const float rr = W[i] * bx.ir_b32[kg];
    return bx.T_b32[kg] * (W[4 * np + i] * bx.ip_b32[kg] - rr) / (1.0f + rr);
}

__device__ void set_wall_node_w(const BoxDev &bx, float *W, const int c[3])
{
    const long long st[3] = {1, bx.n[0], (long long)bx.n[0] * bx.n[1]};
    const long long i = c[0] + st[1] * c[1] + st[2] * c[2];
    const int kg = c[bx.ga];
    const float TbP = bx.T_b32[kg];
    float dT = 0.0f;
    int nw = 0;
    for (int d = 0; d < 3; ++d) {
        int sg;
        if (c[d] == 0)
            sg = 1;
        else if (c[d] == bx.n[d] - 1)
            sg = -1;
        else
            continue;
        const long long s = sg * st[d];
        int k1 = kg, k2 = kg;
        if (d == bx.ga) {
            k1 = kg + sg;
            k2 = kg + 2 * sg;
        }
        const float d1 = (bx.T_b32[k1] - TbP) + temp_dev_w(bx, W, i + s, k1);
        const float d2 = (bx.T_b32[k2] - TbP) + temp_dev_w(bx, W, i + 2 * s, k2);
        dT += (4.0f * d1 - d2) * (1.0f / 3.0f);
        ++nw;
    }
    dT /= (float)nw;
    const long long np = bx.np;
    const float rd = W[i];
    const float Ed = (float)bx.cE * (rd * (TbP + dT) + bx.rho_b32[kg] * dT);
    const float pd = (float)(bx.gamma - 1.0) * Ed;
    W[np + i] = W[2 * np + i] = W[3 * np + i] = 0.0f;
    W[4 * np + i] = pd;
    W[5 * np + i] = Ed + pd;
}

// face nodes: exactly one wall coordinate; node t of 2 (fx + fy + fz)
__host__ __device__ __forceinline__ long long face_count(const BoxDev &bx)
{
    const long long nx = bx.n[0], ny = bx.n[1], nz = bx.n[2];
    return 2 * ((ny - 2) * (nz - 2) + (nx - 2) * (nz - 2) + (nx - 2) * (ny - 2));
}
__device__ __forceinline__ void face_node(const BoxDev &bx, long long t, int c[3])
{
    const int nx = bx.n[0], ny = bx.n[1], nz = bx.n[2];
    const long long fx = (long long)(ny - 2) * (nz - 2), fy = (long long)(nx - 2) * (nz - 2),
                    fz = (long long)(nx - 2) * (ny - 2);
    long long q = t;
    if (q < 2 * fx) {
        int side = (int)(q / fx);
        q %= fx;
        c[0] = side ? nx - 1 : 0;
        c[1] = 1 + (int)(q % (ny - 2));
        c[2] = 1 + (int)(q / (ny - 2));
    } else if ((q -= 2 * fx) < 2 * fy) {
        int side = (int)(q / fy);
        q %= fy;
        c[1] = side ? ny - 1 : 0;
        c[0] = 1 + (int)(q % (nx - 2));
        c[2] = 1 + (int)(q / (nx - 2));
    } else {
        q -= 2 * fy;
        int side = (int)(q / fz);
        q %= fz;
        c[2] = side ? nz - 1 : 0;
        c[0] = 1 + (int)(q % (nx - 2));
        c[1] = 1 + (int)(q / (nx - 2));
    }
}

// edge nodes (two wall coordinates): edges along axis a, the other two axes
// at 0 or n - 1 (4 combinations); every edge node reads only face and
// interior nodes, so the edges run in parallel, and the corners, which read
// edge nodes, follow
__host__ __device__ __forceinline__ long long edge_count(const BoxDev &bx)
{
    return 4LL * (bx.n[0] - 2) + 4LL * (bx.n[1] - 2) + 4LL * (bx.n[2] - 2);
}
__device__ __forceinline__ void edge_node(const BoxDev &bx, long long t, int c[3])
{
    const int n[3] = {bx.n[0], bx.n[1], bx.n[2]};
    long long cnt[3];
    for (int a = 0; a < 3; ++a) cnt[a] = 4LL * (n[a] - 2);
    long long q = t;
    int a = 0;
    while (q >= cnt[a]) {
        q -= cnt[a];
        ++a;
    }
    const int combo = (int)(q / (n[a] - 2));
    const int along = 1 + (int)(q % (n[a] - 2));
    const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    c[a] = along;
    c[b1] = (combo & 1) ? n[b1] - 1 : 0;
    c[b2] = (combo & 2) ? n[b2] - 1 : 0;
}
__device__ __forceinline__ void corner_node(const BoxDev &bx, int t, int c[3])
{
    for (int d = 0; d < 3; ++d) c[d] = (t >> d) & 1 ? bx.n[d] - 1 : 0;
}

// one wall node: on the FP64 state Q (refreshing Dn and Wf when given), or,
// with Q == nullptr, on the FP32 stage primitives Ww
__device__ __forceinline__ void wall_node(const BoxDev &bx, const int c[3], double *Q, float *Dn, float *Wf, float *Ww)
{
    if (Q)
        set_wall_node(bx, Q, c, Dn, Wf);
    else
        set_wall_node_w(bx, Ww, c);
}

}  // namespace

}  // namespace nopcs
