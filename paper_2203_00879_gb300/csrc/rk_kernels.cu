// Point-wise and stencil kernels of one RK stage (arXiv 2203.00879, Sec. 2 and
// Sec. 4): primitive recovery, the second-order explicit viscous terms with
// bulk viscosity, the gravity source, the classical RK4 stage update in FP64,
// the no-slip adiabatic wall conditions, the initial state and the
// diagnostics reduction.
#include <math.h>

#include "fp_bits.cuh"
#include "wall_body.cuh"

namespace nopcs {

namespace {


__device__ __forceinline__ void coords(const BoxDev &bx, long long p, int c[3])
{
    c[0] = (int)(p % bx.n[0]);
    long long q = p / bx.n[0];
    c[1] = (int)(q % bx.n[1]);
    c[2] = (int)(q / bx.n[1]);
}

// ---------------------------------------------------------------------------
// Primitive recovery (Eqs. ge12, ge13, nondimensional): from the FP64 state to
// W = (rho - rho_b, u, v, w, p - p_b, E + p - H_b) in the compute precision,
// with (rho_b, p_b, H_b) the hydrostatic base in the base-subtracted form and
// zero in the plain form.  The mixed form takes the two large differences
// rho - rho_b and E - E_b in FP64 and the rest in FP32, using
// p - p_b = (gamma - 1)(E - E_b - rho |V|^2 / 2) and H - H_b = (E - E_b) + (p - p_b).
// ---------------------------------------------------------------------------
// W (and the deviation D_n, mixed form) of one point of the FP64 state
template <typename T>
__device__ __forceinline__ void prep_point(const BoxDev &bx, long long p, int kg, double r, double mx, double my,
                                           double mz, double E, T *__restrict__ W, float *__restrict__ Dn)
{
    const long long np = bx.np;
    if constexpr (sizeof(T) == 8) {
        const double u = mx / r, v = my / r, w = mz / r;
        const double pr = (bx.gamma - 1.0) * (E - 0.5 * (mx * u + my * v + mz * w));
        W[p] = r - bx.rho_b64[kg];
        W[np + p] = u;
        W[2 * np + p] = v;
        W[3 * np + p] = w;
        W[4 * np + p] = pr - bx.p_b64[kg];
        W[5 * np + p] = E + pr - bx.H_b64[kg];
    } else {
        // deviation of the state from the hydrostatic base (mixed form), then
        // the primitives from it exactly as the stage kernels form them
        const float D[5] = {(float)(r - bx.rho_b64[kg]), (float)mx, (float)my, (float)mz,
                            (float)(E - bx.E_b64[kg])};
        float Wv[6];
        prim_from_deviation(bx.rho_b32[kg], (float)(bx.gamma - 1.0), D, Wv);
#pragma unroll
        for (int k = 0; k < 6; ++k) W[k * np + p] = Wv[k];
        if (Dn) {
#pragma unroll
            for (int k = 0; k < 5; ++k) Dn[k * np + p] = D[k];
        }
    }
}

// grid-stride over (y, z) rows, threads along x: no 64-bit division per point
template <typename T>
__global__ void prep_kernel(const BoxDev bx, const double *__restrict__ Q, T *__restrict__ W,
                            float *__restrict__ Dn)
{
    const long long np = bx.np;
    const int nx = bx.n[0], ny = bx.n[1], rows = bx.n[1] * bx.n[2];
    for (int rw = blockIdx.x; rw < rows; rw += gridDim.x) {
        const int y = rw % ny, z = rw / ny;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const long long p = (long long)rw * nx + x;
            const int kg = bx.ga == 0 ? x : (bx.ga == 1 ? y : z);
            prep_point<T>(bx, p, kg, Q[p], Q[np + p], Q[2 * np + p], Q[3 * np + p], Q[4 * np + p], W, Dn);
        }
    }
}

// Mixed-form filter (Sec. 4): the FP32 deviation D_n was filtered into Fd;
// the state takes the change Fd - D_n in FP64, so its low-order bits survive,
// and W0 and D_n are recomputed from the new state.
__global__ void filter_update_kernel(const BoxDev bx, double *__restrict__ Q, const float *__restrict__ Fd,
                                     float *__restrict__ W, float *__restrict__ Dn)
{
    const long long np = bx.np;
    const int nx = bx.n[0], ny = bx.n[1], rows = bx.n[1] * bx.n[2];
    for (int rw = blockIdx.x; rw < rows; rw += gridDim.x) {
        const int y = rw % ny, z = rw / ny;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const long long p = (long long)rw * nx + x;
            const int kg = bx.ga == 0 ? x : (bx.ga == 1 ? y : z);
            double q[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                q[k] = Q[k * np + p] + (double)(Fd[k * np + p] - Dn[k * np + p]);
                Q[k * np + p] = q[k];
            }
            prep_point<float>(bx, p, kg, q[0], q[1], q[2], q[3], q[4], W, Dn);
        }
    }
}

__global__ void wall_face_kernel(const BoxDev bx, double *Q, float *Dn, float *Wf, float *Ww)
{
    const long long tot = face_count(bx);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int c[3];
        face_node(bx, t, c);
        wall_node(bx, c, Q, Dn, Wf, Ww);
    }
}

__global__ void wall_edge_kernel(const BoxDev bx, double *Q, float *Dn, float *Wf, float *Ww)
{
    const long long tot = edge_count(bx);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int c[3];
        edge_node(bx, t, c);
        wall_node(bx, c, Q, Dn, Wf, Ww);
    }
}

__global__ void wall_corner_kernel(const BoxDev bx, double *Q, float *Dn, float *Wf, float *Ww)
{
    if (threadIdx.x < 8) {
        int c[3];
        corner_node(bx, threadIdx.x, c);
        wall_node(bx, c, Q, Dn, Wf, Ww);
    }
}

// ---------------------------------------------------------------------------
// Initial state (Sec. 2, Fig. 1): quiescent hydrostatic two-temperature box
// plus a uniform velocity perturbation from SplitMix64 (Steele, Lea & Flood,
// 2014) used as a counter-based generator, value 3 p + component.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long c)
{
    unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void initial_state_kernel(const BoxDev bx, unsigned long long seed, double amp, double *Q)
{
    const long long np = bx.np;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np;
         p += (long long)gridDim.x * blockDim.x) {
        int c[3];
        coords(bx, p, c);
        const int kg = c[bx.ga];
        const double rho = bx.rho_h64[kg], pr = bx.p_h64[kg];
        double V[3] = {0.0, 0.0, 0.0};
        const bool wall = c[0] == 0 || c[0] == bx.n[0] - 1 || c[1] == 0 || c[1] == bx.n[1] - 1 || c[2] == 0 ||
                          c[2] == bx.n[2] - 1;
        if (!wall && amp != 0.0) {
            for (int k = 0; k < 3; ++k) {
                const unsigned long long z = splitmix64_at(seed, 3ull * (unsigned long long)p + k);
                const double U = (double)(z >> 11) * (1.0 / 9007199254740992.0);
                V[k] = amp * (2.0 * U - 1.0);
            }
        }
        Q[p] = rho;
        Q[np + p] = rho * V[0];
        Q[2 * np + p] = rho * V[1];
        Q[3 * np + p] = rho * V[2];
        Q[4 * np + p] = pr / (bx.gamma - 1.0) + 0.5 * rho * (V[0] * V[0] + V[1] * V[1] + V[2] * V[2]);
    }
}

// ---------------------------------------------------------------------------
// Diagnostics: per-block partials (fixed grid, fixed order), then one block.
// partial record: mass, mx, my, mz, energy, max|V|^2, max|dp|, max Mach^2, bad
// ---------------------------------------------------------------------------
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_REC = 10;

__global__ void diag_partial_kernel(const BoxDev bx, const double *__restrict__ Q, double *partial)
{
    __shared__ double sh[DIAG_REC][DIAG_THREADS];
    const long long np = bx.np;
    const int nx = bx.n[0], ny = bx.n[1], rows = bx.n[1] * bx.n[2];
    const double gm1 = bx.gamma - 1.0, igam = 1.0 / bx.gamma;
    // maxima of |V|^2 and Mach^2 are kept and their square roots taken once
    // in the final kernel (the square root is monotone).  The FP64 work per
    // point is what decides this kernel's time (GB300 runs FP64 at 1/64 of the
    // FP32 rate): the sums are FP64 at every point; the maxima are evaluated
    // in FP64 (1/rho by two Newton steps instead of a division, the Mach^2
    // division only where it can raise the maximum) only at the points that a
    // binary32 screen cannot rule out; the gravity-axis terms are taken once
    // per row where gravity is not along x.
    double v[DIAG_REC] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double v7t = 0.0;  // v[7] * 0.999999
    // FP32 screen for the maxima: a point goes through the FP64 evaluation
    // below only if its binary32 estimates, with margins well above their
    // rounding error, could reach the current maxima (or are not numbers);
    // the maxima are those of the FP64 values of the points that could raise
    // them, so they are the same as evaluating every point in FP64
    float v5f = 0.0f, v6f = 0.0f, v7f = 0.0f;
    bool screening = true;
    int nseen = 0, ncand = 0;
    const float gm1f = (float)gm1, igamf = (float)igam;
    for (int rw = blockIdx.x; rw < rows; rw += gridDim.x) {
        const int y = rw % ny, z = rw / ny;
        const long long base = (long long)rw * nx;
        // coordinate along gravity of the row (gravity along y or z)
        const int kr = bx.ga == 1 ? y : z;
        const double kgh_r = kr * bx.h[bx.ga];
        const double ph_r = bx.ga != 0 ? bx.p_h64[kr] : 0.0;
        // screen of |p - p_h|: p - p_h = (gamma - 1)(E - E_b - kinetic) + c
        // with c = (gamma - 1) E_b - p_h, so that the binary32 estimate resolves
        // disturbances far smaller than p itself
        const double Eb_r = bx.ga != 0 && bx.E_b64 ? bx.E_b64[kr] : 0.0;
        const float cf_r = narrow_f64(gm1 * Eb_r - ph_r);
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const long long p = base + x;
            const double kgh = bx.ga == 0 ? x * bx.h[0] : kgh_r;
            const double ph = bx.ga == 0 ? bx.p_h64[x] : ph_r;
            const double r = Q[p], mx = Q[np + p], my = Q[2 * np + p], mz = Q[3 * np + p], E = Q[4 * np + p];
            // not finite: exponent field all ones (infinity or NaN), tested on
            // the high words by integer operations instead of FP64 compares
            auto nonfinite = [](double q) { return ((unsigned)__double2hiint(q) & 0x7ff00000u) == 0x7ff00000u; };
            const bool bad = nonfinite(r) || nonfinite(mx) || nonfinite(my) || nonfinite(mz) || nonfinite(E);
            if (bad) v[8] = 1.0;
            v[0] += r;
            v[1] += mx;
            v[2] += my;
            v[3] += mz;
            v[4] += E + r * bx.g * kgh;
            // screen: |V|^2 to ~1e-6 relative; p to tol absolute (a few
            // binary32 ulps of |E| + |kinetic| + |p_h|, with room to spare),
            // so Mach^2 only where p is known to 1e-4 relative
            bool cand = true;
            if (screening) {
                const double Eb = bx.ga == 0 ? (bx.E_b64 ? bx.E_b64[x] : 0.0) : Eb_r;
                const float cf = bx.ga == 0 ? narrow_f64(gm1 * Eb - ph) : cf_r;
                const float rf = narrow_f64(r), mxf = narrow_f64(mx), myf = narrow_f64(my), mzf = narrow_f64(mz);
                const float Ef = narrow_f64(E), phf = narrow_f64(ph), dEf = narrow_f64(E - Eb);
                const float irf = __fdividef(1.0f, rf);
                const float s2f = (mxf * mxf + myf * myf + mzf * mzf) * (irf * irf);
                const float kinf = 0.5f * rf * s2f;
                const float prf = gm1f * (Ef - kinf);
                const float tol = 2e-6f * (fabsf(Ef) + fabsf(kinf) + fabsf(phf));
                // the disturbance pressure to 2e-6 of its own terms, plus 1e-14
                // of E and p_h for the rounding of the FP64 evaluation it
                // stands for
                const float dpf = fabsf(gm1f * (dEf - kinf) + cf);
                const float tol_dp =
                    2e-6f * (fabsf(dEf) + fabsf(kinf) + fabsf(cf)) + 1e-14f * (fabsf(Ef) + fabsf(phf));
                const float machf = __fdividef(s2f * rf * igamf, prf);
                cand = !(s2f < v5f) || !(dpf + tol_dp < v6f) || !(fabsf(prf) > 1e4f * tol) ||
                       !(machf * 1.0003f < v7f);
                // a state whose maxima sit at the FP64 rounding floor (a box at
                // rest) passes every point: the thread then stops screening
                ncand += cand ? 1 : 0;
                if (++nseen == 256) screening = 2 * ncand < nseen;
            }
            if (cand) {
                const double ir = recip_newton(r);
                const double u = mx * ir, vv = my * ir, w = mz * ir;
                const double s2 = u * u + vv * vv + w * w;
                const double pr = gm1 * (E - 0.5 * r * s2);
                v[5] = fmax(v[5], s2);
                v[6] = fmax(v[6], fabs(pr - ph));
                // Mach^2 = num / pr can raise the maximum only where num
                // exceeds v7 pr (for pr > 0; the factor 0.999999 keeps every
                // point whose rounded quotient could exceed v7).  Elsewhere the
                // quotient is at most v7, or not a number, and the maximum
                // stays as it is.
                const double num = s2 * r * igam;
                if (num > v7t * pr) {
                    v[7] = fmax(v[7], num / pr);
                    v7t = v[7] * 0.999999;
                }
                // thresholds a little below the maxima; none while a maximum is
                // too small for the binary32 estimates to resolve
                v5f = v[5] > 1e-30 ? narrow_f64(v[5]) * 0.99999f : 0.0f;
                v6f = narrow_f64(v[6]) * 0.99999f;
                v7f = v[7] > 1e-30 ? narrow_f64(v[7]) * 0.9999f : 0.0f;
            }
        }
    }
    for (int k = 0; k < DIAG_REC; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
            for (int k = 5; k < 9; ++k) sh[k][threadIdx.x] = fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x < DIAG_REC) partial[(size_t)blockIdx.x * DIAG_REC + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void diag_final_kernel(const BoxDev bx, const double *partial, int nblk, double *out)
{
    // one block: each thread folds a fixed stride of partial records, then a
    // fixed-shape tree; the reduction order never changes between calls
    __shared__ double sh[DIAG_REC][DIAG_THREADS];
    double v[DIAG_REC] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        const double *q = partial + (size_t)b * DIAG_REC;
        for (int k = 0; k < 5; ++k) v[k] += q[k];
        for (int k = 5; k < 9; ++k) v[k] = fmax(v[k], q[k]);
    }
    for (int k = 0; k < DIAG_REC; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int w = DIAG_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
            for (int k = 5; k < 9; ++k) sh[k][threadIdx.x] = fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double dV = bx.h[0] * bx.h[1] * bx.h[2];
        for (int k = 0; k < 5; ++k) out[k] = sh[k][0] * dV;
        out[5] = sqrt(sh[5][0]);
        out[6] = sh[6][0];
        out[7] = sqrt(sh[7][0]);
        out[8] = sh[8][0];
        out[9] = 0.0;
    }
}

int grid_for(long long work, int threads)
{
    long long b = (work + threads - 1) / threads;
    const long long cap = 152LL * 16;  // grid-stride beyond 16 blocks per SM
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

static int row_grid(const BoxDev &bx)
{
    const int rows = bx.n[1] * bx.n[2];
    return rows < 152 * 16 ? rows : 152 * 16;
}

template <typename T>
cudaError_t launch_prep(const BoxDev &bx, const double *Q, T *W, float *Dn, cudaStream_t st)
{
    prep_kernel<T><<<row_grid(bx), 256, 0, st>>>(bx, Q, W, Dn);
    return cudaGetLastError();
}

cudaError_t launch_filter_update(const BoxDev &bx, double *Q, const float *Fd, float *W, float *Dn, cudaStream_t st)
{
    filter_update_kernel<<<row_grid(bx), 256, 0, st>>>(bx, Q, Fd, W, Dn);
    return cudaGetLastError();
}

cudaError_t launch_wall_bc(const BoxDev &bx, double *Q, float *Dn, float *Wf, float *Ww, cudaStream_t st)
{
    const long long faces = 2LL * ((long long)(bx.n[1] - 2) * (bx.n[2] - 2) + (long long)(bx.n[0] - 2) * (bx.n[2] - 2) +
                                   (long long)(bx.n[0] - 2) * (bx.n[1] - 2));
    wall_face_kernel<<<grid_for(faces, 256), 256, 0, st>>>(bx, Q, Dn, Wf, Ww);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long edges = 4LL * ((bx.n[0] - 2) + (bx.n[1] - 2) + (bx.n[2] - 2));
    wall_edge_kernel<<<grid_for(edges, 256), 256, 0, st>>>(bx, Q, Dn, Wf, Ww);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    wall_corner_kernel<<<1, 32, 0, st>>>(bx, Q, Dn, Wf, Ww);
    return cudaGetLastError();
}

cudaError_t launch_initial_state(const BoxDev &bx, unsigned long long seed, double amp, double *Q,
                                 cudaStream_t st)
{
    initial_state_kernel<<<grid_for(bx.np, 256), 256, 0, st>>>(bx, seed, amp, Q);
    return cudaGetLastError();
}

int diag_blocks(long long np)
{
    (void)np;
    return 152 * 8;  // grid-stride over (y, z) rows: 8 blocks per SM
}

cudaError_t launch_diagnostics(const BoxDev &bx, const double *Q, double *partial, int nblk, double *out,
                               cudaStream_t st)
{
    diag_partial_kernel<<<nblk, DIAG_THREADS, 0, st>>>(bx, Q, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<1, DIAG_THREADS, 0, st>>>(bx, partial, nblk, out);
    return cudaGetLastError();
}

template cudaError_t launch_prep<float>(const BoxDev &, const double *, float *, float *, cudaStream_t);
template cudaError_t launch_prep<double>(const BoxDev &, const double *, double *, float *, cudaStream_t);
}  // namespace nopcs
