// Internal declarations shared by the translation units of libnopcs.
// Nothing here is part of the public ABI (include/nopcs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nopcs.h"

namespace nopcs {

// KIND_D2: the sixth-order compact second derivative (a symmetric right-hand
// side like the filter's, explicit wall rows like the derivative's)
enum LineKind { KIND_DERIV = 0, KIND_FILTER = 1, KIND_D2 = 2 };
// MODE_FIELD2: one field through a KIND_D2 operator
// MODE_VGRAD: the derivatives of u, v, w, T (from the six stage primitives)
// MODE_VDIV: the derivatives of four viscous-flux fields, added into R[1..4]
enum LineMode { MODE_FIELD = 0, MODE_FLUX = 1, MODE_FILTER = 2, MODE_FIELD2 = 3, MODE_VGRAD = 4, MODE_VDIV = 5 };

// Per-sub-domain record of a line operator (ints, device array of nsub * SUB_REC).
//   [0] s, [1] e            sub-domain rows (inclusive)
//   [2] tile_lo, [3] tile_hi rows that the block stages in shared memory
//   [4] j0_s, [5] len_s, [6] off_s   end row at s: first column, taps, offset in coef
//   [7] j0_e, [8] len_e, [9] off_e   end row at e
//   [10] lo, [11] hi         implicit rows solved by Thomas (lo > hi: none)
//   [12] win_lo, [13] win_hi rows the solve reads (the end-row supports
//                            outside them are consumed while staging)
constexpr int SUB_REC = 14;

// Host copy of a line operator (Sec. 3): partition, end rows, Thomas factors.
struct LineOpHost {
    int N = 0, nsub = 0, nexp = 0, kind = 0, sub_n = 0;
    int maxm = 0, max_tile = 0, max_win = 0;
    double thresh = 0.0, alpha = 0.0;
    double rb[4] = {0, 0, 0, 0};  // interior right-hand-side weights
    double ex[3][5] = {};         // explicit rows next to the low wall (taps at 0..4)
    double ex_sign = 1.0;         // high wall row N-1-r = ex_sign * mirror of row r
    std::vector<int> sub;         // nsub * SUB_REC
    std::vector<double> coef;     // end-row taps
    std::vector<double> cp, inv;  // Thomas factors, maxm entries
    int max_taps = 0;             // longest end row
    int kconv64 = 0, kconv32 = 0; // factors of rows >= kconv equal the limit in that precision
};

// Banded explicit form of a line operator (all rows of the truncated global C).
struct BandHost {
    int N = 0, kind = 0;
    int h = 0;                   // interior half-width: taps at offsets -h .. h
    int in_lo = 0, in_hi = -1;   // rows in_lo .. in_hi use the interior stencil
    std::vector<double> stencil; // 2h + 1 taps
    int W = 0;                   // longest window of a tabulated row
    std::vector<int> wrow, wj0, wlen;  // tabulated rows, first column and length of their windows
    std::vector<double> wtap;    // W slots per tabulated row (taps, then zeros)
};
bool build_band_op(int N, int kind, double alpha_f, double thresh, BandHost &bh, std::string &msg);
void apply_band_host(const BandHost &bh, const double *f, double *g);
// Device copy of the FP32 banded tables (band_kernels.cu).
struct BandDev {
    const float *cg = nullptr;    // interior stencil, centred in the kernel's tap count
    const int *wj0 = nullptr;     // tabulated rows: first column of the window
    const int *wlen = nullptr;    // tabulated rows: window length
    const float *wtap = nullptr;  // tabulated rows: taps
};
struct BandBuf {
    BandHost host;
    BandDev dev;
    void *mem = nullptr;
    cudaError_t upload();
    void release();
};
// the FP32 band kernel handles the table (stencil width, window placement)
bool band_supported(const BandHost &h);
// out = scale * C_band f along `axis` (FP32)
cudaError_t launch_band_field(const BandBuf &op, int axis, const int n[3], const float *f, float *out, double scale,
                              cudaStream_t st);

// Device view passed by value to the line kernels.
struct LineOpDev {
    int N, nsub, nexp, maxm, max_tile, max_taps, max_win;
    int kconv64, kconv32;
    int ncoef;          // end-row taps in the coef tables
    int xpitch[2][4];   // whole-line x sweep: line pitch for 1 / 5 fields and 1..4 lines per block
    double cpL, invL;  // limits of the Thomas factors
    double alpha;
    double rb[4];
    double ex[3][5];
    double ex_sign;
    const int *sub;
    const double *coef64;
    const float *coef32;
    const double *cp64, *inv64;
    const float *cp32, *inv32;
};

// Builds the host tables; returns false (with msg) on bad sizes.
bool build_line_op(int N, int sub_n, int kind, double alpha_f, double thresh, LineOpHost &op,
                   std::string &msg);
int partition_rule(int N, int sub_n, int *start);

// FP64 host evaluation of a line operator (the arithmetic of the line kernels).
void apply_line_host(const LineOpHost &op, const double *f, double *g);

// Dense per-sub-domain operators for the tensor-core forms.  Sub-domain b maps
// its staging window [tile_lo, tile_lo + Kpad) to its n_b outputs:
// g = D_b f_window.  D_b is stored as B operands of tcgen05.mma (N = outputs,
// K = window), K-major, no swizzle, in two splits:
//   - TF32 hi and lo parts (3xTF32 form); element (n, k) of a block sits at
//     float offset (n / 8) * (Kpad / 4) * 32 + (k / 4) * 32 + (n % 8) * 4 + (k % 4);
//   - three BF16 parts, D = D1 + D2 + D3 (BF16x3 form), the window padded to
//     Kpad16 (a multiple of 16, the K of one kind::f16 MMA); element (n, k) at
//     16-bit offset (n / 8) * (Kpad16 / 8) * 64 + (k / 8) * 64 + (n % 8) * 8 + (k % 8).
struct DenseHost {
    int N = 0, nsub = 0, max_npad = 0, max_kpad = 0, max_kpad16 = 0;
    // per sub-domain: s, n_b, Npad, Kpad, window start, float offset, Kpad16,
    // 16-bit offset
    std::vector<int> rec;
    std::vector<float> hi, lo;            // concatenated TF32 parts
    std::vector<uint16_t> b16[3];         // concatenated BF16 parts (bit patterns)
};
constexpr int DENSE_REC = 8;
void build_dense_blocks(const LineOpHost &op, DenseHost &out);

// Device view of the dense blocks (tensor-core form).
struct GemmOpDev {
    int N, nsub, max_npad, max_kpad, max_kpad16;
    const int *rec;
    const float *hi, *lo;
    const uint16_t *b16[3];
};
struct GemmOpBuf {
    DenseHost host;
    GemmOpDev dev{};
    void *mem = nullptr;
    cudaError_t upload();
    void release();
};
cudaError_t init_gemm_kernels();
bool gemm_smem_fits(const DenseHost &h);
// FP32 field derivative by a tensor-core form, 3xTF32 (bf16x3 false) or BF16x3
// (true); err <- 1 if a bounded wait for the tensor cores gave up.
cudaError_t launch_gemm_field(const GemmOpDev &op, bool bf16x3, int axis, const int n[3], const float *f, float *out,
                              double scale, int *err, cudaStream_t st);

// Owns the device copy of a LineOpHost.
struct LineOpBuf {
    LineOpHost host;
    LineOpDev dev{};
    void *mem = nullptr;
    cudaError_t upload();
    void release();
};

// Physics constants of one box passed by value to kernels.
struct BoxDev {
    int n[3];
    long long np;
    double h[3], inv_h[3];
    int ga;            // gravity axis
    double gamma, gm2, Re, M, kq, suth_S, mub_coef0, mub_coef1, g;
    double cE;         // 1 / (gamma (gamma - 1) M^2)
    double dt;
    const double *rho_b64, *p_b64, *H_b64, *E_b64;  // base tables along ga (zeros if plain)
    const float *rho_b32, *p_b32, *H_b32;
    const float *T_b32, *ip_b32, *ir_b32;           // mixed form: T_b, 1/p_b, 1/rho_b
    const double *rho_h64, *p_h64;                  // hydrostatic profile (always)
    int *err;          // device error word: set by a kernel whose bounded wait gave up
};

// Mixed form: the FP32 primitives W = (rho', u, v, w, p', H') of a state from
// its FP32 deviation from the hydrostatic base, D = (rho - rho_b, m_x, m_y,
// m_z, E - E_b), with p' = (gamma - 1)(E' - rho |V|^2 / 2) and H' = E' + p'.
// Every kernel that forms the primitives of a stored state uses this one
// function, so a state has the same FP32 primitives whichever kernel computed
// them (a run resumed from nopcs_set_state continues bit for bit).
__device__ __forceinline__ void prim_from_deviation(float rho_b, float gm1, const float D[5], float Wv[6])
{
    // fixed-order arithmetic (no contraction left to the compiler)
    const float ir = __fdividef(1.0f, __fadd_rn(rho_b, D[0]));
    const float u = __fmul_rn(D[1], ir), v = __fmul_rn(D[2], ir), w = __fmul_rn(D[3], ir);
    const float ke = __fmul_rn(0.5f, __fmaf_rn(D[3], w, __fmaf_rn(D[2], v, __fmul_rn(D[1], u))));
    const float pd = __fmul_rn(gm1, __fadd_rn(D[4], -ke));
    Wv[0] = D[0];
    Wv[1] = u;
    Wv[2] = v;
    Wv[3] = w;
    Wv[4] = pd;
    Wv[5] = __fadd_rn(D[4], pd);
}

// ---- launchers (line_kernels.cu) -------------------------------------------
// Raises the dynamic shared-memory limit of every line-kernel instantiation
// on the current device (called once per context, outside stream capture).
cudaError_t init_line_kernels();
// FIELD: out = scale * L f.  T = float or double.
template <typename T>
cudaError_t launch_line_field(const LineOpDev &op, int axis, const int n[3], const T *f, T *out,
                              double scale, cudaStream_t st);
// FIELD2: out = scale * L2 f with a KIND_D2 operator (scale = 1 / h^2).
template <typename T>
cudaError_t launch_line_field2(const LineOpDev &op, int axis, const int n[3], const T *f, T *out, double scale,
                               cudaStream_t st);
// FLUX: R (= or -=) L(flux_axis(W)) / h.  first != 0 stores, else subtracts.
// lines: lines per block (tile width; 0 = default for the precision).
template <typename T>
cudaError_t launch_line_flux(const LineOpDev &op, int axis, const BoxDev &bx, const T *W, T *R,
                             int first, cudaStream_t st, int lines = 0);
// Compact viscous terms.  VGRAD: G[q] = L(prim_q(W)) / h for q = u, v, w, T
// (4 fields at G, np apart).  VDIV: R[1 + c] += L(F[c]) / h for the 4 fields
// of F (R: the base of the 5 right-hand-side fields).
template <typename T>
cudaError_t launch_line_vgrad(const LineOpDev &op, int axis, const BoxDev &bx, const T *W, T *G, cudaStream_t st);
template <typename T>
cudaError_t launch_line_vdiv(const LineOpDev &op, int axis, const BoxDev &bx, const T *F, T *R, cudaStream_t st);
// Plane diagnostics (plane_kernels.cu): what 0 disturbance pressure, 1 the
// nine vorticity-transport terms.
cudaError_t launch_plane_fields(const BoxDev &bx, const double *Q, int axis, int index, int what, double *out,
                                cudaStream_t st);
// FILTER (FP32, mixed form): out = L(in) on 5 deviation fields (no base).
cudaError_t launch_line_filter32(const LineOpDev &op, int axis, const BoxDev &bx, const float *in, float *out,
                                 cudaStream_t st);
// Mixed-form filter update: Q += (Fd - Dn) per field in FP64 (Fd: the filtered
// FP32 deviation, Dn: the deviation it was filtered from), then W0 and Dn of
// the new state.
cudaError_t launch_filter_update(const BoxDev &bx, double *Q, const float *Fd, float *W, float *Dn, cudaStream_t st);
// FILTER (FP64): Qout = L(Q - base) + base, 5 fields.
cudaError_t launch_line_filter(const LineOpDev &op, int axis, const BoxDev &bx, int base_subtract,
                               const double *Qin, double *Qout, cudaStream_t st);

// ---- launchers (visc_kernel.cu) --------------------------------------------
cudaError_t init_visc_kernels();
// Registers of one RK stage.
//   FP64 form: acc accumulates Q_n + dt sum b_s k_s, Qout receives the next
//     stage state (stage 4: the new Q_n).
//   Mixed form: Kacc accumulates k1 + 2 k2 + 2 k3 (FP32), Dn holds the FP32
//     deviation of Q_n from the hydrostatic base, Wn receives the primitives of
//     the next stage state; stage 4 adds dt/6 (K + k4) to Q_n in FP64 and
//     refreshes Dn.
// stage 0: the right-hand side is written to Rout and nothing else.
template <typename T>
struct StageRegs {
    double *Qn = nullptr, *acc = nullptr, *Qout = nullptr;
    float *Kacc = nullptr, *Dn = nullptr;
    T *Wn = nullptr;
    T *Rout = nullptr;
};
template <typename T>
cudaError_t launch_visc_update(const BoxDev &bx, const T *W, const T *R, int stage, const StageRegs<T> &g,
                               cudaStream_t st);
// Compact viscous terms: G holds 12 fields, field 4 d + q the derivative along
// d of primitive q (u, v, w, T); each node's gradients are replaced in place
// by its viscous fluxes, field 4 d + c component c (x-, y-, z-momentum,
// energy) of the flux along d.
template <typename T>
cudaError_t launch_visc_flux(const BoxDev &bx, const T *W, T *G, cudaStream_t st);
// Gravity source, no-slip walls and the RK stage of launch_visc_update,
// without its viscous terms (R already holds them).
template <typename T>
cudaError_t launch_source_update(const BoxDev &bx, const T *W, const T *R, int stage, const StageRegs<T> &g,
                                 cudaStream_t st);

// ---- launchers (rk_kernels.cu) ---------------------------------------------
// W from the FP64 state; Dn (mixed form, optional): deviation from the base.
template <typename T>
cudaError_t launch_prep(const BoxDev &bx, const double *Q, T *W, float *Dn, cudaStream_t st);
// Wall conditions.  Q != nullptr: on the FP64 state (refreshing Dn and Wf at
// the wall nodes when given); Q == nullptr: on the FP32 stage primitives Ww.
cudaError_t launch_wall_bc(const BoxDev &bx, double *Q, float *Dn, float *Wf, float *Ww, cudaStream_t st);
cudaError_t launch_initial_state(const BoxDev &bx, unsigned long long seed, double amp, double *Q,
                                 cudaStream_t st);
// partial: nblk * 10 doubles scratch; out: 10 doubles (device)
cudaError_t launch_diagnostics(const BoxDev &bx, const double *Q, double *partial, int nblk,
                               double *out, cudaStream_t st);
int diag_blocks(long long np);

// ---- device memory ------------------------------------------------------------
// Every device allocation of the library goes through these two calls.  While
// an entry point of a context runs, they count its bytes against the process
// limit set with nopcs_set_memory_limit; an allocation beyond it fails with
// cudaErrorMemoryAllocation, which the entry points report as NOPCS_ENOMEM.
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);

// ---- one persistent launch per RK step (batch_kernel.cu) -------------------------
// One mixed-form box as the batched kernel sees it: its constants, FP32
// derivative operators, flux-sweep tile widths (0: default) and registers.
struct BatchBoxIn {
    BoxDev bx;
    LineOpDev op[3];
    int lines[3];
    float *W[2], *R, *K, *Dn;
    double *Qn;
};
struct BatchPlan;  // device work list and launch geometry
cudaError_t batch_plan_build(const std::vector<BatchBoxIn> &boxes, BatchPlan **plan, std::string &msg);
// one RK step of every box; err: the context's error word (2 when a bounded
// wait gave up); withhold: test mode, box 0's first dependency never completes
cudaError_t batch_launch(BatchPlan *plan, int *err, double wait_s, int withhold, cudaStream_t st);
void batch_plan_free(BatchPlan *plan);
int batch_plan_items(const BatchPlan *plan);

// ---- context access for entry points outside api.cu ------------------------
// Validates a derivative request on box `box` (the context's device current,
// the box index, axis 0..2, dtype 0 f64 / 1 f32) and gives the box's point
// count.  Returns NOPCS_OK or sets the context's error message.
nopcs_status ctx_derivative_check(nopcs_ctx *ctx, int box, int axis, int dtype, long long *np);
// One NOHAP first derivative along `axis` of a field of box `box`, dst =
// (1/h) L src, in the form nopcs_derivative uses for that box and axis (FP32:
// Thomas, banded or a tensor-core form as chosen at nopcs_init; FP64: Thomas).
// Arguments as validated by ctx_derivative_check.
cudaError_t ctx_first_derivative(nopcs_ctx *ctx, int box, int axis, int dtype, const void *src, void *dst,
                                 cudaStream_t st);
nopcs_status ctx_error(nopcs_ctx *ctx, nopcs_status s, const char *msg);
// Looks up, on the current device, the device address of the static scratch
// array of nopcs_derivative2_noalloc (which loads the array's module there).
cudaError_t noalloc_prepare();

}  // namespace nopcs
