// C ABI of libnopcs (declared in include/nopcs.h): context, state registers,
// the RK4 stage sequence and its CUDA-graph replay, per-kernel event timing.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "nopcs_internal.cuh"

using namespace nopcs;

namespace {

const char *const KERNEL_NAMES[NOPCS_NUM_KERNELS] = {
    "prep",   "sweep_x",     "sweep_y",   "sweep_z",   "visc_rk_update", "wall_bc",
    "filter", "diagnostics", "visc_grad", "visc_flux", "visc_div",       "source_rk_update"};
// K_VGRAD, K_VFLUX, K_VDIV, K_SRC: the compact viscous terms (visc_compact)
enum { K_PREP = 0, K_SX, K_SY, K_SZ, K_VISC, K_BC, K_FILTER, K_DIAG, K_VGRAD, K_VFLUX, K_VDIV, K_SRC };

thread_local std::string g_init_error;

// ---- device memory accounting -------------------------------------------------
// nopcs_set_memory_limit caps the device bytes one context may hold (0: no
// cap).  Each context keeps a ledger of its allocations; while one of its
// entry points runs, t_ledger points to it and dev_alloc / dev_free book
// there.  Allocations outside an entry point (none today) are not counted.
std::atomic<unsigned long long> g_mem_limit{0};

struct Ledger {
    unsigned long long limit = 0, used = 0;
    std::unordered_map<void *, size_t> sizes;
};
thread_local Ledger *t_ledger = nullptr;

// books the context's ledger for the duration of an entry point
struct LedgerScope {
    Ledger *prev;
    explicit LedgerScope(Ledger *l) : prev(t_ledger) { t_ledger = l; }
    ~LedgerScope() { t_ledger = prev; }
};

// Device registers of a box.
//   FP64 form: Q = Qn, Qs, acc (15 FP64 fields); W (6 FP64); R (5 FP64).
//   Mixed form: Q = Qn (5 FP64 fields); W = slab of two FP32 primitive sets
//     W0, W1 (12 fields); R = slab of R, K, Dn (15 FP32 fields).  Between
//     steps W0 and Dn hold the primitives and the base deviation of Qn, and
//     the filter borrows both slabs as FP64 temporaries.
//   Compact viscous terms (visc_compact): Gv, 12 fields of the stage's
//     precision holding the gradients of u, v, w, T, then the viscous fluxes.
struct BoxRes {
    nopcs_box_desc d{};
    BoxDev dev{};
    LineOpBuf dop64[3], dop32[3], fop[3];
    LineOpBuf fop32[3];  // mixed form: the filter with FP32 end-row tables
    LineOpBuf d2op64[3], d2op32[3];  // compact second derivative (nopcs_derivative order 3)
    GemmOpBuf gop[3];  // dense blocks of the FP32 derivative (tensor-core form)
    int sub_n[3] = {0, 0, 0};     // sub-domain length in use per axis (tuned if asked)
    int lines[3] = {0, 0, 0};     // flux-sweep lines per block per axis (0: default)
    bool deriv_gemm[3] = {false, false, false};  // FP32 derivative on the tensor cores
    bool gemm_bf16[3] = {false, false, false};   // ... in the BF16x3 split (else 3xTF32)
    bool deriv_band[3] = {false, false, false};  // FP32 derivative in the banded explicit form
    BandBuf bop[3];                              // banded FP32 tables (forms BANDED and AUTO)
    bool mixed = false;
    double *Q = nullptr;
    void *W = nullptr, *R = nullptr;
    void *Gv = nullptr;
    void *base = nullptr;
    double *partial = nullptr, *diag_out = nullptr;
    void *scratch = nullptr;  // order-2 derivative intermediate (lazy)
    double *stage = nullptr;  // nopcs_stage_state: staged state, 5 np doubles (lazy)
    cudaEvent_t staged_ev = nullptr;     // the staging copy is done
    cudaEvent_t committed_ev = nullptr;  // the last commit has read the staged state
    bool staged = false;
    int nblk_diag = 0;
    long long step = 0;
    double *Qn() const { return Q; }
    double *Qs() const { return Q + 5 * dev.np; }
    double *acc() const { return Q + 10 * dev.np; }
    float *Wm(int k) const { return (float *)W + (size_t)k * 6 * dev.np; }
    float *Rm() const { return (float *)R; }
    float *Km() const { return (float *)R + 5 * dev.np; }
    float *Dn() const { return (float *)R + 10 * dev.np; }
};

struct ProfPair {
    cudaEvent_t a, b;
    int kind;
};

}  // namespace

struct nopcs_ctx {
    int device = 0;
    Ledger ledger;
    nopcs_precision prec = NOPCS_FP64;
    nopcs_form form = NOPCS_FORM_THOMAS;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<BoxRes> boxes;
    std::string err;
    cudaGraphExec_t step_exec = nullptr;
    std::vector<cudaStream_t> branch;  // one capture branch per box
    std::vector<cudaEvent_t> branch_ev;
    int *dev_err = nullptr;  // set by kernels whose bounded waits gave up
    bool profiling = false;
    std::vector<ProfPair> pool;
    size_t pool_used = 0;
    double prof_ms[NOPCS_NUM_KERNELS] = {};
    long long prof_n[NOPCS_NUM_KERNELS] = {};
    int launch_mode = NOPCS_LAUNCH_GRAPH;  // nopcs_set_launch
    double wait_s = 2.0;                   // bound of the batched kernel's waits
    BatchPlan *plan = nullptr;             // persistent launch: work list
    cudaStream_t copy_stream = nullptr;    // nopcs_stage_state's copies (lazy)
    // large host-to-device copies are split over NSPLIT streams (the stream
    // that orders the copy and NSPLIT - 1 helpers): a single copy ran at 60 to
    // 210 GB/s depending on the box, split copies at the link's 210 GB/s
    cudaStream_t split_helper[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    cudaEvent_t split_ev[2][4] = {{nullptr, nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr, nullptr}};
};

namespace {

nopcs_status fail(nopcs_ctx *c, nopcs_status s, const std::string &m)
{
    if (c)
        c->err = m;
    else
        g_init_error = m;
    return s;
}

// an allocation that failed (the device is full, or the context's memory
// limit is reached) is NOPCS_ENOMEM; every other CUDA error NOPCS_ECUDA
nopcs_status cuda_fail(nopcs_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, e == cudaErrorMemoryAllocation ? NOPCS_ENOMEM : NOPCS_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

bool valid_box(const nopcs_box_desc &d, std::string &m)
{
    for (int a = 0; a < 3; ++a) {
        if (d.n[a] < 5) {
            m = "each axis needs at least 5 points";
            return false;
        }
        if (!(d.len[a] > 0.0)) {
            m = "box lengths must be positive";
            return false;
        }
        if (d.sub_n[a] < -1 || (d.sub_n[a] > 0 && d.sub_n[a] < 3)) {
            m = "sub_n must be -1 (tune), 0 or >= 3";
            return false;
        }
    }
    if ((long long)d.n[0] * d.n[1] * d.n[2] >= (1LL << 31)) {
        m = "a box holds fewer than 2^31 points (kernels index a field with 32 bits)";
        return false;
    }
    if (d.gravity_axis < 0 || d.gravity_axis > 2) {
        m = "gravity_axis must be 0, 1 or 2";
        return false;
    }
    if (!(d.Re > 0 && d.M > 0 && d.Pr > 0 && d.gamma > 1.0 && d.dt > 0 && d.Ts_kelvin > 0 && d.mu_s_si > 0 &&
          d.T_upper > 0 && d.T_lower > 0 && d.suth_S >= 0)) {
        m = "physical parameters out of range";
        return false;
    }
    if (d.filter_every < 0 || !(d.filter_alpha > -0.5 && d.filter_alpha < 0.5)) {
        m = "filter_every must be >= 0 and |filter_alpha| < 0.5";
        return false;
    }
    if (d.visc_compact != 0 && d.visc_compact != 1) {
        m = "visc_compact must be 0 or 1";
        return false;
    }
    return true;
}

// Hydrostatic base (Sec. 2): dp/dz = -rho g, rho = gamma M^2 p / T, constant T
// in each half, p = 1 / (gamma M^2) at the mid-plane.
void hydrostatic(const nopcs_box_desc &d, std::vector<double> &rho, std::vector<double> &p)
{
    const int ga = d.gravity_axis, N = d.n[ga];
    const double h = d.len[ga] / (N - 1), zI = 0.5 * d.len[ga];
    const double gm2 = d.gamma * d.M * d.M;
    rho.resize(N);
    p.resize(N);
    for (int k = 0; k < N; ++k) {
        const double z = k * h;
        const double T = z < zI ? d.T_lower : d.T_upper;
        p[k] = exp(-gm2 * d.g * (z - zI) / T) / gm2;
        rho[k] = gm2 * p[k] / T;
    }
}

size_t esize(const nopcs_ctx *c) { return c->prec == NOPCS_MIXED ? 4 : 8; }

void free_box(BoxRes &b)
{
    for (int a = 0; a < 3; ++a) {
        b.dop64[a].release();
        b.dop32[a].release();
        b.fop[a].release();
        b.fop32[a].release();
        b.d2op64[a].release();
        b.d2op32[a].release();
        b.gop[a].release();
        b.bop[a].release();
    }
    if (b.Q) dev_free(b.Q);
    if (b.W) dev_free(b.W);
    if (b.R) dev_free(b.R);
    if (b.Gv) dev_free(b.Gv);
    if (b.base) dev_free(b.base);
    if (b.partial) dev_free(b.partial);
    if (b.scratch) dev_free(b.scratch);
    if (b.stage) dev_free(b.stage);
    if (b.staged_ev) cudaEventDestroy(b.staged_ev);
    if (b.committed_ev) cudaEventDestroy(b.committed_ev);
    b.stage = nullptr;
    b.staged_ev = b.committed_ev = nullptr;
    b.staged = false;
    b.Q = nullptr;
    b.W = b.R = b.Gv = b.base = b.scratch = nullptr;
    b.partial = b.diag_out = nullptr;
}

// operator tables of one axis for the box's current sub-domain length
nopcs_status build_axis_ops(nopcs_ctx *ctx, BoxRes &b, int a)
{
    const nopcs_box_desc &d = b.d;
    std::string msg;
    const int sn = b.sub_n[a];
    if (!build_line_op(d.n[a], sn, KIND_DERIV, 0.0, 1e-16, b.dop64[a].host, msg) ||
        !build_line_op(d.n[a], sn, KIND_DERIV, 0.0, 1e-8, b.dop32[a].host, msg) ||
        !build_line_op(d.n[a], sn, KIND_FILTER, d.filter_alpha, 1e-16, b.fop[a].host, msg))
        return fail(ctx, NOPCS_EINVAL, msg);
    CK(b.dop64[a].upload(), "operator upload");
    CK(b.dop32[a].upload(), "operator upload");
    CK(b.fop[a].upload(), "operator upload");
    if (!build_line_op(d.n[a], sn, KIND_D2, 0.0, 1e-16, b.d2op64[a].host, msg) ||
        !build_line_op(d.n[a], sn, KIND_D2, 0.0, 1e-8, b.d2op32[a].host, msg))
        return fail(ctx, NOPCS_EINVAL, msg);
    CK(b.d2op64[a].upload(), "operator upload");
    CK(b.d2op32[a].upload(), "operator upload");
    if (b.mixed) {
        if (!build_line_op(d.n[a], sn, KIND_FILTER, d.filter_alpha, 1e-8, b.fop32[a].host, msg))
            return fail(ctx, NOPCS_EINVAL, msg);
        CK(b.fop32[a].upload(), "operator upload");
    }
    if (ctx->form == NOPCS_FORM_BANDED || ctx->form == NOPCS_FORM_AUTO) {
        b.bop[a].release();
        if (!build_band_op(d.n[a], KIND_DERIV, 0.0, 1e-8, b.bop[a].host, msg)) return fail(ctx, NOPCS_EINVAL, msg);
        if (band_supported(b.bop[a].host)) {
            CK(b.bop[a].upload(), "banded operator upload");
        } else if (ctx->form == NOPCS_FORM_BANDED) {
            return fail(ctx, NOPCS_EUNSUPPORTED, "the banded form's tables do not fit its kernel for this line length");
        }
    }
    const bool gemm_form = ctx->form == NOPCS_FORM_GEMM_3XTF32 || ctx->form == NOPCS_FORM_GEMM_BF16X3;
    if (gemm_form || ctx->form == NOPCS_FORM_AUTO) {
        build_dense_blocks(b.dop32[a].host, b.gop[a].host);
        if (gemm_smem_fits(b.gop[a].host)) {
            CK(b.gop[a].upload(), "dense operator upload");
        } else {
            b.gop[a].release();
            if (gemm_form)
                return fail(ctx, NOPCS_EUNSUPPORTED, "the tensor-core forms need sub-domains of at most 240 points");
        }
    }
    return NOPCS_OK;
}

// mixed form: primitives W0 and base deviation Dn of the FP64 state Qn
cudaError_t refresh_mixed(BoxRes &b, cudaStream_t st)
{
    if (!b.mixed) return cudaSuccess;
    return launch_prep<float>(b.dev, b.Qn(), b.Wm(0), b.Dn(), st);
}

// ---- autotuner ---------------------------------------------------------------
// Per axis, the flux sweep's tile width (16 or 32 lines per block) and, where
// the descriptor asks with sub_n = -1, the sub-domain length (32, 64 or 128)
// are chosen by timing the sweep the RK path uses (the context precision) on
// this GPU; under NOPCS_FORM_AUTO each axis's FP32 derivative takes the Thomas
// or the tensor-core form, whichever measured faster.  Times come from CUDA
// events on the context stream (one warm-up, three timed launches); choices
// are cached per box shape for the process.  Boxes below 2^20 points keep the
// defaults unless a sub-domain length is requested.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;

float time_launches(cudaStream_t st, const std::function<cudaError_t()> &fn, cudaError_t &err)
{
    cudaEvent_t e0, e1;
    err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err != cudaSuccess) return 1e30f;
    err = fn();
    if (err == cudaSuccess) err = cudaEventRecord(e0, st);
    for (int i = 0; i < 3 && err == cudaSuccess; ++i) err = fn();
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 1e30f;
    if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

nopcs_status autotune_box(nopcs_ctx *ctx, BoxRes &b)
{
    cudaStream_t st = ctx->stream;
    const BoxDev &x = b.dev;
    char key0[96];
    snprintf(key0, sizeof(key0), "%d,%d,%d,%d", x.n[0], x.n[1], x.n[2], b.mixed ? 1 : 0);
    // primitives of the current state feed the timed sweeps
    if (!b.mixed) CK(launch_prep<double>(x, b.Qn(), (double *)b.W, nullptr, st), "autotune");
    for (int a = 0; a < 3; ++a) {
        const bool tune_sub = b.d.sub_n[a] == -1;
        if (!tune_sub && x.np < (1LL << 20)) continue;
        const std::string key = std::string(key0) + ",s" + std::to_string(a) + "," + std::to_string(b.d.sub_n[a]);
        int best = -1;  // sub_n * 1000 + lines per block
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) best = it->second;
        }
        if (best < 0) {
            float tbest = 1e30f;
            std::vector<int> cands;
            if (tune_sub)
                cands = {32, 64, 128};
            else
                cands = {b.sub_n[a]};
            for (int cand : cands) {
                if (tune_sub && cand >= x.n[a] && cand != 32) continue;
                if (tune_sub) {
                    b.sub_n[a] = cand;
                    nopcs_status s2 = build_axis_ops(ctx, b, a);
                    if (s2 != NOPCS_OK) return s2;
                }
                for (int ln : {16, 32}) {
                    cudaError_t e;
                    float ms = b.mixed ? time_launches(st, [&] { return launch_line_flux<float>(b.dop32[a].dev, a, x, b.Wm(0), b.Rm(), 1, st, ln); }, e)
                                       : time_launches(st, [&] { return launch_line_flux<double>(b.dop64[a].dev, a, x, (double *)b.W, (double *)b.R, 1, st, ln); }, e);
                    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
                    if (ms < tbest) {
                        tbest = ms;
                        best = cand * 1000 + ln;
                    }
                }
            }
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[key] = best;
        }
        b.lines[a] = best % 1000;
        if (!tune_sub) continue;
        best /= 1000;
        b.sub_n[a] = best;
        nopcs_status s2 = build_axis_ops(ctx, b, a);
        if (s2 != NOPCS_OK) return s2;
    }
    if (ctx->form == NOPCS_FORM_AUTO) {
        // scratch FP32 fields inside the right-hand-side buffer (>= 2 np floats)
        float *fin = (float *)b.R, *fout = fin + x.np;
        CK(cudaMemsetAsync(fin, 0, 2 * (size_t)x.np * sizeof(float), st), "autotune");
        for (int a = 0; a < 3; ++a) {
            b.deriv_gemm[a] = false;
            b.gemm_bf16[a] = false;
            b.deriv_band[a] = false;
            if (!b.gop[a].mem && !b.bop[a].mem) continue;
            const std::string key = std::string(key0) + ",g" + std::to_string(a) + "," + std::to_string(b.sub_n[a]);
            int choice = -1;
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto it = g_tune_cache.find(key);
                if (it != g_tune_cache.end()) choice = it->second;
            }
            if (choice < 0) {
                // 0 Thomas, 1 3xTF32, 2 banded, 3 BF16x3: the fastest
                cudaError_t e[4] = {cudaSuccess, cudaSuccess, cudaSuccess, cudaSuccess};
                float t[4];
                t[0] = time_launches(st, [&] { return launch_line_field<float>(b.dop32[a].dev, a, x.n, fin, fout, 1.0, st); }, e[0]);
                t[1] = b.gop[a].mem ? time_launches(st, [&] { return launch_gemm_field(b.gop[a].dev, false, a, x.n, fin, fout, 1.0, ctx->dev_err, st); }, e[1]) : 1e30f;
                t[2] = b.bop[a].mem ? time_launches(st, [&] { return launch_band_field(b.bop[a], a, x.n, fin, fout, 1.0, st); }, e[2]) : 1e30f;
                t[3] = b.gop[a].mem ? time_launches(st, [&] { return launch_gemm_field(b.gop[a].dev, true, a, x.n, fin, fout, 1.0, ctx->dev_err, st); }, e[3]) : 1e30f;
                for (cudaError_t ei : e)
                    if (ei != cudaSuccess) return cuda_fail(ctx, ei, "autotune");
                choice = 0;
                for (int k = 1; k < 4; ++k)
                    if (t[k] < t[choice]) choice = k;
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune_cache[key] = choice;
            }
            b.deriv_gemm[a] = choice == 1 || choice == 3;
            b.gemm_bf16[a] = choice == 3;
            b.deriv_band[a] = choice == 2;
        }
    }
    return NOPCS_OK;
}

nopcs_status setup_box(nopcs_ctx *ctx, BoxRes &b)
{
    const nopcs_box_desc &d = b.d;
    BoxDev &x = b.dev;
    for (int a = 0; a < 3; ++a) {
        x.n[a] = d.n[a];
        x.h[a] = d.len[a] / (d.n[a] - 1);
        x.inv_h[a] = 1.0 / x.h[a];
    }
    x.np = (long long)d.n[0] * d.n[1] * d.n[2];
    x.ga = d.gravity_axis;
    x.gamma = d.gamma;
    x.gm2 = d.gamma * d.M * d.M;
    x.Re = d.Re;
    x.M = d.M;
    x.kq = 1.0 / ((d.gamma - 1.0) * d.Pr * d.Re * d.M * d.M);
    x.suth_S = d.suth_S;
    // Eq. reg over mu_s: mu_b / mu_s = mub_scale 1e-4 (3.381 T T_s - 7.383) / mu_s
    x.mub_coef0 = d.mub_scale * 1.0e-4 * 3.381 * d.Ts_kelvin / d.mu_s_si;
    x.mub_coef1 = -d.mub_scale * 1.0e-4 * 7.383 / d.mu_s_si;
    x.g = d.g;
    x.cE = 1.0 / (d.gamma * (d.gamma - 1.0) * d.M * d.M);
    x.dt = d.dt;
    b.mixed = ctx->prec == NOPCS_MIXED;

    for (int a = 0; a < 3; ++a) {
        b.sub_n[a] = d.sub_n[a] == -1 ? 64 : d.sub_n[a];
        b.deriv_gemm[a] = ctx->form == NOPCS_FORM_GEMM_3XTF32 || ctx->form == NOPCS_FORM_GEMM_BF16X3;
        b.gemm_bf16[a] = ctx->form == NOPCS_FORM_GEMM_BF16X3;
        b.deriv_band[a] = ctx->form == NOPCS_FORM_BANDED;
        nopcs_status st = build_axis_ops(ctx, b, a);
        if (st != NOPCS_OK) return st;
    }
    // base tables
    std::vector<double> rh, ph;
    hydrostatic(d, rh, ph);
    const int Ng = d.n[d.gravity_axis];
    const bool bs = d.base_subtract != 0;
    // layout: rho_h, p_h, rho_b, p_b, E_b, H_b (double) then
    //         rho_b, p_b, H_b, T_b, 1/p_b, 1/rho_b (float)
    std::vector<double> t64(6 * (size_t)Ng, 0.0);
    std::vector<float> t32(6 * (size_t)Ng, 0.0f);
    for (int k = 0; k < Ng; ++k) {
        t64[k] = rh[k];
        t64[Ng + k] = ph[k];
        if (bs) {
            const double Eb = ph[k] / (d.gamma - 1.0);
            t64[2 * Ng + k] = rh[k];
            t64[3 * Ng + k] = ph[k];
            t64[4 * Ng + k] = Eb;
            t64[5 * Ng + k] = Eb + ph[k];
            t32[k] = (float)rh[k];
            t32[Ng + k] = (float)ph[k];
            t32[2 * Ng + k] = (float)(Eb + ph[k]);
            const double zk = k * (d.len[d.gravity_axis] / (Ng - 1));
            t32[3 * Ng + k] = (float)(zk < 0.5 * d.len[d.gravity_axis] ? d.T_lower : d.T_upper);
            t32[4 * Ng + k] = (float)(1.0 / ph[k]);
            t32[5 * Ng + k] = (float)(1.0 / rh[k]);
        }
    }
    const size_t b64 = t64.size() * 8, b32 = t32.size() * 4;
    CK(dev_alloc(&b.base, b64 + b32 + 256), "base tables");
    CK(cudaMemcpy(b.base, t64.data(), b64, cudaMemcpyHostToDevice), "base tables");
    CK(cudaMemcpy((char *)b.base + b64, t32.data(), b32, cudaMemcpyHostToDevice), "base tables");
    const double *p64 = (const double *)b.base;
    const float *p32 = (const float *)((const char *)b.base + b64);
    x.rho_h64 = p64;
    x.p_h64 = p64 + Ng;
    x.rho_b64 = p64 + 2 * Ng;
    x.p_b64 = p64 + 3 * Ng;
    x.E_b64 = p64 + 4 * Ng;
    x.H_b64 = p64 + 5 * Ng;
    x.rho_b32 = p32;
    x.p_b32 = p32 + Ng;
    x.H_b32 = p32 + 2 * Ng;
    x.T_b32 = p32 + 3 * Ng;
    x.ip_b32 = p32 + 4 * Ng;
    x.ir_b32 = p32 + 5 * Ng;
    x.err = ctx->dev_err;

    // state registers and scratch
    const size_t np = (size_t)x.np;
    cudaError_t e = dev_alloc((void **)&b.Q, (b.mixed ? 5 : 15) * np * sizeof(double));
    if (e != cudaSuccess) {
        b.Q = nullptr;
        return fail(ctx, e == cudaErrorMemoryAllocation ? NOPCS_ENOMEM : NOPCS_ECUDA, "state registers");
    }
    e = dev_alloc(&b.W, (b.mixed ? 12 : 6) * np * esize(ctx));
    if (e != cudaSuccess) {
        b.W = nullptr;
        return fail(ctx, e == cudaErrorMemoryAllocation ? NOPCS_ENOMEM : NOPCS_ECUDA, "primitive buffer");
    }
    e = dev_alloc(&b.R, (b.mixed ? 15 : 5) * np * esize(ctx));
    if (e != cudaSuccess) {
        b.R = nullptr;
        return fail(ctx, e == cudaErrorMemoryAllocation ? NOPCS_ENOMEM : NOPCS_ECUDA, "right-hand-side buffer");
    }
    if (d.visc_compact) {
        e = dev_alloc(&b.Gv, 12 * np * esize(ctx));
        if (e != cudaSuccess) {
            b.Gv = nullptr;
            return fail(ctx, e == cudaErrorMemoryAllocation ? NOPCS_ENOMEM : NOPCS_ECUDA,
                        "compact viscous-term buffer");
        }
    }
    b.nblk_diag = diag_blocks(x.np);
    CK(dev_alloc((void **)&b.partial, ((size_t)b.nblk_diag * 10 + 16) * sizeof(double)), "diagnostics scratch");
    b.diag_out = b.partial + (size_t)b.nblk_diag * 10;
    CK(launch_initial_state(x, d.seed, d.perturb_amp, b.Qn(), ctx->stream), "initial state");
    CK(refresh_mixed(b, ctx->stream), "initial state");
    if (d.sub_n[0] == -1 || d.sub_n[1] == -1 || d.sub_n[2] == -1 || ctx->form == NOPCS_FORM_AUTO ||
        x.np >= (1LL << 20)) {
        nopcs_status st = autotune_box(ctx, b);
        if (st != NOPCS_OK) return st;
        CK(refresh_mixed(b, ctx->stream), "initial state");
    }
    b.step = 0;
    return NOPCS_OK;
}

// ---- profiling --------------------------------------------------------------
void harvest(nopcs_ctx *c)
{
    for (size_t i = 0; i < c->pool_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->pool[i].a, c->pool[i].b) == cudaSuccess) {
            c->prof_ms[c->pool[i].kind] += ms;
            c->prof_n[c->pool[i].kind] += 1;
        }
    }
    c->pool_used = 0;
}

struct Timed {
    nopcs_ctx *c;
    cudaStream_t st;
    int kind;
    ProfPair *pp = nullptr;
    Timed(nopcs_ctx *c_, cudaStream_t s, int k) : c(c_), st(s), kind(k)
    {
        if (!c->profiling) return;
        if (c->pool_used == c->pool.size()) {
            cudaStreamSynchronize(st);
            harvest(c);
        }
        pp = &c->pool[c->pool_used++];
        pp->kind = kind;
        cudaEventRecord(pp->a, st);
    }
    ~Timed()
    {
        if (pp) cudaEventRecord(pp->b, st);
    }
};

// ---- the RK stage sequence --------------------------------------------------
// Sweeps x, y, z accumulate the convective right-hand side of W into R, then
// the fused viscous/source/RK kernel finishes the stage.
template <typename T>
cudaError_t enqueue_rhs_sweeps(nopcs_ctx *ctx, BoxRes &b, const T *W, T *R, cudaStream_t st)
{
    const bool f32 = sizeof(T) == 4;
    for (int a = 0; a < 3; ++a) {
        Timed t(ctx, st, K_SX + a);
        cudaError_t e =
            launch_line_flux<T>(f32 ? b.dop32[a].dev : b.dop64[a].dev, a, b.dev, W, R, a == 0, st, b.lines[a]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Compact viscous terms (visc_compact): the derivatives of u, v, w, T along
// every axis by the NOHAP operator (Sec. 3) into Gv, the nodal viscous fluxes
// in their place, and the NOHAP derivative of each flux along its own axis
// added into R[1..4].
template <typename T>
cudaError_t enqueue_compact_visc(nopcs_ctx *ctx, BoxRes &b, const T *W, T *R, cudaStream_t st)
{
    const bool f32 = sizeof(T) == 4;
    T *G = (T *)b.Gv;
    const size_t np = (size_t)b.dev.np;
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        Timed t(ctx, st, K_VGRAD);
        e = launch_line_vgrad<T>(f32 ? b.dop32[a].dev : b.dop64[a].dev, a, b.dev, W, G + 4 * a * np, st);
    }
    if (e != cudaSuccess) return e;
    {
        Timed t(ctx, st, K_VFLUX);
        e = launch_visc_flux<T>(b.dev, W, G, st);
    }
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        Timed t(ctx, st, K_VDIV);
        e = launch_line_vdiv<T>(f32 ? b.dop32[a].dev : b.dop64[a].dev, a, b.dev, G + 4 * a * np, R, st);
    }
    return e;
}

// The rest of a stage after the convective sweeps: the fused viscous, source
// and RK kernel, or, with compact viscous terms, those terms and then the
// source and RK kernel.
template <typename T>
cudaError_t enqueue_visc_stage(nopcs_ctx *ctx, BoxRes &b, const T *W, T *R, int stage, const StageRegs<T> &g,
                               cudaStream_t st)
{
    if (!b.d.visc_compact) {
        Timed t(ctx, st, K_VISC);
        return launch_visc_update<T>(b.dev, W, R, stage, g, st);
    }
    cudaError_t e = enqueue_compact_visc<T>(ctx, b, W, R, st);
    if (e != cudaSuccess) return e;
    Timed t(ctx, st, K_SRC);
    return launch_source_update<T>(b.dev, W, R, stage, g, st);
}

// FP64 form: stage s of classical RK4 from the FP64 stage state Qin
cudaError_t enqueue_stage_fp64(nopcs_ctx *ctx, BoxRes &b, int stage, const double *Qin, double *Rout,
                               cudaStream_t st)
{
    const BoxDev &x = b.dev;
    double *W = (double *)b.W, *R = (double *)b.R;
    cudaError_t e;
    {
        Timed t(ctx, st, K_PREP);
        e = launch_prep<double>(x, Qin, W, nullptr, st);
    }
    if (e != cudaSuccess) return e;
    if ((e = enqueue_rhs_sweeps<double>(ctx, b, W, R, st)) != cudaSuccess) return e;
    StageRegs<double> g;
    g.Qn = b.Qn();
    g.acc = b.acc();
    g.Qout = stage == 4 ? b.Qn() : b.Qs();
    g.Rout = Rout;
    e = enqueue_visc_stage<double>(ctx, b, W, R, stage, g, st);
    if (e != cudaSuccess || stage == 0) return e;
    Timed t(ctx, st, K_BC);
    return launch_wall_bc(x, g.Qout, nullptr, nullptr, nullptr, st);
}

// Mixed form: stage s reads the primitives W_in (W0 for stages 1 and 3, W1
// for 2 and 4) and writes those of the next stage state to the other set, so
// every step starts and ends on W0.
cudaError_t enqueue_stage_mixed(nopcs_ctx *ctx, BoxRes &b, int stage, cudaStream_t st)
{
    const BoxDev &x = b.dev;
    float *Win = b.Wm((stage - 1) & 1), *Wout = b.Wm(stage & 1);
    cudaError_t e = enqueue_rhs_sweeps<float>(ctx, b, Win, b.Rm(), st);
    if (e != cudaSuccess) return e;
    StageRegs<float> g;
    g.Qn = b.Qn();
    g.Kacc = b.Km();
    g.Dn = b.Dn();
    g.Wn = Wout;
    e = enqueue_visc_stage<float>(ctx, b, Win, b.Rm(), stage, g, st);
    if (e != cudaSuccess) return e;
    Timed t(ctx, st, K_BC);
    if (stage < 4) return launch_wall_bc(x, nullptr, nullptr, nullptr, Wout, st);
    return launch_wall_bc(x, b.Qn(), b.Dn(), Wout, nullptr, st);
}

// right-hand side of an FP64 state q into r (stage 0), for tests
cudaError_t enqueue_rhs_only(nopcs_ctx *ctx, BoxRes &b, const double *q, void *r, cudaStream_t st)
{
    if (!b.mixed) return enqueue_stage_fp64(ctx, b, 0, q, (double *)r, st);
    // W1 is free between steps
    float *W = b.Wm(1);
    cudaError_t e = launch_prep<float>(b.dev, q, W, nullptr, st);
    if (e != cudaSuccess) return e;
    if ((e = enqueue_rhs_sweeps<float>(ctx, b, W, b.Rm(), st)) != cudaSuccess) return e;
    StageRegs<float> g;
    g.Rout = (float *)r;
    return enqueue_visc_stage<float>(ctx, b, W, b.Rm(), 0, g, st);
}

cudaError_t enqueue_filter(nopcs_ctx *ctx, BoxRes &b, cudaStream_t st)
{
    Timed t(ctx, st, K_FILTER);
    const BoxDev &x = b.dev;
    if (b.mixed) {
        // FP32 filter of the deviation D_n (already base-subtracted), x -> y
        // -> z through the W slab, R and K, then Q_n += F(D_n) - D_n in FP64
        float *t1 = b.Wm(0), *t2 = b.Rm(), *t3 = b.Km();
        cudaError_t e = launch_line_filter32(b.fop32[0].dev, 0, x, b.Dn(), t1, st);
        if (e != cudaSuccess) return e;
        e = launch_line_filter32(b.fop32[1].dev, 1, x, t1, t2, st);
        if (e != cudaSuccess) return e;
        e = launch_line_filter32(b.fop32[2].dev, 2, x, t2, t3, st);
        if (e != cudaSuccess) return e;
        return launch_filter_update(x, b.Qn(), t3, b.Wm(0), b.Dn(), st);
    }
    const int bs = b.d.base_subtract;
    // two FP64 temporaries: acc and Qs
    double *t1 = b.acc(), *t2 = b.Qs();
    cudaError_t e = launch_line_filter(b.fop[0].dev, 0, x, bs, b.Qn(), t1, st);
    if (e != cudaSuccess) return e;
    e = launch_line_filter(b.fop[1].dev, 1, x, bs, t1, t2, st);
    if (e != cudaSuccess) return e;
    return launch_line_filter(b.fop[2].dev, 2, x, bs, t2, b.Qn(), st);
}

cudaError_t enqueue_step(nopcs_ctx *ctx, BoxRes &b, cudaStream_t st)
{
    for (int s = 1; s <= 4; ++s) {
        cudaError_t e = b.mixed ? enqueue_stage_mixed(ctx, b, s, st)
                                : enqueue_stage_fp64(ctx, b, s, s == 1 ? b.Qn() : b.Qs(), nullptr, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Every entry point that takes a context runs on the context's device: a
// caller that switched devices gets NOPCS_EINVAL, not launches on another GPU.
nopcs_status check_ctx(nopcs_ctx *ctx)
{
    if (!ctx) return NOPCS_EINVAL;
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetDevice");
    if (dev != ctx->device)
        return fail(ctx, NOPCS_EINVAL,
                    "the current CUDA device (" + std::to_string(dev) + ") is not the context's device (" +
                        std::to_string(ctx->device) + "); call cudaSetDevice first");
    return NOPCS_OK;
}

nopcs_status check_box(nopcs_ctx *ctx, int box)
{
    nopcs_status s = check_ctx(ctx);
    if (s != NOPCS_OK) return s;
    if (box < 0 || box >= (int)ctx->boxes.size()) return fail(ctx, NOPCS_EINVAL, "box index out of range");
    return NOPCS_OK;
}

// one NOHAP first derivative in the form chosen for the box and axis
cudaError_t first_derivative(nopcs_ctx *ctx, BoxRes &b, int axis, int dtype, const void *src, void *dst,
                             cudaStream_t st)
{
    const double scale = b.dev.inv_h[axis];
    if (dtype == 0)
        return launch_line_field<double>(b.dop64[axis].dev, axis, b.dev.n, (const double *)src, (double *)dst, scale,
                                         st);
    if (b.deriv_gemm[axis])
        return launch_gemm_field(b.gop[axis].dev, b.gemm_bf16[axis], axis, b.dev.n, (const float *)src, (float *)dst,
                                 scale, ctx->dev_err, st);
    if (b.deriv_band[axis])
        return launch_band_field(b.bop[axis], axis, b.dev.n, (const float *)src, (float *)dst, scale, st);
    return launch_line_field<float>(b.dop32[axis].dev, axis, b.dev.n, (const float *)src, (float *)dst, scale, st);
}

}  // namespace

namespace nopcs {

nopcs_status ctx_derivative_check(nopcs_ctx *ctx, int box, int axis, int dtype, long long *np)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    if (axis < 0 || axis > 2) return fail(ctx, NOPCS_EINVAL, "axis must be 0, 1 or 2");
    if (dtype != 0 && dtype != 1) return fail(ctx, NOPCS_EINVAL, "dtype must be 0 (f64) or 1 (f32)");
    *np = ctx->boxes[box].dev.np;
    return NOPCS_OK;
}

cudaError_t ctx_first_derivative(nopcs_ctx *ctx, int box, int axis, int dtype, const void *src, void *dst,
                                 cudaStream_t st)
{
    return first_derivative(ctx, ctx->boxes[box], axis, dtype, src, dst, st);
}

cudaError_t dev_alloc(void **p, size_t bytes)
{
    *p = nullptr;
    Ledger *l = t_ledger;
    if (l && l->limit && l->used + bytes > l->limit) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();  // an allocation failure is not sticky: clear it
        return e;
    }
    if (l) {
        l->used += bytes;
        l->sizes[*p] = bytes;
    }
    return cudaSuccess;
}

void dev_free(void *p)
{
    if (!p) return;
    Ledger *l = t_ledger;
    if (l) {
        auto it = l->sizes.find(p);
        if (it != l->sizes.end()) {
            l->used -= it->second;
            l->sizes.erase(it);
        }
    }
    cudaFree(p);
}

nopcs_status ctx_error(nopcs_ctx *ctx, nopcs_status s, const char *msg) { return fail(ctx, s, msg); }

}  // namespace nopcs

// ============================================================================
extern "C" {

nopcs_status nopcs_init(const nopcs_box_desc *boxes, int nboxes, nopcs_precision prec, nopcs_form form,
                        void *stream, nopcs_ctx **out)
{
    if (!out) return fail(nullptr, NOPCS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!boxes || nboxes < 1) return fail(nullptr, NOPCS_EINVAL, "need at least one box");
    if (prec != NOPCS_FP64 && prec != NOPCS_MIXED) return fail(nullptr, NOPCS_EINVAL, "bad precision");
    if (form < NOPCS_FORM_AUTO || form > NOPCS_FORM_BANDED) return fail(nullptr, NOPCS_EINVAL, "bad form");
    for (int i = 0; i < nboxes; ++i) {
        std::string m;
        if (!valid_box(boxes[i], m)) return fail(nullptr, NOPCS_EINVAL, "box " + std::to_string(i) + ": " + m);
    }
    nopcs_ctx *ctx = new nopcs_ctx();
    ctx->prec = prec;
    ctx->form = form;
    ctx->stream = (cudaStream_t)stream;
    ctx->ledger.limit = g_mem_limit.load();
    LedgerScope scope(&ctx->ledger);
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = init_line_kernels();
    if (e == cudaSuccess) e = init_visc_kernels();
    if (e == cudaSuccess && (ctx->form == NOPCS_FORM_GEMM_3XTF32 || ctx->form == NOPCS_FORM_GEMM_BF16X3 ||
                             ctx->form == NOPCS_FORM_AUTO))
        e = init_gemm_kernels();
    // the static scratch of nopcs_derivative2_noalloc becomes resident on this
    // device now, so that no later call loads its module
    if (e == cudaSuccess) e = noalloc_prepare();
    if (e == cudaSuccess) e = dev_alloc((void **)&ctx->dev_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->dev_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        g_init_error = std::string("CUDA: ") + cudaGetErrorString(e);
        nopcs_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? NOPCS_ENOMEM : NOPCS_ECUDA;
    }
    ctx->boxes.resize(nboxes);
    for (int i = 0; i < nboxes; ++i) {
        ctx->boxes[i].d = boxes[i];
        if (prec == NOPCS_MIXED) ctx->boxes[i].d.base_subtract = 1;
        nopcs_status s = setup_box(ctx, ctx->boxes[i]);
        if (s != NOPCS_OK) {
            g_init_error = ctx->err;
            nopcs_destroy(ctx);
            return s;
        }
    }
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        g_init_error = std::string("initial state: ") + cudaGetErrorString(e);
        nopcs_destroy(ctx);
        return NOPCS_ECUDA;
    }
    *out = ctx;
    return NOPCS_OK;
}

void nopcs_destroy(nopcs_ctx *ctx)
{
    if (!ctx) return;
    // free on the context's device, whatever device the caller has current
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) cur = -1;
    if (cur != ctx->device) cudaSetDevice(ctx->device);
    LedgerScope scope(&ctx->ledger);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    for (auto &g : ctx->split_helper)
        for (auto h : g)
            if (h) cudaStreamSynchronize(h);
    if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
    for (auto st : ctx->branch) cudaStreamDestroy(st);
    for (auto ev : ctx->branch_ev) cudaEventDestroy(ev);
    for (auto &p : ctx->pool) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    batch_plan_free(ctx->plan);
    for (auto &b : ctx->boxes) free_box(b);
    if (ctx->dev_err) dev_free(ctx->dev_err);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    for (int g = 0; g < 2; ++g) {
        for (auto &h : ctx->split_helper[g])
            if (h) {
                cudaStreamSynchronize(h);
                cudaStreamDestroy(h);
            }
        for (auto &e : ctx->split_ev[g])
            if (e) cudaEventDestroy(e);
    }
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    const int dev = ctx->device;
    delete ctx;
    if (cur >= 0 && cur != dev) cudaSetDevice(cur);
}

const char *nopcs_last_error(const nopcs_ctx *ctx)
{
    if (!ctx) return g_init_error.c_str();
    return ctx->err.c_str();
}

namespace {

// A copy of `bytes` from src to dst ordered on stream st (work enqueued on st
// before it runs first, work enqueued after it waits for all of it), split in
// four parts run side by side on st and three helper streams of group g.
cudaError_t split_copy(nopcs_ctx *ctx, int g, void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    constexpr int NSPLIT = 4;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < NSPLIT - 1 && e == cudaSuccess; ++i)
        if (!ctx->split_helper[g][i]) e = cudaStreamCreateWithFlags(&ctx->split_helper[g][i], cudaStreamNonBlocking);
    for (int i = 0; i < NSPLIT && e == cudaSuccess; ++i)
        if (!ctx->split_ev[g][i]) e = cudaEventCreateWithFlags(&ctx->split_ev[g][i], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    if (bytes < ((size_t)64 << 20)) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
    // part i is bytes [at(i), at(i + 1)), parts of whole 8-byte words (the
    // state is FP64), the last one up to the end
    const size_t part = (bytes / 8 + NSPLIT - 1) / NSPLIT * 8;
    auto at = [&](int i) { return i >= NSPLIT ? bytes : std::min(bytes, (size_t)i * part); };
    e = cudaEventRecord(ctx->split_ev[g][NSPLIT - 1], st);
    for (int i = 1; i < NSPLIT && e == cudaSuccess; ++i) {
        cudaStream_t h = ctx->split_helper[g][i - 1];
        e = cudaStreamWaitEvent(h, ctx->split_ev[g][NSPLIT - 1], 0);
        if (e == cudaSuccess && at(i + 1) > at(i))
            e = cudaMemcpyAsync((char *)dst + at(i), (const char *)src + at(i), at(i + 1) - at(i), cudaMemcpyDefault, h);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->split_ev[g][i - 1], h);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, at(1), cudaMemcpyDefault, st);
    for (int i = 1; i < NSPLIT && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(st, ctx->split_ev[g][i - 1], 0);
    return e;
}

}  // namespace

nopcs_status nopcs_set_state(nopcs_ctx *ctx, int box, const double *q)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    if (!q) return fail(ctx, NOPCS_EINVAL, "q is NULL");
    BoxRes &b = ctx->boxes[box];
    CK(split_copy(ctx, 0, b.Qn(), q, 5 * (size_t)b.dev.np * sizeof(double), ctx->stream), "set_state");
    CK(refresh_mixed(b, ctx->stream), "set_state");
    CK(cudaStreamSynchronize(ctx->stream), "set_state");
    return NOPCS_OK;
}

nopcs_status nopcs_stage_state(nopcs_ctx *ctx, int box, const double *q)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    if (!q) return fail(ctx, NOPCS_EINVAL, "q is NULL");
    BoxRes &b = ctx->boxes[box];
    const size_t bytes = 5 * (size_t)b.dev.np * sizeof(double);
    if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "stage_state");
    if (!b.staged_ev) CK(cudaEventCreateWithFlags(&b.staged_ev, cudaEventDisableTiming), "stage_state");
    if (!b.committed_ev) {
        CK(cudaEventCreateWithFlags(&b.committed_ev, cudaEventDisableTiming), "stage_state");
        // nothing has read the buffer yet: the first wait below passes at once
        CK(cudaEventRecord(b.committed_ev, ctx->copy_stream), "stage_state");
    }
    if (!b.stage) {
        LedgerScope scope(&ctx->ledger);
        CK(dev_alloc((void **)&b.stage, bytes), "stage_state");
    }
    // the previous commit must have copied the staged state out first
    CK(cudaStreamWaitEvent(ctx->copy_stream, b.committed_ev, 0), "stage_state");
    CK(split_copy(ctx, 1, b.stage, q, bytes, ctx->copy_stream), "stage_state");
    CK(cudaEventRecord(b.staged_ev, ctx->copy_stream), "stage_state");
    b.staged = true;
    return NOPCS_OK;
}

nopcs_status nopcs_commit_state(nopcs_ctx *ctx, int box)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    BoxRes &b = ctx->boxes[box];
    if (!b.staged) return fail(ctx, NOPCS_EINVAL, "no state is staged for this box");
    CK(cudaStreamWaitEvent(ctx->stream, b.staged_ev, 0), "commit_state");
    CK(cudaMemcpyAsync(b.Qn(), b.stage, 5 * (size_t)b.dev.np * sizeof(double), cudaMemcpyDeviceToDevice,
                       ctx->stream),
       "commit_state");
    CK(cudaEventRecord(b.committed_ev, ctx->stream), "commit_state");
    CK(refresh_mixed(b, ctx->stream), "commit_state");
    b.staged = false;
    return NOPCS_OK;
}

nopcs_status nopcs_get_state(nopcs_ctx *ctx, int box, double *q)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    if (!q) return fail(ctx, NOPCS_EINVAL, "q is NULL");
    BoxRes &b = ctx->boxes[box];
    CK(cudaMemcpyAsync(q, b.Qn(), 5 * (size_t)b.dev.np * sizeof(double), cudaMemcpyDefault, ctx->stream),
       "get_state");
    CK(cudaStreamSynchronize(ctx->stream), "get_state");
    return NOPCS_OK;
}

nopcs_status nopcs_reset_state(nopcs_ctx *ctx, int box)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    BoxRes &b = ctx->boxes[box];
    CK(launch_initial_state(b.dev, b.d.seed, b.d.perturb_amp, b.Qn(), ctx->stream), "reset_state");
    CK(refresh_mixed(b, ctx->stream), "reset_state");
    b.step = 0;
    return NOPCS_OK;
}

nopcs_status nopcs_set_step(nopcs_ctx *ctx, int box, long long step)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    if (step < 0) return fail(ctx, NOPCS_EINVAL, "step must be >= 0");
    ctx->boxes[box].step = step;
    return NOPCS_OK;
}

nopcs_status nopcs_set_memory_limit(unsigned long long bytes)
{
    g_mem_limit.store(bytes);
    return NOPCS_OK;
}

nopcs_status nopcs_derivative(nopcs_ctx *ctx, int box, int axis, int order, int dtype, const void *f, void *df,
                              void *stream)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    if (axis < 0 || axis > 2) return fail(ctx, NOPCS_EINVAL, "axis must be 0, 1 or 2");
    if (order != 1 && order != 2 && order != NOPCS_ORDER_D2_COMPACT)
        return fail(ctx, NOPCS_EINVAL, "order must be 1, 2 or NOPCS_ORDER_D2_COMPACT");
    if (dtype != 0 && dtype != 1) return fail(ctx, NOPCS_EINVAL, "dtype must be 0 (f64) or 1 (f32)");
    if (!f || !df) return fail(ctx, NOPCS_EINVAL, "null field pointer");
    BoxRes &b = ctx->boxes[box];
    const size_t es = dtype == 0 ? 8 : 4;
    const size_t bytes = (size_t)b.dev.np * es;
    const char *fc = (const char *)f, *dc = (const char *)df;
    if (fc < dc + bytes && dc < fc + bytes) return fail(ctx, NOPCS_EINVAL, "f and df overlap");
    cudaStream_t st = (cudaStream_t)stream;
    const double scale = b.dev.inv_h[axis];
    if (order == NOPCS_ORDER_D2_COMPACT) {
        const double s2 = scale * scale;
        cudaError_t e = dtype == 0 ? launch_line_field2<double>(b.d2op64[axis].dev, axis, b.dev.n, (const double *)f,
                                                                (double *)df, s2, st)
                                   : launch_line_field2<float>(b.d2op32[axis].dev, axis, b.dev.n, (const float *)f,
                                                               (float *)df, s2, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "derivative");
        return NOPCS_OK;
    }
    const void *src = f;
    if (order == 2) {
        if (!b.scratch) {
            LedgerScope scope(&ctx->ledger);
            cudaError_t e = dev_alloc(&b.scratch, (size_t)b.dev.np * 8);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "order-2 scratch");
        }
        cudaError_t e = first_derivative(ctx, b, axis, dtype, f, b.scratch, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "derivative");
        src = b.scratch;
    }
    cudaError_t e = first_derivative(ctx, b, axis, dtype, src, df, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "derivative");
    return NOPCS_OK;
}

nopcs_status nopcs_rk_step(nopcs_ctx *ctx, int nsteps)
{
    nopcs_status s0 = check_ctx(ctx);
    if (s0 != NOPCS_OK) return s0;
    if (nsteps < 0) return fail(ctx, NOPCS_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return NOPCS_OK;
    if (!ctx->profiling && !ctx->step_exec && ctx->launch_mode == NOPCS_LAUNCH_GRAPH) {
        // capture one step of every box once, replayed for every later step;
        // each box's stage chain is its own branch of the graph (the boxes are
        // independent), so the GPU runs small boxes side by side
        const int nb = (int)ctx->boxes.size();
        if ((int)ctx->branch.size() < nb) {
            while ((int)ctx->branch.size() < nb) {
                cudaStream_t st;
                CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "graph branches");
                ctx->branch.push_back(st);
            }
            while ((int)ctx->branch_ev.size() < nb + 1) {
                cudaEvent_t ev;
                CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "graph branches");
                ctx->branch_ev.push_back(ev);
            }
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "graph capture");
        cudaError_t e = cudaEventRecord(ctx->branch_ev[nb], ctx->cap_stream);
        for (int i = 0; i < nb && e == cudaSuccess; ++i) {
            e = cudaStreamWaitEvent(ctx->branch[i], ctx->branch_ev[nb], 0);
            if (e == cudaSuccess) e = enqueue_step(ctx, ctx->boxes[i], ctx->branch[i]);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->branch_ev[i], ctx->branch[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap_stream, ctx->branch_ev[i], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(ctx, e, "graph capture");
        }
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "graph capture");
        e = cudaGraphInstantiate(&ctx->step_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ctx->step_exec = nullptr;
            return cuda_fail(ctx, e, "graph instantiate");
        }
    }
    for (int it = 0; it < nsteps; ++it) {
        if (ctx->profiling) {
            for (auto &b : ctx->boxes) CK(enqueue_step(ctx, b, ctx->stream), "rk step");
        } else if (ctx->launch_mode != NOPCS_LAUNCH_GRAPH) {
            CK(batch_launch(ctx->plan, ctx->dev_err, ctx->wait_s, ctx->launch_mode == NOPCS_LAUNCH_PERSISTENT_WITHHOLD,
                            ctx->stream),
               "persistent step");
        } else {
            CK(cudaGraphLaunch(ctx->step_exec, ctx->stream), "graph launch");
        }
        for (auto &b : ctx->boxes) {
            b.step += 1;
            if (b.d.filter_every > 0 && b.step % b.d.filter_every == 0)
                CK(enqueue_filter(ctx, b, ctx->stream), "filter");
        }
    }
    return NOPCS_OK;
}

nopcs_status nopcs_rhs(nopcs_ctx *ctx, int box, const double *q, void *r)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    if (!q || !r) return fail(ctx, NOPCS_EINVAL, "null pointer");
    BoxRes &b = ctx->boxes[box];
    cudaError_t e = enqueue_rhs_only(ctx, b, q, r, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rhs");
    CK(cudaStreamSynchronize(ctx->stream), "rhs");
    return NOPCS_OK;
}

nopcs_status nopcs_filter(nopcs_ctx *ctx, int box)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    CK(enqueue_filter(ctx, ctx->boxes[box], ctx->stream), "filter");
    return NOPCS_OK;
}

nopcs_status nopcs_diagnostics(nopcs_ctx *ctx, int box, nopcs_diag *out)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    if (!out) return fail(ctx, NOPCS_EINVAL, "out is NULL");
    BoxRes &b = ctx->boxes[box];
    {
        Timed t(ctx, ctx->stream, K_DIAG);
        CK(launch_diagnostics(b.dev, b.Qn(), b.partial, b.nblk_diag, b.diag_out, ctx->stream), "diagnostics");
    }
    double v[10];
    CK(cudaMemcpyAsync(v, b.diag_out, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream), "diagnostics");
    CK(cudaStreamSynchronize(ctx->stream), "diagnostics");
    out->mass = v[0];
    out->momentum[0] = v[1];
    out->momentum[1] = v[2];
    out->momentum[2] = v[3];
    out->energy_total = v[4];
    out->max_speed = v[5];
    out->max_dp = v[6];
    out->max_mach = v[7];
    out->nonfinite = v[8] != 0.0;
    out->step = b.step;
    if (out->nonfinite) return fail(ctx, NOPCS_EUNSTABLE, "non-finite values in the state");
    return NOPCS_OK;
}

nopcs_status nopcs_box_info(nopcs_ctx *ctx, int box, int *sub_n, int *deriv_form, int *tile_lines)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    const BoxRes &b = ctx->boxes[box];
    for (int a = 0; a < 3; ++a) {
        if (sub_n) sub_n[a] = b.sub_n[a];
        if (deriv_form)
            deriv_form[a] = b.deriv_gemm[a] ? (b.gemm_bf16[a] ? NOPCS_FORM_GEMM_BF16X3 : NOPCS_FORM_GEMM_3XTF32)
                                            : (b.deriv_band[a] ? NOPCS_FORM_BANDED : NOPCS_FORM_THOMAS);
        if (tile_lines) tile_lines[a] = b.lines[a];
    }
    return NOPCS_OK;
}

nopcs_status nopcs_plane_fields(nopcs_ctx *ctx, int box, int axis, int index, int what, double *out)
{
    nopcs_status s = check_box(ctx, box);
    if (s != NOPCS_OK) return s;
    if (axis < 0 || axis > 2) return fail(ctx, NOPCS_EINVAL, "axis must be 0, 1 or 2");
    BoxRes &b = ctx->boxes[box];
    if (index < 0 || index >= b.dev.n[axis]) return fail(ctx, NOPCS_EINVAL, "plane index out of range");
    if (what != NOPCS_PLANE_DP && what != NOPCS_PLANE_VORTICITY_TERMS)
        return fail(ctx, NOPCS_EINVAL, "what must be NOPCS_PLANE_DP or NOPCS_PLANE_VORTICITY_TERMS");
    if (!out) return fail(ctx, NOPCS_EINVAL, "out is NULL");
    CK(launch_plane_fields(b.dev, b.Qn(), axis, index, what, out, ctx->stream), "plane fields");
    return NOPCS_OK;
}

nopcs_status nopcs_synchronize(nopcs_ctx *ctx)
{
    nopcs_status s0 = check_ctx(ctx);
    if (s0 != NOPCS_OK) return s0;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
    CK(cudaDeviceSynchronize(), "synchronize");
    int flag = 0;
    CK(cudaMemcpy(&flag, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost), "synchronize");
    if (flag) {
        CK(cudaMemset(ctx->dev_err, 0, sizeof(int)), "synchronize");
        return fail(ctx, NOPCS_ETIMEOUT,
                    flag == 2 ? "a bounded wait of the persistent step kernel gave up (the box states are undefined)"
                              : "a bounded wait for the tensor cores gave up");
    }
    return NOPCS_OK;
}

nopcs_status nopcs_set_launch(nopcs_ctx *ctx, int mode, double wait_limit_s)
{
    nopcs_status s0 = check_ctx(ctx);
    if (s0 != NOPCS_OK) return s0;
    if (mode < NOPCS_LAUNCH_GRAPH || mode > NOPCS_LAUNCH_PERSISTENT_WITHHOLD)
        return fail(ctx, NOPCS_EINVAL, "mode must be NOPCS_LAUNCH_GRAPH, _PERSISTENT or _PERSISTENT_WITHHOLD");
    if (!(wait_limit_s > 0.0) || wait_limit_s > 3600.0)
        return fail(ctx, NOPCS_EINVAL, "wait_limit_s must be in (0, 3600]");
    if (mode != NOPCS_LAUNCH_GRAPH && !ctx->plan) {
        std::vector<BatchBoxIn> in;
        for (auto &b : ctx->boxes) {
            if (!b.mixed || b.d.visc_compact)
                return fail(ctx, NOPCS_EUNSUPPORTED,
                            "the persistent launch runs mixed-precision boxes with the explicit viscous terms");
            BatchBoxIn x;
            x.bx = b.dev;
            for (int a = 0; a < 3; ++a) {
                x.op[a] = b.dop32[a].dev;
                x.lines[a] = b.lines[a];
            }
            x.W[0] = b.Wm(0);
            x.W[1] = b.Wm(1);
            x.R = b.Rm();
            x.K = b.Km();
            x.Dn = b.Dn();
            x.Qn = b.Qn();
            in.push_back(x);
        }
        LedgerScope scope(&ctx->ledger);
        std::string msg;
        const cudaError_t e = batch_plan_build(in, &ctx->plan, msg);
        if (e != cudaSuccess)
            return msg.empty() ? cuda_fail(ctx, e, "persistent launch plan") : fail(ctx, NOPCS_EUNSUPPORTED, msg);
    }
    ctx->launch_mode = mode;
    ctx->wait_s = wait_limit_s;
    return NOPCS_OK;
}

nopcs_status nopcs_set_profiling(nopcs_ctx *ctx, int on)
{
    nopcs_status s0 = check_ctx(ctx);
    if (s0 != NOPCS_OK) return s0;
    if (on && ctx->pool.empty()) {
        ctx->pool.resize(4096);
        for (auto &p : ctx->pool) {
            CK(cudaEventCreate(&p.a), "event");
            CK(cudaEventCreate(&p.b), "event");
        }
    }
    if (!on && ctx->profiling) {
        CK(cudaStreamSynchronize(ctx->stream), "profiling");
        harvest(ctx);
    }
    ctx->profiling = on != 0;
    return NOPCS_OK;
}

nopcs_status nopcs_profile_read(nopcs_ctx *ctx, double *ms, long long *launches, int reset)
{
    nopcs_status s0 = check_ctx(ctx);
    if (s0 != NOPCS_OK) return s0;
    CK(cudaStreamSynchronize(ctx->stream), "profile read");
    harvest(ctx);
    for (int k = 0; k < NOPCS_NUM_KERNELS; ++k) {
        if (ms) ms[k] = ctx->prof_ms[k];
        if (launches) launches[k] = ctx->prof_n[k];
        if (reset) {
            ctx->prof_ms[k] = 0.0;
            ctx->prof_n[k] = 0;
        }
    }
    return NOPCS_OK;
}

const char *nopcs_kernel_name(int kind)
{
    if (kind < 0 || kind >= NOPCS_NUM_KERNELS) return nullptr;
    return KERNEL_NAMES[kind];
}

}  // extern "C"
