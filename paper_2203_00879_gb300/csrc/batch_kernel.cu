// One persistent launch per RK step for all boxes of a context (mixed form).
//
// A box's RK4 step is a chain of phases -- per stage the x, y and z flux
// sweeps (Sec. 3), the fused viscous / source / RK kernel (Sec. 2, Sec. 4) and
// the wall conditions (faces, then edges and corners) -- and each phase is a
// set of independent blocks: the blocks the stand-alone kernels would launch.
// Here one kernel runs them all.  The host lists work items (box, stage,
// phase, a run of blocks), each box's phases in order; every block of the
// persistent grid takes the next item from an atomic counter, waits until the
// box's previous phase has completed all its items, runs the item's blocks
// with the same device code as the stand-alone kernels (line_body.cuh,
// visc_body.cuh, wall_body.cuh), and counts the item done.  Boxes advance
// independently, so small boxes fill the GPU side by side without a launch
// per kernel and box.
//
// An item only ever waits for items listed before it, which blocks that were
// already running took, so the grid needs no co-residency to make progress.
// Each wait is bounded (globaltimer): when it gives up it sets the batch's
// abort word and the context's error word (the host reports NOPCS_ETIMEOUT),
// every later wait returns at once, and the kernel ends.  The completion
// counters use release / acquire at GPU scope; the data of a finished phase is
// read by plain (coherent) loads after the acquiring thread's barrier.
#include <string>
#include <vector>

#include "line_body.cuh"
#include "visc_body.cuh"
#include "wall_body.cuh"

namespace nopcs {

namespace {

constexpr int BT = 256;             // threads per block (the viscous tile's)
// wall nodes per tile of the face and edge phases: four passes of a block,
// so that a box's wall phases spread over many blocks instead of holding the
// box's next phase behind a few long items
constexpr int WALL_CHUNK = 4 * BT;
enum { PH_SX = 0, PH_SY, PH_SZ, PH_VISC, PH_FACE, PH_EDGE, PH_CORNER, NPH };

struct BStage {
    LineArgs<float> la[3];
    VArgs<float> va;
    double *Q;  // wall conditions: the FP64 state (stage 4) or null (stage state Ww)
    float *Dn, *Wf, *Ww;
};

struct BBox {
    LineOpDev op[3];
    BoxDev bx;
    int nt[3];       // working threads of each sweep (those of its stand-alone launch)
    int xline;       // the x sweep is the whole-line kernel
    int ntile[NPH];  // blocks of the stand-alone launch per phase
    int chunk[NPH];  // blocks per item
    int nitem[NPH];  // items per phase
    int gx, gy;      // viscous grid in x and y
    BStage st[4];
};

struct BItem {
    int box, stage, phase, first;
};

struct BParams {
    const BBox *boxes;
    const BItem *items;
    int nitems;
    int *next;   // work counter
    int *abort;  // set when a wait gave up
    int *done;   // [box][stage][phase] finished items
    int *err;    // the context's error word (2: a wait gave up)
    unsigned long long wait_ns;
    int withhold;  // test: box 0's first dependency needs one item more than exists
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int *p, int v)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until *ctr >= need, at most wait_ns; false if the wait gave up or the
// batch was aborted.
__device__ bool wait_at_least(const BParams &p, const int *ctr, int need)
{
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (ld_acquire(ctr) >= need) return true;
        if (ld_acquire(p.abort) != 0) return false;
        if (now_ns() - t0 > p.wait_ns) {
            atomicExch(p.abort, 1);
            atomicCAS(p.err, 0, 2);
            return false;
        }
        __nanosleep(256);
    }
}

// The phase bodies are separate (not inlined) functions, so that each gets the
// kernel's whole register budget instead of all of them sharing one
// allocation inside the item loop.
__device__ __noinline__ void run_sweep_x(const LineOpDev &op, const LineArgs<float> &la, int v, unsigned char *sm,
                                         int nt, int xline)
{
    if (xline)
        xline_body<float, MODE_FLUX>(op, la, v);
    else
        line_body<float, MODE_FLUX, 0>(op, la, v, nt);
}
__device__ __noinline__ void run_sweep_y(const LineOpDev &op, const LineArgs<float> &la, int v, unsigned char *sm,
                                         int nt)
{
    line_body<float, MODE_FLUX, 1>(op, la, v, nt);
}
__device__ __noinline__ void run_sweep_z(const LineOpDev &op, const LineArgs<float> &la, int v, unsigned char *sm,
                                         int nt)
{
    line_body<float, MODE_FLUX, 2>(op, la, v, nt);
}
// the viscous stage kernel in the same specialisation as the stand-alone
// launch (per stage, gravity along z) or the generic one
template <class S>
__device__ __noinline__ void run_visc(const VArgs<float> &va, int bx, int by, int bz, unsigned char *sm)
{
    visc_rk_block<float, S>(va, bx, by, bz, sm);
}
__device__ __forceinline__ void run_visc_any(const VArgs<float> &va, int bx, int by, int bz, unsigned char *sm)
{
    if (va.ga == 2) {
        switch (va.stage) {
        case 1: run_visc<Spec<1, 2>>(va, bx, by, bz, sm); return;
        case 2: run_visc<Spec<2, 2>>(va, bx, by, bz, sm); return;
        case 3: run_visc<Spec<3, 2>>(va, bx, by, bz, sm); return;
        case 4: run_visc<Spec<4, 2>>(va, bx, by, bz, sm); return;
        }
    }
    run_visc<RunSpec>(va, bx, by, bz, sm);
}

__global__ void __launch_bounds__(BT, 3) batch_step_kernel(const BParams p)
{
    extern __shared__ __align__(32) unsigned char smraw[];
    __shared__ int s_item, s_go;
    // the item's arguments, copied from the device box table: the phase code
    // then reads its pointers and constants from shared memory instead of
    // through global loads ahead of every data access
    constexpr int ARGW = (int)((sizeof(VArgs<float>) > sizeof(LineOpDev) + sizeof(LineArgs<float>)
                                    ? sizeof(VArgs<float>)
                                    : sizeof(LineOpDev) + sizeof(LineArgs<float>)) /
                               8);
    __shared__ unsigned long long s_args[ARGW];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(p.next, 1);
        __syncthreads();
        const int i = s_item;
        if (i >= p.nitems) return;
        const BItem it = p.items[i];
        const BBox &B = p.boxes[it.box];
        if (threadIdx.x == 0) {
            // the previous phase of this box (of the previous stage for the
            // first phase of a stage)
            int ds = it.stage, dp = it.phase - 1;
            if (dp < 0) {
                ds -= 1;
                dp = NPH - 1;
            }
            bool ok = ld_acquire(p.abort) == 0;
            if (ok && ds >= 0) {
                const int need = B.nitem[dp] + (p.withhold && it.box == 0 && ds == 0 && dp == PH_SX ? 1 : 0);
                ok = wait_at_least(p, p.done + (it.box * 4 + ds) * NPH + dp, need);
            }
            s_go = ok;
            // acquire at GPU scope before the block's barrier: the block's
            // plain loads after it see the finished phase's data (the L1 lines
            // of this SM are not left stale by it); the whole block's loads
            // going to L2 only instead (-dlcm=cg) gave the same bits and was
            // three times slower
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
        }
        __syncthreads();
        if (s_go) {
            const BStage &S = B.st[it.stage];
            LineOpDev *sop = reinterpret_cast<LineOpDev *>(s_args);
            LineArgs<float> *sla = reinterpret_cast<LineArgs<float> *>(s_args + sizeof(LineOpDev) / 8);
            VArgs<float> *sva = reinterpret_cast<VArgs<float> *>(s_args);
            {
                auto copy = [&](void *dst, const void *src, int bytes) {
                    const unsigned long long *a = (const unsigned long long *)src;
                    unsigned long long *b = (unsigned long long *)dst;
                    for (int k = threadIdx.x; k < bytes / 8; k += BT) b[k] = a[k];
                };
                if (it.phase <= PH_SZ) {
                    copy(sop, &B.op[it.phase], (int)sizeof(LineOpDev));
                    copy(sla, &S.la[it.phase], (int)sizeof(LineArgs<float>));
                } else if (it.phase == PH_VISC) {
                    copy(sva, &S.va, (int)sizeof(VArgs<float>));
                }
                __syncthreads();
            }
            const int last = min(it.first + B.chunk[it.phase], B.ntile[it.phase]);
            for (int v = it.first; v < last; ++v) {
                switch (it.phase) {
                case PH_SX: run_sweep_x(*sop, *sla, v, smraw, B.nt[0], B.xline); break;
                case PH_SY: run_sweep_y(*sop, *sla, v, smraw, B.nt[1]); break;
                case PH_SZ: run_sweep_z(*sop, *sla, v, smraw, B.nt[2]); break;
                case PH_VISC: run_visc_any(*sva, v % B.gx, (v / B.gx) % B.gy, v / (B.gx * B.gy), smraw); break;
                case PH_FACE: {
                    const long long tot = face_count(B.bx);
                    const long long t1 = min(tot, (long long)(v + 1) * WALL_CHUNK);
                    for (long long t = (long long)v * WALL_CHUNK + threadIdx.x; t < t1; t += BT) {
                        int c[3];
                        face_node(B.bx, t, c);
                        wall_node(B.bx, c, S.Q, S.Dn, S.Wf, S.Ww);
                    }
                    break;
                }
                case PH_EDGE: {
                    const long long tot = edge_count(B.bx);
                    const long long t1 = min(tot, (long long)(v + 1) * WALL_CHUNK);
                    for (long long t = (long long)v * WALL_CHUNK + threadIdx.x; t < t1; t += BT) {
                        int c[3];
                        edge_node(B.bx, t, c);
                        wall_node(B.bx, c, S.Q, S.Dn, S.Wf, S.Ww);
                    }
                    break;
                }
                default: {  // the corners, which read the edges
                    if (threadIdx.x < 8) {
                        int c[3];
                        corner_node(B.bx, threadIdx.x, c);
                        wall_node(B.bx, c, S.Q, S.Dn, S.Wf, S.Ww);
                    }
                }
                }
                __syncthreads();  // the next block of the item reuses the shared memory
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            red_release_add(p.done + (it.box * 4 + it.stage) * NPH + it.phase, 1);
        }
    }
}

}  // namespace

struct BatchPlan {
    void *mem = nullptr;      // boxes, items, counters
    BParams p{};
    int grid = 0;
    size_t smem = 0;
    size_t counter_bytes = 0;
    int *counters = nullptr;  // next, abort, done[]
};

cudaError_t batch_plan_build(const std::vector<BatchBoxIn> &in, BatchPlan **out, std::string &msg)
{
    *out = nullptr;
    const int nb = (int)in.size();
    std::vector<BBox> boxes(nb);
    std::vector<BItem> items;
    size_t smem = ring_bytes<float>();
    for (int b = 0; b < nb; ++b) {
        const BatchBoxIn &I = in[b];
        BBox &B = boxes[b];
        B.bx = I.bx;
        for (int a = 0; a < 3; ++a) B.op[a] = I.op[a];
        const long long np = I.bx.np;
        for (int s = 1; s <= 4; ++s) {
            BStage &S = B.st[s - 1];
            const float *Win = I.W[(s - 1) & 1];
            float *Wout = I.W[s & 1];
            for (int a = 0; a < 3; ++a) {
                LineArgs<float> &la = S.la[a];
                la = LineArgs<float>{};
                for (int d = 0; d < 3; ++d) la.n[d] = I.bx.n[d];
                for (int k = 0; k < 6; ++k) la.in[k] = Win + (size_t)k * np;
                for (int k = 0; k < 5; ++k) la.out[k] = I.R + (size_t)k * np;
                la.scale = (float)I.bx.inv_h[a];
                la.first = a == 0;
                la.ga = I.bx.ga;
                la.b0 = I.bx.rho_b32;
                la.b1 = I.bx.H_b32;
                // the stand-alone launch's geometry (same tile width and
                // working threads, so the same arithmetic and rounding)
                LineGrid g;
                const int pref = I.lines[a] > 0 ? I.lines[a] : 32;
                bool ok = a == 0 ? line_grid<float, MODE_FLUX, 0>(I.op[a], la, pref, 0, XLINE_MAX_LINES, g)
                                 : (a == 1 ? line_grid<float, MODE_FLUX, 1>(I.op[a], la, pref, 0, XLINE_MAX_LINES, g)
                                           : line_grid<float, MODE_FLUX, 2>(I.op[a], la, pref, 0, XLINE_MAX_LINES, g));
                const int cols = g.xline ? I.op[0].nsub * 5 * la.lines : 0;
                if (!ok || g.nblk > 0x7fffffff || (g.xline ? cols > BT : g.threads > BT)) {
                    msg = "a flux sweep of a box does not fit the batched kernel's blocks";
                    return cudaErrorInvalidConfiguration;
                }
                if (g.smem > smem) smem = g.smem;
                B.ntile[PH_SX + a] = (int)g.nblk;
                B.nt[a] = g.threads;
                if (a == 0) B.xline = g.xline ? 1 : 0;
            }
            StageRegs<float> r;
            r.Qn = I.Qn;
            r.Kacc = I.K;
            r.Dn = I.Dn;
            r.Wn = Wout;
            S.va = make_vargs<float>(I.bx, Win, I.R, s, r);
            B.gx = (I.bx.n[0] + TX - 1) / TX;
            B.gy = (I.bx.n[1] + TY - 1) / TY;
            // z chunk of the stand-alone launch (8 to 32 planes per block)
            const long long want = 152LL * 8;
            const int nzc = (int)((want + (long long)B.gx * B.gy - 1) / ((long long)B.gx * B.gy));
            int zc = (I.bx.n[2] + nzc - 1) / nzc;
            zc = zc < 8 ? 8 : (zc > 32 ? 32 : zc);
            S.va.zc = zc;
            B.ntile[PH_VISC] = B.gx * B.gy * ((I.bx.n[2] + zc - 1) / zc);
            if (s < 4) {
                S.Q = nullptr;
                S.Dn = nullptr;
                S.Wf = nullptr;
                S.Ww = Wout;
            } else {
                S.Q = I.Qn;
                S.Dn = I.Dn;
                S.Wf = Wout;
                S.Ww = nullptr;
            }
        }
        const long long nface = 2 * ((long long)(I.bx.n[1] - 2) * (I.bx.n[2] - 2) +
                                     (long long)(I.bx.n[0] - 2) * (I.bx.n[2] - 2) +
                                     (long long)(I.bx.n[0] - 2) * (I.bx.n[1] - 2));
        B.ntile[PH_FACE] = (int)((nface + WALL_CHUNK - 1) / WALL_CHUNK);
        B.ntile[PH_EDGE] = (int)((edge_count(I.bx) + WALL_CHUNK - 1) / WALL_CHUNK);
        B.ntile[PH_CORNER] = 1;
        // blocks per item: about a quarter of a GPU wave per phase of a big
        // box, single blocks for small ones
        for (int ph = 0; ph < NPH; ++ph) {
            const int nt = B.ntile[ph] > 0 ? B.ntile[ph] : 1;
            int ch = nt / (152 * 3 * 16);
            B.chunk[ph] = ch < 1 ? 1 : ch;
            B.nitem[ph] = (nt + B.chunk[ph] - 1) / B.chunk[ph];
        }
    }
    // Items on diagonals: box b's phase g (= stage x NPH + phase) on diagonal
    // g + b, diagonals in order, boxes in order within one.  Every box's
    // phases stay in order (the dependency rule), and consecutive phases of a
    // box are a whole diagonal apart: while a block waits for box b's
    // previous phase, the items behind it belong to other boxes at other
    // phases, whose dependencies are older.  (Stage-major order, every box at
    // the same phase, left blocks waiting at each phase boundary.)
    for (int d = 0; d < 4 * NPH + nb - 1; ++d)
        for (int b = 0; b < nb; ++b) {
            const int g = d - b;
            if (g < 0 || g >= 4 * NPH) continue;
            const int s = g / NPH, ph = g % NPH;
            for (int k = 0; k < boxes[b].nitem[ph]; ++k) items.push_back(BItem{b, s, ph, k * boxes[b].chunk[ph]});
        }
    if (smem > 227 * 1024) {
        msg = "the batched kernel's blocks need more shared memory than a block can have";
        return cudaErrorInvalidConfiguration;
    }
    BatchPlan *P = new BatchPlan();
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t bb = al(sizeof(BBox) * nb), ib = al(sizeof(BItem) * items.size());
    P->counter_bytes = sizeof(int) * (2 + (size_t)nb * 4 * NPH);
    cudaError_t e = dev_alloc(&P->mem, bb + ib + P->counter_bytes);
    if (e != cudaSuccess) {
        delete P;
        return e;
    }
    char *base = (char *)P->mem;
    e = cudaMemcpy(base, boxes.data(), sizeof(BBox) * nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + bb, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0, nsm = 0, dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_step_kernel, BT, smem);
    if (e != cudaSuccess || per_sm < 1) {
        dev_free(P->mem);
        delete P;
        msg = "the batched kernel does not fit an SM";
        return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
    }
    P->counters = (int *)(base + bb + ib);
    P->p.boxes = (const BBox *)base;
    P->p.items = (const BItem *)(base + bb);
    P->p.nitems = (int)items.size();
    P->p.next = P->counters;
    P->p.abort = P->counters + 1;
    P->p.done = P->counters + 2;
    P->grid = per_sm * nsm < P->p.nitems ? per_sm * nsm : P->p.nitems;
    P->smem = smem;
    *out = P;
    return cudaSuccess;
}

cudaError_t batch_launch(BatchPlan *P, int *err, double wait_s, int withhold, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(P->counters, 0, P->counter_bytes, st);
    if (e != cudaSuccess) return e;
    BParams p = P->p;
    p.err = err;
    p.wait_ns = (unsigned long long)(wait_s * 1e9);
    p.withhold = withhold;
    batch_step_kernel<<<P->grid, BT, P->smem, st>>>(p);
    return cudaGetLastError();
}

void batch_plan_free(BatchPlan *P)
{
    if (!P) return;
    if (P->mem) dev_free(P->mem);
    delete P;
}

int batch_plan_items(const BatchPlan *P) { return P ? P->p.nitems : 0; }

}  // namespace nopcs
