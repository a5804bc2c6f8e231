// One box split into z-slabs across ranks (arXiv 2203.00879, Sec. 3 and the
// rank grid of Sec. 4): the NOHAP derivative of a slab's own sub-domains from
// the slab's planes plus halo planes received from the neighbouring ranks.
//
// NOHAP closes every sub-domain with the end rows of the global equivalent
// explicit scheme C = A^-1 B (Eqs. CS:fpCf, CS:fpCf_i), which reach n_b points
// (48 in FP64, 24 in FP32 at the tap threshold) into the neighbours, and
// solves the rows between by Thomas.  A rank that owns whole sub-domains
// [z0, z1) of a line therefore needs only the planes those end rows and the
// interior stencil reach, [lo, z0) and [z1, hi); with them in its own memory
// it computes exactly what a single-domain solve of the whole line gives on
// its sub-domains, bit for bit, with no further exchange.
//
// The slab's z operator is the global line operator (built for the whole
// line, so the end-row taps near a wall are the global rows) restricted to
// the own sub-domains, with every row index shifted to the local plane range
// [lo, hi) and the line length set to hi - lo: the wall-closure rows then
// fall on the true wall only in the first and the last slab, and the same
// line kernels run on it unchanged.  Along x and y a slab's planes are whole
// lines: the box's own operators apply.
#include <string>

#include "nopcs_internal.cuh"

struct nopcs_slab {
    int device = 0;
    int n[3] = {0, 0, 0};  // global nx, ny, nz
    int z0 = 0, z1 = 0;
    double inv_h[3] = {0, 0, 0};
    int lo[2] = {0, 0}, hi[2] = {0, 0};  // held planes per dtype (0 f64, 1 f32)
    nopcs::LineOpBuf zop[2], xop[2], yop[2];
    std::string err;
};

namespace nopcs {

namespace {

thread_local std::string g_slab_error;

// Restrict a global line operator to its sub-domains inside [z0, z1) and
// shift every row index to the local range; off and nloc give the local
// origin and length.  False if [z0, z1) does not start and end on sub-domain
// boundaries.
bool slice_line_op(const LineOpHost &g, int z0, int z1, LineOpHost &out, int &off, int &nloc, std::string &msg)
{
    int b0 = -1, b1 = -1;
    for (int b = 0; b < g.nsub; ++b) {
        const int *rec = &g.sub[(size_t)b * SUB_REC];
        if (rec[0] == z0) b0 = b;
        if (rec[1] == z1 - 1) b1 = b + 1;
    }
    if (b0 < 0 || b1 <= b0) {
        msg = "the slab [z0, z1) must start and end on NOHAP sub-domain boundaries of the line";
        return false;
    }
    int tlo = g.N, thi = -1;
    for (int b = b0; b < b1; ++b) {
        const int *rec = &g.sub[(size_t)b * SUB_REC];
        tlo = rec[2] < tlo ? rec[2] : tlo;
        thi = rec[3] > thi ? rec[3] : thi;
    }
    off = tlo;
    nloc = thi + 1 - tlo;
    out = g;
    out.N = nloc;
    out.nsub = b1 - b0;
    out.sub.assign(g.sub.begin() + (size_t)b0 * SUB_REC, g.sub.begin() + (size_t)b1 * SUB_REC);
    // row fields of a record: s, e, tile_lo, tile_hi, the two end rows' first
    // columns, the implicit run, the solve window; lengths and tap offsets stay
    static const int ROWS[] = {0, 1, 2, 3, 4, 7, 10, 11, 12, 13};
    for (int b = 0; b < out.nsub; ++b)
        for (int k : ROWS) out.sub[(size_t)b * SUB_REC + k] -= off;
    return true;
}

bool build_slab_line(int N, int sub_n, int kind, double thresh, int z0, int z1, LineOpHost &out, int &off, int &nloc,
                     std::string &msg)
{
    LineOpHost g;
    if (!build_line_op(N, sub_n, kind, 0.0, thresh, g, msg)) return false;
    return slice_line_op(g, z0, z1, out, off, nloc, msg);
}

nopcs_status slab_fail(nopcs_slab *s, nopcs_status st, const std::string &m)
{
    if (s)
        s->err = m;
    else
        g_slab_error = m;
    return st;
}

}  // namespace

}  // namespace nopcs

using namespace nopcs;

extern "C" {

nopcs_status nopcs_slab_create(const nopcs_box_desc *box, int z0, int z1, nopcs_slab **out)
{
    if (!out) return slab_fail(nullptr, NOPCS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!box) return slab_fail(nullptr, NOPCS_EINVAL, "box is NULL");
    for (int a = 0; a < 3; ++a) {
        if (box->n[a] < 5 || !(box->len[a] > 0.0))
            return slab_fail(nullptr, NOPCS_EINVAL, "each axis needs at least 5 points and a positive length");
        if (box->sub_n[a] < 0 || (box->sub_n[a] > 0 && box->sub_n[a] < 3))
            return slab_fail(nullptr, NOPCS_EINVAL, "sub_n must be 0 or >= 3 (no tuning for slabs)");
    }
    if (!(z0 >= 0 && z1 > z0 && z1 <= box->n[2]))
        return slab_fail(nullptr, NOPCS_EINVAL, "need 0 <= z0 < z1 <= n[2]");
    nopcs_slab *s = new nopcs_slab();
    for (int a = 0; a < 3; ++a) {
        s->n[a] = box->n[a];
        s->inv_h[a] = (box->n[a] - 1) / box->len[a];
    }
    s->z0 = z0;
    s->z1 = z1;
    std::string msg;
    const double th[2] = {1e-16, 1e-8};
    for (int d = 0; d < 2; ++d) {
        int off = 0, nloc = 0;
        if (!build_slab_line(box->n[2], box->sub_n[2], KIND_DERIV, th[d], z0, z1, s->zop[d].host, off, nloc, msg) ||
            (long long)box->n[0] * box->n[1] * nloc >= (1LL << 31) ||
            !build_line_op(box->n[0], box->sub_n[0], KIND_DERIV, 0.0, th[d], s->xop[d].host, msg) ||
            !build_line_op(box->n[1], box->sub_n[1], KIND_DERIV, 0.0, th[d], s->yop[d].host, msg)) {
            delete s;
            return slab_fail(nullptr, NOPCS_EINVAL, msg.empty() ? "slab too large" : msg);
        }
        s->lo[d] = off;
        s->hi[d] = off + nloc;
    }
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = init_line_kernels();
    for (int d = 0; d < 2 && e == cudaSuccess; ++d) {
        e = s->zop[d].upload();
        if (e == cudaSuccess) e = s->xop[d].upload();
        if (e == cudaSuccess) e = s->yop[d].upload();
    }
    if (e != cudaSuccess) {
        nopcs_slab_destroy(s);
        return slab_fail(nullptr, e == cudaErrorMemoryAllocation ? NOPCS_ENOMEM : NOPCS_ECUDA,
                         std::string("slab tables: ") + cudaGetErrorString(e));
    }
    *out = s;
    return NOPCS_OK;
}

void nopcs_slab_destroy(nopcs_slab *s)
{
    if (!s) return;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) cur = -1;
    if (cur != s->device) cudaSetDevice(s->device);
    for (int d = 0; d < 2; ++d) {
        s->zop[d].release();
        s->xop[d].release();
        s->yop[d].release();
    }
    const int dev = s->device;
    delete s;
    if (cur >= 0 && cur != dev) cudaSetDevice(cur);
}

const char *nopcs_slab_last_error(const nopcs_slab *s) { return s ? s->err.c_str() : g_slab_error.c_str(); }

nopcs_status nopcs_slab_extent(const nopcs_slab *s, int dtype, int *lo, int *hi)
{
    if (!s || (dtype != 0 && dtype != 1)) return NOPCS_EINVAL;
    if (lo) *lo = s->lo[dtype];
    if (hi) *hi = s->hi[dtype];
    return NOPCS_OK;
}

nopcs_status nopcs_slab_derivative(nopcs_slab *s, int axis, int dtype, const void *f, void *df, void *stream)
{
    if (!s) return NOPCS_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != s->device)
        return slab_fail(s, NOPCS_EINVAL, "the current CUDA device is not the slab's device");
    if (axis < 0 || axis > 2) return slab_fail(s, NOPCS_EINVAL, "axis must be 0, 1 or 2");
    if (dtype != 0 && dtype != 1) return slab_fail(s, NOPCS_EINVAL, "dtype must be 0 (f64) or 1 (f32)");
    if (!f || !df) return slab_fail(s, NOPCS_EINVAL, "null field pointer");
    const size_t es = dtype == 0 ? 8 : 4, plane = (size_t)s->n[0] * s->n[1];
    const int lo = s->lo[dtype], hi = s->hi[dtype];
    const char *fc = (const char *)f, *dc = (const char *)df;
    if (fc < dc + plane * (s->z1 - s->z0) * es && dc < fc + plane * (hi - lo) * es)
        return slab_fail(s, NOPCS_EINVAL, "f and df overlap");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (axis == 2) {
        // the kernel writes the own rows [z0 - lo, z1 - lo) of a local field;
        // df holds only those, so it is passed as the base they are offset from
        const int n[3] = {s->n[0], s->n[1], hi - lo};
        const size_t shift = plane * (size_t)(s->z0 - lo) * es;
        e = dtype == 0 ? launch_line_field<double>(s->zop[0].dev, 2, n, (const double *)f,
                                                   (double *)(void *)((char *)df - shift), s->inv_h[2], st)
                       : launch_line_field<float>(s->zop[1].dev, 2, n, (const float *)f,
                                                  (float *)(void *)((char *)df - shift), s->inv_h[2], st);
    } else {
        // whole lines: the own planes alone
        const int n[3] = {s->n[0], s->n[1], s->z1 - s->z0};
        const LineOpDev &op = axis == 0 ? s->xop[dtype].dev : s->yop[dtype].dev;
        const char *own = fc + plane * (size_t)(s->z0 - lo) * es;
        e = dtype == 0 ? launch_line_field<double>(op, axis, n, (const double *)own, (double *)df, s->inv_h[axis], st)
                       : launch_line_field<float>(op, axis, n, (const float *)own, (float *)df, s->inv_h[axis], st);
    }
    if (e != cudaSuccess) return slab_fail(s, NOPCS_ECUDA, std::string("slab derivative: ") + cudaGetErrorString(e));
    return NOPCS_OK;
}

nopcs_status nopcs_slab_line_apply(int N, int sub_n, double thresh, int z0, int z1, const double *f, double *g,
                                   int *lo, int *hi)
{
    LineOpHost op;
    int off = 0, nloc = 0;
    std::string msg;
    if (!(thresh > 0.0) || !build_slab_line(N, sub_n, KIND_DERIV, thresh, z0, z1, op, off, nloc, msg))
        return NOPCS_EINVAL;
    if (lo) *lo = off;
    if (hi) *hi = off + nloc;
    if (!f && !g) return NOPCS_OK;
    if (!f || !g) return NOPCS_EINVAL;
    std::vector<double> loc((size_t)nloc, 0.0);
    apply_line_host(op, f, loc.data());
    for (int i = z0; i < z1; ++i) g[i - z0] = loc[(size_t)(i - off)];
    return NOPCS_OK;
}

}  // extern "C"
