// Host construction of the NOHAP line operators (arXiv 2203.00879, Sec. 3).
//
// For a line of N nodes the global compact system is [A]{g} = [B]{f}:
//   derivative (OUCS3, eta = 0): implicit rows 2..N-3 with A = (alpha, 1, alpha),
//     B = (-b2, -b1, 0, b1, b2) (interior coefficients printed after Eq.
//     CS:AfpBf; the printed "+-" signs are read as an antisymmetric B), and
//     explicit wall closures in rows 0, 1, N-2, N-1 (A = identity there);
//   filter: implicit rows 3..N-4 with A = (alpha_f, 1, alpha_f) and the
//     symmetric 7-point sixth-order right-hand side; rows 0..2 and N-3..N-1 are
//     left unfiltered (identity).
// NOHAP takes every sub-domain end value from the equivalent explicit scheme
// g_i = sum_j C_ij f_j with C = A^-1 B (Eqs. CS:fpCf, CS:fpCf_i), keeping the
// taps with |C_ij| >= thresh.  Row i of C is computed here as y^T B with
// A^T y = e_i: one tridiagonal solve per end row instead of inverting A.
// The implicit rows between two known values are solved by the Thomas
// algorithm, whose factors depend only on the position in the run and are
// tabulated once.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "nopcs_internal.cuh"

namespace nopcs {

static const double OUCS3_ALPHA = 0.3793894912;
static const double OUCS3_B1 = 0.7877868952;
static const double OUCS3_B2 = 0.045801298;
static const double WALL_BETA = -0.025;

int partition_rule(int N, int sub_n, int *start)
{
    // blocks of sub_n; a remainder of >= 3 points forms its own last block,
    // a remainder of 1 or 2 points is appended to the previous block
    if (sub_n <= 0 || sub_n >= N) {
        start[0] = 0;
        start[1] = N;
        return 1;
    }
    int full = N / sub_n, rest = N % sub_n;
    int nb = rest >= 3 ? full + 1 : full;
    for (int b = 0; b < nb; ++b) start[b] = b * sub_n;
    start[nb] = N;
    return nb;
}

namespace {

struct Banded {
    // B stored by rows with up to 7 taps: row r covers columns c0[r] .. c0[r] + 6
    int N;
    std::vector<int> c0;
    std::vector<double> w;  // N * 7
    double at(int r, int c) const
    {
        int k = c - c0[r];
        return (k >= 0 && k < 7) ? w[(size_t)r * 7 + k] : 0.0;
    }
};

bool is_explicit(const LineOpHost &op, int i) { return i < op.nexp || i > op.N - 1 - op.nexp; }

// A^T y = e_i for the tridiagonal A of `op` (diagonally dominant: no pivoting).
void solve_At(const LineOpHost &op, int i, std::vector<double> &y)
{
    int N = op.N;
    // A[r][r-1] = A[r][r+1] = alpha on implicit rows r, 0 otherwise.
    // (A^T)[r][r-1] = A[r-1][r], (A^T)[r][r+1] = A[r+1][r].
    std::vector<double> lo(N), di(N), up(N), d(N, 0.0);
    for (int r = 0; r < N; ++r) {
        lo[r] = (r > 0 && !is_explicit(op, r - 1)) ? op.alpha : 0.0;
        up[r] = (r < N - 1 && !is_explicit(op, r + 1)) ? op.alpha : 0.0;
        di[r] = 1.0;
    }
    d[i] = 1.0;
    for (int r = 1; r < N; ++r) {
        double m = lo[r] / di[r - 1];
        di[r] -= m * up[r - 1];
        d[r] -= m * d[r - 1];
    }
    y.assign(N, 0.0);
    y[N - 1] = d[N - 1] / di[N - 1];
    for (int r = N - 2; r >= 0; --r) y[r] = (d[r] - up[r] * y[r + 1]) / di[r];
}

// banded B of the global system: explicit closure rows, then the interior
// right-hand side (antisymmetric for the derivative, symmetric for the filter)
void fill_B(const LineOpHost &op, Banded &B)
{
    const int N = op.N;
    auto setB = [&](int r, int c, double v) {
        int k = c - B.c0[r];
        B.w[(size_t)r * 7 + k] = v;
    };
    for (int r = 0; r < N; ++r) {
        if (r < op.nexp) {
            B.c0[r] = 0;
            for (int j = 0; j < 5 && j < N; ++j) setB(r, j, op.ex[r][j]);
        } else if (r > N - 1 - op.nexp) {
            int rr = N - 1 - r;
            B.c0[r] = N - 7 < 0 ? 0 : N - 7;
            for (int j = 0; j < 5; ++j)
                if (op.ex[rr][j] != 0.0) setB(r, N - 1 - j, op.ex_sign * op.ex[rr][j]);
        } else {
            B.c0[r] = r - 3;
            if (op.kind == KIND_DERIV) {
                setB(r, r - 2, -op.rb[1]);
                setB(r, r - 1, -op.rb[0]);
                setB(r, r + 1, op.rb[0]);
                setB(r, r + 2, op.rb[1]);
            } else {
                setB(r, r, op.rb[0]);
                for (int k = 1; k <= 3; ++k) {
                    setB(r, r - k, op.rb[k]);
                    setB(r, r + k, op.rb[k]);
                }
            }
        }
    }
}

// row i of the global C = A^-1 B (dense, length N): explicit rows are their
// own B rows; implicit rows are y^T B with A^T y = e_i
void global_C_row(const LineOpHost &op, const Banded &B, int i, std::vector<double> &y, std::vector<double> &crow)
{
    const int N = op.N;
    crow.assign(N, 0.0);
    if (is_explicit(op, i)) {
        for (int j = 0; j < N; ++j) crow[j] = B.at(i, j);
        return;
    }
    solve_At(op, i, y);
    for (int r = 0; r < N; ++r) {
        if (y[r] == 0.0) continue;
        for (int k = 0; k < 7; ++k) {
            int c = B.c0[r] + k;
            if (c >= 0 && c < N) crow[c] += y[r] * B.w[(size_t)r * 7 + k];
        }
    }
}

}  // namespace

bool build_line_op(int N, int sub_n, int kind, double alpha_f, double thresh, LineOpHost &op,
                   std::string &msg)
{
    if (N < 5) {
        msg = "a line needs at least 5 points";
        return false;
    }
    if (sub_n > 0 && sub_n < 3) {
        msg = "sub-domain length must be >= 3 (or 0 for a single sub-domain)";
        return false;
    }
    if (!(thresh > 0.0)) {
        msg = "truncation threshold must be positive";
        return false;
    }
    op = LineOpHost();
    op.N = N;
    op.kind = kind;
    op.sub_n = sub_n;
    op.thresh = thresh;
    Banded B;
    B.N = N;
    B.c0.assign(N, 0);
    B.w.assign((size_t)N * 7, 0.0);
    int w;  // half-width of the interior right-hand side
    if (kind == KIND_DERIV) {
        op.nexp = 2;
        op.alpha = OUCS3_ALPHA;
        op.rb[0] = OUCS3_B1;
        op.rb[1] = OUCS3_B2;
        w = 2;
        // wall closure rows (explicit): one-sided second order at the wall, the
        // fourth-order beta family next to it; mirrored antisymmetrically
        const double be = WALL_BETA;
        const double r0[5] = {-1.5, 2.0, -0.5, 0.0, 0.0};
        const double r1[5] = {2.0 * be / 3.0 - 1.0 / 3.0, -(8.0 * be / 3.0 + 0.5), 4.0 * be + 1.0,
                              -(8.0 * be / 3.0 + 1.0 / 6.0), 2.0 * be / 3.0};
        for (int j = 0; j < 5; ++j) {
            op.ex[0][j] = r0[j];
            op.ex[1][j] = r1[j];
        }
        op.ex_sign = -1.0;
    } else if (kind == KIND_D2) {
        // Lele's sixth-order tridiagonal second derivative: alpha = 2/11,
        // a = 12/11, b = 3/11, right-hand side
        // a (f[i+1] - 2 f[i] + f[i-1]) + (b/4)(f[i+2] - 2 f[i] + f[i-2]) (times
        // h^2); wall rows (a reading: the paper gives none): one-sided
        // (2, -5, 4, -1) at rows 0 and N-1, central (1, -2, 1) at rows 1 and N-2
        op.nexp = 2;
        op.alpha = 2.0 / 11.0;
        const double a = 12.0 / 11.0, b = 3.0 / 11.0;
        op.rb[0] = -2.0 * a - 0.5 * b;
        op.rb[1] = a;
        op.rb[2] = 0.25 * b;
        op.rb[3] = 0.0;
        w = 2;
        const double r0[5] = {2.0, -5.0, 4.0, -1.0, 0.0};
        const double r1[5] = {1.0, -2.0, 1.0, 0.0, 0.0};
        for (int j = 0; j < 5; ++j) {
            op.ex[0][j] = r0[j];
            op.ex[1][j] = r1[j];
        }
        op.ex_sign = 1.0;
    } else {
        op.nexp = 3;
        op.alpha = alpha_f;
        const double af = alpha_f;
        op.rb[0] = (11.0 + 10.0 * af) / 16.0;
        op.rb[1] = 0.5 * (15.0 + 34.0 * af) / 32.0;
        op.rb[2] = 0.5 * (-3.0 + 6.0 * af) / 16.0;
        op.rb[3] = 0.5 * (1.0 - 2.0 * af) / 32.0;
        w = 3;
        for (int r = 0; r < 3; ++r) op.ex[r][r] = 1.0;
        op.ex_sign = 1.0;
    }
    fill_B(op, B);
    // partition and end rows
    std::vector<int> start(N + 2);
    op.nsub = partition_rule(N, sub_n, start.data());
    op.sub.assign((size_t)op.nsub * SUB_REC, 0);
    std::vector<double> y, crow(N);
    auto end_row = [&](int i, int &j0, int &len) {
        j0 = op.coef.size();  // placeholder
        if (is_explicit(op, i)) {
            // explicit rows are their own C rows
            int a = N, b = -1;
            for (int j = 0; j < N; ++j)
                if (B.at(i, j) != 0.0) {
                    a = j < a ? j : a;
                    b = j;
                }
            j0 = a;
            len = b - a + 1;
            for (int j = a; j <= b; ++j) op.coef.push_back(B.at(i, j));
            return;
        }
        solve_At(op, i, y);
        for (int j = 0; j < N; ++j) crow[j] = 0.0;
        for (int r = 0; r < N; ++r) {
            if (y[r] == 0.0) continue;
            for (int k = 0; k < 7; ++k) {
                int c = B.c0[r] + k;
                if (c >= 0 && c < N) crow[c] += y[r] * B.w[(size_t)r * 7 + k];
            }
        }
        int a = N, b = -1;
        for (int j = 0; j < N; ++j)
            if (fabs(crow[j]) >= thresh) {
                a = j < a ? j : a;
                b = j;
            }
        if (b < a) {
            a = i;
            b = i;
        }
        j0 = a;
        len = b - a + 1;
        for (int j = a; j <= b; ++j) op.coef.push_back(fabs(crow[j]) >= thresh ? crow[j] : 0.0);
    };
    for (int b = 0; b < op.nsub; ++b) {
        int *rec = &op.sub[(size_t)b * SUB_REC];
        int s = start[b], e = start[b + 1] - 1;
        rec[0] = s;
        rec[1] = e;
        int j0, len;
        rec[6] = (int)op.coef.size();
        end_row(s, j0, len);
        rec[4] = j0;
        rec[5] = len;
        if (e != s) {
            rec[9] = (int)op.coef.size();
            end_row(e, j0, len);
            rec[7] = j0;
            rec[8] = len;
        } else {
            rec[7] = rec[4];
            rec[8] = 0;
            rec[9] = rec[6];
        }
        int lo = s + 1 > op.nexp ? s + 1 : op.nexp;
        int hi = e - 1 < N - 1 - op.nexp ? e - 1 : N - 1 - op.nexp;
        rec[10] = lo;
        rec[11] = hi;
        // rows the solve reads (window) and rows the block must stage (the
        // window plus the end-row supports)
        int wlo = s, whi = e;
        auto cover_w = [&](int a, int c) {
            if (a < wlo) wlo = a;
            if (c > whi) whi = c;
        };
        if (lo <= hi) cover_w(lo - w, hi + w);
        for (int r = 0; r < op.nexp; ++r) {
            if (r > s && r < e) cover_w(0, 4 < N - 1 ? 4 : N - 1);
            if (N - 1 - r > s && N - 1 - r < e) cover_w(N - 5 > 0 ? N - 5 : 0, N - 1);
        }
        if (wlo < 0) wlo = 0;
        if (whi > N - 1) whi = N - 1;
        int tlo = wlo, thi = whi;
        auto cover = [&](int a, int c) {
            if (a < tlo) tlo = a;
            if (c > thi) thi = c;
        };
        cover(rec[4], rec[4] + rec[5] - 1);
        if (rec[8] > 0) cover(rec[7], rec[7] + rec[8] - 1);
        if (tlo < 0) tlo = 0;
        if (thi > N - 1) thi = N - 1;
        rec[2] = tlo;
        rec[3] = thi;
        rec[12] = wlo;
        rec[13] = whi;
        int m = hi - lo + 1;
        if (m > op.maxm) op.maxm = m;
        if (thi - tlo + 1 > op.max_tile) op.max_tile = thi - tlo + 1;
        if (whi - wlo + 1 > op.max_win) op.max_win = whi - wlo + 1;
    }
    // Thomas factors for a run of implicit rows after a known value
    int mm = op.maxm > 0 ? op.maxm : 1;
    op.cp.assign(mm, 0.0);
    op.inv.assign(mm, 0.0);
    for (int r = 0; r < mm; ++r) {
        double den = r == 0 ? 1.0 : 1.0 - op.alpha * op.cp[r - 1];
        op.inv[r] = 1.0 / den;
        op.cp[r] = op.alpha * op.inv[r];
    }
    // The factors converge geometrically to the root of alpha c^2 - c + alpha = 0.
    // Past kconv they equal the last tabulated value in that precision, so the
    // kernels keep only the first kconv entries and a register limit.
    op.kconv64 = mm;
    while (op.kconv64 > 1 && op.cp[op.kconv64 - 2] == op.cp[mm - 1] && op.inv[op.kconv64 - 2] == op.inv[mm - 1])
        --op.kconv64;
    op.kconv32 = mm;
    while (op.kconv32 > 1 && (float)op.cp[op.kconv32 - 2] == (float)op.cp[mm - 1] &&
           (float)op.inv[op.kconv32 - 2] == (float)op.inv[mm - 1])
        --op.kconv32;
    for (int b = 0; b < op.nsub; ++b) {
        const int *rec = &op.sub[(size_t)b * SUB_REC];
        op.max_taps = rec[5] > op.max_taps ? rec[5] : op.max_taps;
        op.max_taps = rec[8] > op.max_taps ? rec[8] : op.max_taps;
    }
    return true;
}

void apply_line_host(const LineOpHost &op, const double *f, double *g)
{
    const int N = op.N;
    const double al = op.alpha;
    auto explicit_row = [&](int i) {
        double acc = 0.0;
        if (i < op.nexp) {
            for (int j = 0; j < 5 && j < N; ++j) acc += op.ex[i][j] * f[j];
        } else {
            const int r = N - 1 - i;
            for (int j = 0; j < 5 && j < N; ++j) acc += op.ex_sign * op.ex[r][j] * f[N - 1 - j];
        }
        return acc;
    };
    std::vector<double> dp;
    for (int b = 0; b < op.nsub; ++b) {
        const int *rec = &op.sub[(size_t)b * SUB_REC];
        const int s = rec[0], e = rec[1], lo = rec[10], hi = rec[11];
        double gs = 0.0, ge = 0.0;
        for (int k = 0; k < rec[5]; ++k) gs += op.coef[rec[6] + k] * f[rec[4] + k];
        for (int k = 0; k < rec[8]; ++k) ge += op.coef[rec[9] + k] * f[rec[7] + k];
        for (int i = s + 1; i < e; ++i)
            if (i < op.nexp || i > N - 1 - op.nexp) g[i] = explicit_row(i);
        if (lo <= hi) {
            const int m = hi - lo + 1;
            const double gL = lo == s + 1 ? gs : g[op.nexp - 1];
            const double gR = hi == e - 1 ? ge : g[N - op.nexp];
            dp.assign(m, 0.0);
            for (int r = 0; r < m; ++r) {
                const int i = lo + r;
                double rhs;
                if (op.kind == KIND_DERIV)
                    rhs = op.rb[0] * (f[i + 1] - f[i - 1]) + op.rb[1] * (f[i + 2] - f[i - 2]);
                else if (op.kind == KIND_D2)
                    rhs = op.rb[0] * f[i] + op.rb[1] * (f[i + 1] + f[i - 1]) + op.rb[2] * (f[i + 2] + f[i - 2]);
                else
                    rhs = op.rb[0] * f[i] + op.rb[1] * (f[i + 1] + f[i - 1]) + op.rb[2] * (f[i + 2] + f[i - 2]) +
                          op.rb[3] * (f[i + 3] + f[i - 3]);
                if (r == 0) rhs -= al * gL;
                if (r == m - 1) rhs -= al * gR;
                dp[r] = (rhs - al * (r ? dp[r - 1] : 0.0)) * op.inv[r];
            }
            double x = dp[m - 1];
            g[hi] = x;
            for (int r = m - 2; r >= 0; --r) {
                x = dp[r] - op.cp[r] * x;
                g[lo + r] = x;
            }
        }
        g[s] = gs;
        if (rec[8] > 0) g[e] = ge;
    }
}

void build_dense_blocks(const LineOpHost &op, DenseHost &out)
{
    out = DenseHost();
    out.N = op.N;
    out.nsub = op.nsub;
    out.rec.assign((size_t)op.nsub * DENSE_REC, 0);
    const int N = op.N;
    std::vector<double> f(N, 0.0), g(N, 0.0);
    // nearest TF32 value (ties away from zero), as cvt.rna.tf32.f32
    auto tf32 = [](float x) {
        unsigned u;
        memcpy(&u, &x, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;
        float y;
        memcpy(&y, &u, 4);
        return y;
    };
    // nearest BF16 value (ties to even): its bit pattern and its value
    auto bf16 = [](double x, uint16_t &bits) {
        const float xf = (float)x;
        unsigned u;
        memcpy(&u, &xf, 4);
        u += 0x7FFFu + ((u >> 16) & 1u);
        bits = (uint16_t)(u >> 16);
        const unsigned v = (unsigned)bits << 16;
        float y;
        memcpy(&y, &v, 4);
        return (double)y;
    };
    for (int b = 0; b < op.nsub; ++b) {
        const int *rec = &op.sub[(size_t)b * SUB_REC];
        const int s = rec[0], e = rec[1], tlo = rec[2], thi = rec[3];
        const int nb = e - s + 1, K = thi - tlo + 1;
        const int npad = (nb + 15) / 16 * 16, kpad = (K + 7) / 8 * 8, kpad16 = (K + 15) / 16 * 16;
        int *r = &out.rec[(size_t)b * DENSE_REC];
        r[0] = s;
        r[1] = nb;
        r[2] = npad;
        r[3] = kpad;
        r[4] = tlo;
        r[5] = (int)out.hi.size();
        r[6] = kpad16;
        r[7] = (int)out.b16[0].size();
        out.max_npad = npad > out.max_npad ? npad : out.max_npad;
        out.max_kpad = kpad > out.max_kpad ? kpad : out.max_kpad;
        out.max_kpad16 = kpad16 > out.max_kpad16 ? kpad16 : out.max_kpad16;
        const size_t base = out.hi.size(), base16 = out.b16[0].size();
        out.hi.resize(base + (size_t)npad * kpad, 0.0f);
        out.lo.resize(base + (size_t)npad * kpad, 0.0f);
        for (auto &v : out.b16) v.resize(base16 + (size_t)npad * kpad16, 0);
        for (int k = 0; k < K; ++k) {
            std::fill(f.begin(), f.end(), 0.0);
            f[tlo + k] = 1.0;
            apply_line_host(op, f.data(), g.data());
            for (int n = 0; n < nb; ++n) {
                const double d = g[s + n];
                const float h = tf32((float)d);
                const float l = tf32((float)(d - (double)h));
                const size_t o = base + (size_t)(n / 8) * (kpad / 4) * 32 + (size_t)(k / 4) * 32 + (n % 8) * 4 + (k % 4);
                out.hi[o] = h;
                out.lo[o] = l;
                // three BF16 parts, each of what the earlier ones leave
                const size_t o16 =
                    base16 + (size_t)(n / 8) * (kpad16 / 8) * 64 + (size_t)(k / 8) * 64 + (n % 8) * 8 + (k % 8);
                double rest = d;
                for (int q = 0; q < 3; ++q) rest -= bf16(rest, out.b16[q][o16]);
            }
        }
    }
}

cudaError_t LineOpBuf::upload()
{
    release();
    const LineOpHost &h = host;
    size_t nsub_b = h.sub.size() * sizeof(int);
    size_t nc = h.coef.size() > 0 ? h.coef.size() : 1;
    size_t nm = h.cp.size();
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o_sub = 0, o_c64 = al(nsub_b), o_c32 = o_c64 + al(nc * 8), o_cp64 = o_c32 + al(nc * 4),
           o_inv64 = o_cp64 + al(nm * 8), o_cp32 = o_inv64 + al(nm * 8), o_inv32 = o_cp32 + al(nm * 4),
           tot = o_inv32 + al(nm * 4);
    cudaError_t e = dev_alloc(&mem, tot);
    if (e != cudaSuccess) {
        mem = nullptr;
        return e;
    }
    std::vector<char> stage(tot, 0);
    memcpy(stage.data() + o_sub, h.sub.data(), nsub_b);
    for (size_t i = 0; i < h.coef.size(); ++i) {
        ((double *)(stage.data() + o_c64))[i] = h.coef[i];
        ((float *)(stage.data() + o_c32))[i] = (float)h.coef[i];
    }
    for (size_t i = 0; i < nm; ++i) {
        ((double *)(stage.data() + o_cp64))[i] = h.cp[i];
        ((double *)(stage.data() + o_inv64))[i] = h.inv[i];
        ((float *)(stage.data() + o_cp32))[i] = (float)h.cp[i];
        ((float *)(stage.data() + o_inv32))[i] = (float)h.inv[i];
    }
    e = cudaMemcpy(mem, stage.data(), tot, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    char *b = (char *)mem;
    dev.N = h.N;
    dev.nsub = h.nsub;
    dev.nexp = h.nexp;
    dev.maxm = h.maxm;
    dev.max_tile = h.max_tile;
    dev.max_win = h.max_win;
    dev.max_taps = h.max_taps;
    dev.kconv64 = h.kconv64;
    dev.kconv32 = h.kconv32;
    dev.ncoef = (int)h.coef.size();
    // Whole-line x sweep (line_kernels.cu): a block holds L lines of 1 or 5
    // fields, [field][line][row] with one pad word per 32 rows, and thread c
    // solves sub-domain c % nsub of line (c / nsub) % L, field c / (nsub L).
    // Pick, from 32 candidates, the line pitch that puts the first rows of a
    // warp's columns in the fewest shared-memory bank collisions.
    {
        auto xrow = [](int g) { return g + (g >> 5); };
        const int base = xrow(h.N - 1) + 1;
        for (int fi = 0; fi < 2; ++fi) {
            const int nf = fi ? 5 : 1;
            for (int L = 1; L <= 4; ++L) {
                const int cols = h.nsub * nf * L;
                int best = base, best_score = 1 << 30;
                for (int d = 0; d < 32; ++d) {
                    const int ls = base + d;
                    int score = 0;
                    for (int w = 0; w * 32 < cols; ++w) {
                        for (int k : {0, 17}) {
                            int cnt[32] = {0};
                            int mx = 0;
                            for (int c = 32 * w; c < cols && c < 32 * w + 32; ++c) {
                                const int b = c % h.nsub, l = (c / h.nsub) % L, f = c / (h.nsub * L);
                                const int sb = h.sub[(size_t)b * SUB_REC];
                                const long long addr = (long long)f * L * ls + (long long)l * ls + xrow(sb + k);
                                const int bank = (int)(addr % 32);
                                if (++cnt[bank] > mx) mx = cnt[bank];
                            }
                            score += mx;
                        }
                    }
                    if (score < best_score) {
                        best_score = score;
                        best = ls;
                    }
                }
                dev.xpitch[fi][L - 1] = best;
            }
        }
    }
    dev.cpL = h.cp.back();
    dev.invL = h.inv.back();
    dev.alpha = h.alpha;
    for (int i = 0; i < 4; ++i) dev.rb[i] = h.rb[i];
    memcpy(dev.ex, h.ex, sizeof(dev.ex));
    dev.ex_sign = h.ex_sign;
    dev.sub = (const int *)(b + o_sub);
    dev.coef64 = (const double *)(b + o_c64);
    dev.coef32 = (const float *)(b + o_c32);
    dev.cp64 = (const double *)(b + o_cp64);
    dev.inv64 = (const double *)(b + o_inv64);
    dev.cp32 = (const float *)(b + o_cp32);
    dev.inv32 = (const float *)(b + o_inv32);
    return cudaSuccess;
}

void LineOpBuf::release()
{
    if (mem) dev_free(mem);
    mem = nullptr;
}



// Banded explicit form (the equivalent explicit scheme applied at every row):
// all rows of the global C = A^-1 B, truncated at thresh.  Rows far enough
// from both walls equal one translation-invariant stencil (to within thresh);
// the rest are tabulated with their own windows.
bool build_band_op(int N, int kind, double alpha_f, double thresh, BandHost &bh, std::string &msg)
{
    LineOpHost op;
    if (!build_line_op(N, 0, kind, alpha_f, thresh, op, msg)) return false;
    Banded B;
    B.N = N;
    B.c0.assign(N, 0);
    B.w.assign((size_t)N * 7, 0.0);
    fill_B(op, B);
    std::vector<std::vector<double>> C(N);
    std::vector<double> y;
    std::vector<int> lo(N), hi(N);
    for (int i = 0; i < N; ++i) {
        global_C_row(op, B, i, y, C[i]);
        lo[i] = N;
        hi[i] = -1;
        for (int j = 0; j < N; ++j) {
            if (fabs(C[i][j]) < thresh) {
                C[i][j] = 0.0;
            } else {
                lo[i] = j < lo[i] ? j : lo[i];
                hi[i] = j;
            }
        }
        if (hi[i] < lo[i]) lo[i] = hi[i] = i;
    }
    bh = BandHost();
    bh.N = N;
    bh.kind = kind;
    // interior stencil from the middle row
    const int im = N / 2;
    int h = im - lo[im] > hi[im] - im ? im - lo[im] : hi[im] - im;
    bh.h = h;
    bh.stencil.assign(2 * h + 1, 0.0);
    for (int k = -h; k <= h; ++k)
        if (im + k >= 0 && im + k < N) bh.stencil[k + h] = C[im][im + k];
    auto matches = [&](int i) {
        if (i - h < 0 || i + h > N - 1 || lo[i] < i - h || hi[i] > i + h) return false;
        for (int k = -h; k <= h; ++k)
            if (fabs(C[i][i + k] - bh.stencil[k + h]) > thresh) return false;
        return true;
    };
    // the interior run around the middle row
    int a = im, b = im;
    if (matches(im)) {
        while (a - 1 >= 0 && matches(a - 1)) --a;
        while (b + 1 < N && matches(b + 1)) ++b;
        bh.in_lo = a;
        bh.in_hi = b;
    } else {
        bh.in_lo = N;  // no interior rows: every row is tabulated
        bh.in_hi = N - 1;
    }
    // tabulated rows: 0 .. in_lo-1 and in_hi+1 .. N-1
    int W = 1;
    for (int i = 0; i < N; ++i)
        if (i < bh.in_lo || i > bh.in_hi) W = hi[i] - lo[i] + 1 > W ? hi[i] - lo[i] + 1 : W;
    bh.W = W;
    bh.wrow.clear();
    bh.wj0.clear();
    bh.wlen.clear();
    bh.wtap.clear();
    for (int i = 0; i < N; ++i) {
        if (i >= bh.in_lo && i <= bh.in_hi) continue;
        bh.wrow.push_back(i);
        bh.wj0.push_back(lo[i]);
        bh.wlen.push_back(hi[i] - lo[i] + 1);
        for (int k = 0; k < W; ++k) bh.wtap.push_back(lo[i] + k <= hi[i] ? C[i][lo[i] + k] : 0.0);
    }
    return true;
}

// out = C_band f on one line (host, FP64 taps): the banded form's arithmetic
// in the order the kernel sums it (interior stencil from -h to h, tabulated
// rows over their windows)
void apply_band_host(const BandHost &bh, const double *f, double *g)
{
    const int N = bh.N, h = bh.h;
    for (int i = bh.in_lo; i <= bh.in_hi && i < N; ++i) {
        double acc = 0.0;
        for (int k = -h; k <= h; ++k) acc += bh.stencil[k + h] * f[i + k];
        g[i] = acc;
    }
    for (size_t t = 0; t < bh.wrow.size(); ++t) {
        double acc = 0.0;
        for (int k = 0; k < bh.wlen[t]; ++k) acc += bh.wtap[t * bh.W + k] * f[bh.wj0[t] + k];
        g[bh.wrow[t]] = acc;
    }
}

}  // namespace nopcs

using namespace nopcs;

extern "C" nopcs_status nopcs_band_apply(int N, int kind, double alpha_f, double thresh, const double *f, double *g,
                                         int *half_width, int *interior_lo, int *interior_hi)
{
    if (kind != KIND_DERIV && kind != KIND_FILTER && kind != KIND_D2) return NOPCS_EINVAL;
    if (!f || !g) return NOPCS_EINVAL;
    BandHost bh;
    std::string msg;
    if (!build_band_op(N, kind, alpha_f, thresh, bh, msg)) return NOPCS_EINVAL;
    apply_band_host(bh, f, g);
    if (half_width) *half_width = bh.h;
    if (interior_lo) *interior_lo = bh.in_lo;
    if (interior_hi) *interior_hi = bh.in_hi;
    return NOPCS_OK;
}

extern "C" nopcs_status nopcs_operator_rows(int N, int sub_n, int kind, double alpha_f, double thresh,
                                            int *nsub, int *starts, int *end_j0, int *end_len,
                                            double *coef, int max_coef)
{
    if (kind != KIND_DERIV && kind != KIND_FILTER && kind != KIND_D2) return NOPCS_EINVAL;
    LineOpHost op;
    std::string msg;
    if (!build_line_op(N, sub_n, kind, alpha_f, thresh, op, msg)) return NOPCS_EINVAL;
    if ((int)op.coef.size() > max_coef) return NOPCS_EINVAL;
    if (nsub) *nsub = op.nsub;
    for (int b = 0; b < op.nsub; ++b) {
        const int *rec = &op.sub[(size_t)b * SUB_REC];
        if (starts) starts[b] = rec[0];
        if (end_j0) {
            end_j0[2 * b] = rec[4];
            end_j0[2 * b + 1] = rec[7];
        }
        if (end_len) {
            end_len[2 * b] = rec[5];
            end_len[2 * b + 1] = rec[8];
        }
    }
    if (starts) starts[op.nsub] = N;
    if (coef)
        for (size_t i = 0; i < op.coef.size(); ++i) coef[i] = op.coef[i];
    return NOPCS_OK;
}

extern "C" nopcs_status nopcs_operator_apply(int N, int sub_n, int kind, double alpha_f, double thresh,
                                             const double *f, double *g)
{
    if (kind != KIND_DERIV && kind != KIND_FILTER && kind != KIND_D2) return NOPCS_EINVAL;
    if (!f || !g) return NOPCS_EINVAL;
    LineOpHost op;
    std::string msg;
    if (!build_line_op(N, sub_n, kind, alpha_f, thresh, op, msg)) return NOPCS_EINVAL;
    apply_line_host(op, f, g);
    return NOPCS_OK;
}
