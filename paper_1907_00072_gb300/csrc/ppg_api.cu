// ppg_api.cu -- the C ABI (include/ppg.h) and the solver driver of the GB300 PP-GMRES library.
//
// Host-side orchestration only: every arithmetic step of the method runs in the
// library's kernels (ppg_spmv.cu, ppg_ortho.cu, ppg_small.cu).  The driver keeps
// the iteration state on the device (ppg::Cycle), so an iteration is a fixed
// sequence of launches that reads the iteration index from device memory; the host
// only enqueues and, once per restart cycle, reads back a few bytes of status.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <stdlib.h>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ppg.h"
#include "ppg_internal.h"

using namespace ppg;

namespace {

thread_local std::string g_last_error;

ppg_status fail(ppg_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
ppg_status fail(ppg_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define PPG_CK(call)                                                                                      \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? PPG_ERR_OOM : PPG_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                      \
    } while (0)

#define PPG_TRY(expr)                     \
    do {                                  \
        ppg_status s_ = (expr);           \
        if (s_ < 0) return s_;            \
    } while (0)

constexpr int kNumVecs = 8;  // working vectors in the workspace

// Number of bytes of Cycle read back by the host (everything before the arrays).
constexpr size_t kCycleHeader = offsetof(Cycle, sigma);

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

constexpr int kMaxRounds = 4096;  // rounds of the two-step kernel's persistent grid

}  // namespace

struct ppg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    DevMatrix A{};
    int *d_rowptr = nullptr;
    int *d_colidx = nullptr;
    short *d_coloff = nullptr;
    double *d_vals = nullptr;
    float *d_vals32 = nullptr;
    int *d_sptr = nullptr;       // sliced ELL copy (DevMatrix::sptr ...)
    short *d_soff = nullptr;
    int *d_scol = nullptr;
    double *d_svals64 = nullptr;
    float *d_svals32 = nullptr;
    int *d_rounds = nullptr;     // two-step chain kernel: kMaxRounds round counters, a ticket, 8 diagnostics
    int *d_twin = nullptr;       // x windows per tile (DevMatrix::twin)
    short *d_lidx = nullptr;     // window-buffer index per entry (DevMatrix::lidx)
    float *d_evals = nullptr;    // tile-ELL copy (DevMatrix::evals, eidx, toff)
    short *d_eidx = nullptr;
    int *d_toff = nullptr;
    int *d_etwin = nullptr;
    double *d_evals64 = nullptr;
    int fuse = 0;                // pair consecutive links of the p(A) chain into one launch (measured slower)
    int spmv_alternate = 1;      // consecutive tile-ELL links visit their tiles in opposite orders
    unsigned long long spmv_links = 0;
    int gs_alternate = 1;        // Gram-Schmidt pass 2 visits its tiles in the opposite order of passes 1, 3
    WaitCfg waits;               // limits of the software waits (set per solve from ppg_opts)
    // ILU(0) on the left (ppg_set_left_ilu0): factors on A's pattern, the rows of each triangle sorted
    // by level, the triangular solves' abort word, and five vectors of ld doubles (the SpMV's result and
    // the two solves' outputs of a composed link, which also mark their rows ready; a residual and its
    // M^{-1} image)
    int ilu_on = 0;
    double *d_lu64 = nullptr;
    float *d_lu32 = nullptr;
    int *d_ilu_diag = nullptr, *d_lorder = nullptr, *d_uorder = nullptr;
    double *d_ilu_rd64 = nullptr;  // 1 / u_ii (the upper solve multiplies by it)
    float *d_ilu_rd32 = nullptr;
    int ilu_red = 32;              // lanes a row's sum is reduced over: a power of two >= the longest row
    int *d_ilu_abort = nullptr;
    char *ilu_vec = nullptr;
    char *noalloc_base = nullptr; // device address of the allocation-free apply's scratch (n <= its limit)
    // s-step solves (ppg_opts.sstep): the block's device state and the passes' per-CTA sums, allocated
    // on the first such solve
    SStep *d_sstep = nullptr;
    double *d_bgs_partials = nullptr;
    int bgs_pld = 0;

    // CUDA graphs of single iterations (ppg_opts.use_graph): one per iteration index, precision and
    // polynomial presence, valid while the signature captured with it (workspace addresses,
    // storage format, pairing, the polynomial itself) is unchanged
    struct IterGraph {
        cudaGraphExec_t exec = nullptr;
        long long launches = 0;
        std::vector<double> sig;
    };
    std::vector<IterGraph> igraphs;
    cudaStream_t cap_stream = nullptr;  // private stream the graphs are captured on
    bool graphs_broken = false;         // capture failed once: launch directly from then on
    long long ld = 0;  // padded vector length

    // polynomial (host copy; coefficients enter kernels as launch arguments)
    int has_poly = 0;
    int basis = PPG_BASIS_POWER;
    int degree = 0;
    std::vector<double> coef;   // power: degree + 1
    std::vector<double> roots;  // roots: 2 (degree + 1) (re, im)
    std::vector<double> table;  // roots: 2 (degree + 1) per-step coefficients
    double poly_resid = NAN;

    Cycle *st = nullptr;      // device state
    Cycle *h_st = nullptr;    // pinned host mirror (header)
    double *d_small = nullptr;  // 4 * kKmax doubles: construction outputs
    int *d_info = nullptr;      // 16 ints
    int *h_info = nullptr;      // pinned
    double *h_small = nullptr;  // pinned, 4 * kKmax
    int *h_prog = nullptr;      // pinned, mapped: the device's progress word (Cycle::prog)
    int *d_prog = nullptr;      // its device address

    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = true;

    ppg_ctx *tctx = nullptr;  // transposed matrix (adjoint)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    long long launches = 0;

    // profiling (ppg_opts.profile): an event pair around every SpMV / Gram-Schmidt launch
    struct ProfRec {
        int cls;  // 0 SpMV, 1 Gram-Schmidt
        cudaEvent_t a, b;
        double bytes;    // algorithmic bytes (Gram-Schmidt: per basis column in kcol_bytes)
        double kcol_bytes;
        int j;           // iteration index of the launch within its cycle, -2 at the cycle end
        int valid;
    };
    bool prof = false;
    bool prof_open = false;
    int prof_j = -1;
    std::vector<ProfRec> recs;
    size_t rec_first = 0;  // first record of the current cycle
    std::vector<cudaEvent_t> evpool;
    size_t evnext = 0;
};

namespace {

// ---------------------------------------------------------------- workspace

struct Layout {
    double *partials;
    int partial_blocks;  // capacity in CTAs for (kKmax + 1) columns
    char *basis;         // ncols columns of ld elements
    int ncols;
    char *vec[kNumVecs];  // working vectors of ld elements
    size_t esize;
    char *zbasis;  // float32 layouts: the preconditioned basis Z (ncols - 1 columns) of flexible solves,
                   // in the half of the float64-sized region that float32 columns leave free
};

size_t partial_doubles(const ppg_ctx *c)
{
    const size_t gs = (size_t)(kKmax + 1) * (size_t)gs_max_blocks(c->num_sms);
    const size_t gram = (size_t)(kSmallMax * (kSmallMax + 1) / 2) * (size_t)gram_grid(c->num_sms);
    const size_t resid = (size_t)c->A.resid_blocks;
    return std::max(gs, std::max(gram, resid));
}

size_t layout_bytes(const ppg_ctx *c, int ncols)
{
    const size_t p = round_up((long long)(partial_doubles(c) * sizeof(double)), 4096);
    return p + (size_t)(ncols + kNumVecs) * (size_t)c->ld * sizeof(double);
}

ppg_status get_layout(ppg_ctx *c, int ncols, size_t esize, Layout *L)
{
    const size_t need = layout_bytes(c, ncols);
    if (need > c->ws_bytes) {
        if (!c->ws_owned)
            return fail(PPG_ERR_OOM, "workspace of %zu bytes is smaller than the %zu bytes needed", c->ws_bytes,
                        need);
        if (c->ws) cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
        PPG_CK(cudaMalloc(&c->ws, need));
        c->ws_bytes = need;
    }
    const size_t p = round_up((long long)(partial_doubles(c) * sizeof(double)), 4096);
    L->partials = reinterpret_cast<double *>(c->ws);
    L->partial_blocks = gs_max_blocks(c->num_sms);
    L->basis = c->ws + p;
    L->ncols = ncols;
    L->esize = esize;
    for (int i = 0; i < kNumVecs; ++i) L->vec[i] = L->basis + (size_t)(ncols + i) * c->ld * esize;
    // (ncols + kNumVecs) float64 columns hold, in float32, the basis, the vectors and Z
    L->zbasis = esize == sizeof(float) ? L->basis + (size_t)(ncols + kNumVecs) * c->ld * esize : nullptr;
    const int zcols = L->zbasis ? ncols - 1 : 0;
    // rows n..ld-1 of every column and vector must read as zero
    if (c->ld > c->A.n) {
        PPG_CK(cudaMemset2DAsync(L->basis + (size_t)c->A.n * esize, c->ld * esize, 0, (c->ld - c->A.n) * esize,
                                 ncols + kNumVecs + zcols, c->stream));
    }
    return PPG_OK;
}

// L2 residency of the float32 matrix blocks (off unless PPG_L2_PERSIST=1 in the environment): each
// link of a p(A) chain reads the same blocks, so keeping them in L2 between launches would leave only
// the vectors to come from HBM.  The process's persisting-L2 set-aside (a limit of this CUDA context,
// released with it) is raised to cover the window when the device allows.  Measured on the 128^3
// stencil (84.7 MB set-aside for an 87.5 MB window): the SpMV chain of a solve took 13.9 ms against
// 12.0 ms without it, so it stays off.
void l2_residency(ppg_ctx *c, const void *base, size_t bytes)
{
    c->A.l2_base = base;
    c->A.l2_bytes = 0;
    c->A.l2_hit = 0.f;
    const char *env = getenv("PPG_L2_PERSIST");
    if (!env || atoi(env) != 1) return;
    int maxp = 0, maxw = 0;
    if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, c->device) != cudaSuccess || maxp <= 0 ||
        maxw <= 0) {
        cudaGetLastError();
        return;
    }
    const size_t win = std::min(bytes, (size_t)maxw);
    size_t cur = 0;
    cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    const size_t want = std::min(win, (size_t)maxp);
    if (cur < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    c->A.l2_bytes = win;
    c->A.l2_hit = (float)std::min(1.0, (double)cur / (double)win);
}

ppg_status ensure_f32(ppg_ctx *c)
{
    if (c->d_vals32) return PPG_OK;
    PPG_CK(cudaMalloc(&c->d_vals32, (size_t)(c->A.nnz + 8) * sizeof(float)));
    PPG_CK(cudaMemsetAsync(c->d_vals32, 0, (size_t)(c->A.nnz + 8) * sizeof(float), c->stream));
    if (c->A.nnz > 0) PPG_CK(launch_cast_f32(c->d_vals, c->d_vals32, c->A.nnz, c->stream));
    c->A.vals32 = c->d_vals32;
    if (c->A.nslices > 0) {
        PPG_CK(cudaMalloc(&c->d_svals32, (size_t)c->A.spadded * sizeof(float)));
        PPG_CK(launch_cast_f32(c->d_svals64, c->d_svals32, c->A.spadded, c->stream));
        c->A.svals32 = c->d_svals32;
    }
    return PPG_OK;
}

// ---------------------------------------------------------------- operand helpers

VecRef vfix(const void *p) { return VecRef{p, 0, 0, 0}; }
VecRef vcol(const void *base, long long ld, int off) { return VecRef{base, ld, off, 1}; }
VecRef vnone() { return VecRef{nullptr, 0, 0, 0}; }
Scalar simm(double v) { return Scalar{v, nullptr, 0, 0, nullptr, 0, 0}; }
// v * sigma[j] (sigma follows the iteration index) when sig is set
Scalar sscaled(double v, const double *sig) { return Scalar{v, sig, 0, sig ? 1 : 0, nullptr, 0, 0}; }

SpmvEpi epi_none()
{
    SpmvEpi e;
    e.x = e.x2 = vnone();
    e.out0 = e.u0 = e.w0 = e.out1 = e.u1 = e.w1 = vnone();
    e.a0 = e.b0 = e.c0 = e.a1 = e.b1 = e.c1 = e.s2 = simm(0.0);
    e.rev = 0;
    return e;
}

// ---------------------------------------------------------------- profiling helpers

cudaEvent_t prof_event(ppg_ctx *c)
{
    if (c->evnext == c->evpool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->evpool.push_back(e);
    }
    return c->evpool[c->evnext++];
}

// Profiling works on segments: runs of consecutive launches of one class (the SpMV chain of an
// iteration, its three Gram-Schmidt passes, ...) enqueued back to back.  One event pair brackets
// each segment, so the measured time is the device time of those launches without per-launch
// event overhead; each launch adds its algorithmic bytes to the open segment.
void prof_open(ppg_ctx *c, cudaStream_t s, int cls)
{
    if (!c->prof) return;
    cudaEvent_t a = prof_event(c);
    if (!a) return;
    cudaEventRecord(a, s);
    c->recs.push_back(ppg_ctx::ProfRec{cls, a, nullptr, 0.0, 0.0, c->prof_j, 1});
    c->prof_open = true;
}

void prof_close(ppg_ctx *c, cudaStream_t s)
{
    if (!c->prof || !c->prof_open) return;
    c->prof_open = false;
    cudaEvent_t b = prof_event(c);
    if (!b) {
        c->recs.pop_back();
        return;
    }
    cudaEventRecord(b, s);
    c->recs.back().b = b;
}

void prof_add(ppg_ctx *c, double bytes, double kcol_bytes)
{
    if (!c->prof || !c->prof_open) return;
    c->recs.back().bytes += bytes;
    c->recs.back().kcol_bytes += kcol_bytes;
}

bool same_vec(const VecRef &u, const VecRef &v)
{
    return u.base == v.base && u.ld == v.ld && u.col == v.col && u.follow == v.follow;
}

// Algorithmic bytes of one SpMV launch: values and column indices once in the stored format
// (row-block CSR: int16 offsets or int32 indices plus row pointers; sliced ELL: the padded
// entries plus slice offsets), each distinct vector read once and each output written once.
double spmv_bytes(const DevMatrix &A, int prec, const SpmvEpi &e)
{
    const double es = prec == kF64 ? 8.0 : 4.0;
    double b;
    if (A.format == kFmtSell && A.nslices > 0)
        b = (double)A.spadded * (es + (A.soff ? 2.0 : 4.0)) + 4.0 * (A.nslices + 1.0);
    else
        b = (double)A.nnz * (es + (A.coloff ? 2.0 : 4.0)) + 4.0 * (A.n + 1.0);
    const VecRef *reads[6] = {&e.x, &e.x2, &e.u0, &e.w0, &e.u1, &e.w1};
    int distinct = 0;
    for (int i = 0; i < 6; ++i) {
        if (!reads[i]->base) continue;
        bool seen = false;
        for (int q = 0; q < i; ++q) seen = seen || (reads[q]->base && same_vec(*reads[q], *reads[i]));
        if (!seen) ++distinct;
    }
    const int writes = (e.out0.base ? 1 : 0) + (e.out1.base ? 1 : 0);
    return b + (double)A.n * es * (distinct + writes);
}

// The two-step chain kernel applies to the row-block CSR kernel when the matrix bandwidth spans at
// most as many tiles as its persistent grid has CTAs (and the rounds fit the counters).
bool chain_pairs(const DevMatrix &A, int prec, bool have_counters)
{
    if (!have_counters || A.format != kFmtCsr || A.n <= 0) return false;
    const long long R = A.rows_per_tile;
    const long long ntiles = (A.n + R - 1) / R;
    long long grid = prec == kF64 ? A.spmv2_blocks64 : A.spmv2_blocks32;
    if (grid > ntiles) grid = ntiles;
    const long long halo = ((long long)A.bw + R - 1) / R;
    return grid > 0 && halo <= grid && (ntiles + grid - 1) / grid <= kMaxRounds;
}

struct Exec {
    ppg_ctx *c;
    const DevMatrix *A;
    int prec;
    cudaStream_t s;
    bool plain = false;  // y = A x even when ILU(0) is on (ppg_spmv)

    // Links of a p(A) chain are issued through spmv(); inside a chain (depth > 0) each link is held
    // back one call so that two consecutive links can share one launch (launch_spmv2).
    int chain_depth = 0;
    bool has_pending = false;
    SpmvEpi pending;
    int pending_check = 0;

    ppg_status launch_one(const SpmvEpi &e, int check)
    {
        if (c->ilu_on && !plain) return launch_ilu_link(e, check);
        c->launches++;
        SpmvEpi ed = e;
        if (c->spmv_alternate) ed.rev = (int)(c->spmv_links++ & 1);
        PPG_CK(launch_spmv(*A, prec, ed, c->st, check, s));
        prof_add(c, spmv_bytes(*A, prec, e), 0.0);
        return PPG_OK;
    }

    // One link with ILU(0) on the left (Section VI): the link's A becomes B = M^{-1} A = U^{-1} L^{-1} A:
    // t1 = A (x + s2 x2), t2 = L^{-1} t1, then U^{-1} t2 with the link's epilogue applied to it.
    char *ilu_v(int q) const { return c->ilu_vec + (size_t)q * c->ld * sizeof(double); }
    ppg_status ilu_solve(bool lower, VecRef x, void *y, const SpmvEpi &epi, int check)
    {
        IluSolveArgs a{};
        a.n = A->n;
        a.rp = c->d_rowptr;
        a.ci = c->d_colidx;
        a.lu = prec == kF64 ? (const void *)c->d_lu64 : (const void *)c->d_lu32;
        a.order = lower ? c->d_lorder : c->d_uorder;
        a.abort = c->d_ilu_abort;
        a.x = x;
        a.y = y;
        a.e = epi;
        a.st = c->st;
        a.check = check;
        a.wait_ns = c->waits.ns;
        a.unreachable = c->waits.extra_need ? 1 : 0;
        a.rdiag = prec == kF64 ? (const void *)c->d_ilu_rd64 : (const void *)c->d_ilu_rd32;
        a.red = c->ilu_red;
        c->launches++;
        PPG_CK(launch_ilu_solve(prec, lower, a, c->num_sms, s));
        const double sv = prec == kF64 ? 8.0 : 4.0;
        prof_add(c, (double)A->nnz * (sv + 4.0) + 4.0 * (A->n + 1) + 4.0 * A->n * (2.0 + sv), 0.0);
        return PPG_OK;
    }
    ppg_status launch_ilu_link(const SpmvEpi &e, int check)
    {
        SpmvEpi s1 = epi_none();
        s1.x = e.x;
        s1.x2 = e.x2;
        s1.s2 = e.s2;
        s1.out0 = vfix(ilu_v(0));
        s1.a0 = simm(1.0);
        c->launches++;
        PPG_CK(launch_spmv(*A, prec, s1, c->st, check, s));
        prof_add(c, spmv_bytes(*A, prec, s1), 0.0);
        PPG_TRY(ilu_solve(true, vfix(ilu_v(0)), ilu_v(1), epi_none(), check));
        SpmvEpi ep = e;
        ep.x = ep.x2 = vnone();
        return ilu_solve(false, vfix(ilu_v(1)), ilu_v(2), ep, check);
    }
    // dst = M^{-1} src (float64 vectors), skipped once the solve has stopped
    ppg_status ilu_apply64(const double *src, double *dst)
    {
        const int keep = prec;
        prec = kF64;
        ppg_status st = ilu_solve(true, vfix(src), ilu_v(1), epi_none(), kSkipIfStop);
        if (st >= 0) {
            SpmvEpi ep = epi_none();
            ep.out0 = vfix(dst);
            ep.a0 = simm(1.0);
            st = ilu_solve(false, vfix(ilu_v(1)), ilu_v(2), ep, kSkipIfStop);
        }
        prec = keep;
        return st;
    }
    // e2 consumes an output of e1 by gather and writes neither of its own gathered inputs, and the
    // matrix allows pairing (chain_pairs)
    bool can_pair(const SpmvEpi &e1, const SpmvEpi &e2) const
    {
        if (!c->fuse || (c->ilu_on && !plain) || !chain_pairs(*A, prec, c->d_rounds != nullptr)) return false;
        auto is_out = [&](const VecRef &v) {
            return v.base && ((e1.out0.base && same_vec(v, e1.out0)) || (e1.out1.base && same_vec(v, e1.out1)));
        };
        if (!is_out(e2.x) || (e2.x2.base && !is_out(e2.x2))) return false;
        for (const VecRef *o : {&e2.out0, &e2.out1})
            if (o->base && (same_vec(*o, e2.x) || (e2.x2.base && same_vec(*o, e2.x2)))) return false;
        return true;
    }
    ppg_status spmv(const SpmvEpi &e, int check)
    {
        if (has_pending) {
            has_pending = false;
            if (pending_check == check && can_pair(pending, e)) {
                const cudaError_t err = launch_spmv2(*A, prec, pending, e, c->st, check, c->d_rounds,
                                                     reinterpret_cast<unsigned int *>(c->d_rounds + kMaxRounds),
                                                     c->d_rounds + kMaxRounds + 8, c->waits, s);
                if (err == cudaSuccess) {
                    c->launches++;
                    const double mat = spmv_bytes(*A, prec, epi_none());  // the matrix, read once for both
                    prof_add(c, spmv_bytes(*A, prec, pending) + spmv_bytes(*A, prec, e) - mat, 0.0);
                    return PPG_OK;
                }
                // the grid cannot be resident at once (or the launch is refused): one link per launch
                cudaGetLastError();
                c->fuse = 0;
                PPG_TRY(launch_one(pending, pending_check));
                return launch_one(e, check);
            }
            PPG_TRY(launch_one(pending, check == pending_check ? check : pending_check));
        }
        if (chain_depth > 0 && c->fuse) {
            pending = e;
            pending_check = check;
            has_pending = true;
            return PPG_OK;
        }
        return launch_one(e, check);
    }
    ppg_status flush()
    {
        if (!has_pending) return PPG_OK;
        has_pending = false;
        return launch_one(pending, pending_check);
    }
    void chain_begin() { ++chain_depth; }
    ppg_status chain_end()
    {
        if (--chain_depth == 0) return flush();
        return PPG_OK;
    }
    ppg_status axpy(const SpmvEpi &e, int check)
    {
        PPG_TRY(flush());
        c->launches++;
        PPG_CK(launch_axpy(A->n, prec, e, c->st, check, s));
        return PPG_OK;
    }

    // dst = p(A) (scale * src).  sig: device sigma array (follows j) or null for 1.
    // tmp: 3 distinct working vectors, none of them src or dst.
    // When defer is given and the product form ends with a real root, the last update
    // dst += t P is not performed: *defer receives P and t so that the caller can fold it
    // into the SpMV that consumes dst (A (dst + t P)).
    struct Deferred {
        bool active = false;
        VecRef P;
        Scalar t;
    };
    ppg_status poly_apply(VecRef src, const double *sig, VecRef dst, char *const tmp[3], int check,
                          Deferred *defer = nullptr)
    {
        chain_begin();
        PPG_TRY(poly_apply_links(src, sig, dst, tmp, check, defer));
        return chain_end();
    }
    ppg_status poly_apply_links(VecRef src, const double *sig, VecRef dst, char *const tmp[3], int check,
                                Deferred *defer)
    {
        if (!c->has_poly) {
            SpmvEpi e = epi_none();
            e.out0 = dst;
            e.u0 = src;
            e.b0 = sscaled(1.0, sig);
            return axpy(e, check);
        }
        if (c->basis == PPG_BASIS_POWER) {
            const int d = c->degree;
            const std::vector<double> &y = c->coef;
            if (d == 0) {
                SpmvEpi e = epi_none();
                e.out0 = dst;
                e.u0 = src;
                e.b0 = sscaled(y[0], sig);
                return axpy(e, check);
            }
            // Horner: t_1 = y_d A v + y_{d-1} v;  t_i = A t_{i-1} + y_{d-i} v;  p(A) v = t_d
            VecRef prev = src;
            for (int i = 1; i <= d; ++i) {
                VecRef out = ((d - i) % 2 == 0) ? dst : vfix(tmp[0]);
                SpmvEpi e = epi_none();
                e.x = prev;
                e.out0 = out;
                e.a0 = (i == 1) ? sscaled(y[d], sig) : simm(1.0);
                e.u0 = src;
                e.b0 = sscaled(y[d - i], sig);
                PPG_TRY(spmv(e, check));
                prev = out;
            }
            return PPG_OK;
        }
        // product form over the Leja-ordered roots; y accumulates in dst
        const int k = c->degree + 1;
        const double *tb = c->table.data();
        const double *rt = c->roots.data();
        VecRef P = src;
        bool first = true;
        int pp = 0;  // which of tmp[0], tmp[1] receives the next P
        VecRef T = vfix(tmp[2]);
        for (int i = 0; i < k;) {
            const bool real = rt[2 * i + 1] == 0.0;
            const double *S = first ? sig : nullptr;
            if (real) {
                const double t = tb[2 * i];
                SpmvEpi e = epi_none();
                e.out0 = dst;
                e.u0 = P;
                e.b0 = sscaled(t, S);
                if (!first) {
                    e.w0 = dst;
                    e.c0 = simm(1.0);
                }
                if (i == k - 1) {
                    if (defer && !first) {
                        defer->active = true;
                        defer->P = P;
                        defer->t = e.b0;
                    } else {
                        PPG_TRY(axpy(e, check));
                    }
                } else {
                    VecRef Pn = vfix(tmp[pp]);
                    e.x = P;
                    e.a0 = simm(0.0);
                    e.out1 = Pn;
                    e.a1 = sscaled(-t, S);
                    e.u1 = P;
                    e.b1 = sscaled(1.0, S);
                    PPG_TRY(spmv(e, check));
                    P = Pn;
                    pp ^= 1;
                }
                i += 1;
            } else {
                const double c2a = tb[2 * i], cq = tb[2 * i + 1];
                const bool last = (i + 2 >= k);
                SpmvEpi e = epi_none();
                e.x = P;
                e.out0 = dst;
                e.a0 = sscaled(-cq, S);
                e.u0 = P;
                e.b0 = sscaled(c2a, S);
                if (!first) {
                    e.w0 = dst;
                    e.c0 = simm(1.0);
                }
                e.out1 = T;
                e.a1 = sscaled(1.0, S);
                PPG_TRY(spmv(e, check));
                if (!last) {
                    VecRef Pn = vfix(tmp[pp]);
                    SpmvEpi f = epi_none();
                    f.x = T;
                    f.out0 = Pn;
                    f.a0 = simm(cq);
                    f.u0 = T;
                    f.b0 = simm(-c2a);
                    f.w0 = P;
                    f.c0 = sscaled(1.0, S);
                    PPG_TRY(spmv(f, check));
                    P = Pn;
                    pp ^= 1;
                }
                i += 2;
            }
            first = false;
        }
        return PPG_OK;
    }

    // w = A p(A) (scale * src) - shift * (scale * src), fusing the scalar cases into one SpMV; the
    // shift (the s-step Newton basis) rides on the last SpMV's epilogue.
    ppg_status poly_then_A(VecRef src, const double *sig, VecRef w, char *const tmp[4], int check,
                           double shift = 0.0)
    {
        chain_begin();
        PPG_TRY(poly_then_A_links(src, sig, w, tmp, check, shift));
        return chain_end();
    }
    ppg_status poly_then_A_links(VecRef src, const double *sig, VecRef w, char *const tmp[4], int check,
                                 double shift)
    {
        if (!c->has_poly || (c->basis == PPG_BASIS_POWER && c->degree == 0)) {
            const double s0 = c->has_poly ? c->coef[0] : 1.0;
            SpmvEpi e = epi_none();
            e.x = src;
            e.out0 = w;
            e.a0 = sscaled(s0, sig);
            if (shift != 0.0) {
                e.u0 = src;
                e.b0 = sscaled(-shift, sig);
            }
            return spmv(e, check);
        }
        char *t3[3] = {tmp[1], tmp[2], tmp[3]};
        Deferred d;
        PPG_TRY(poly_apply(src, sig, vfix(tmp[0]), t3, check, &d));
        SpmvEpi e = epi_none();
        e.x = vfix(tmp[0]);
        if (d.active) {  // w = A (y + t P): the last root step rides on this SpMV's gather
            e.x2 = d.P;
            e.s2 = d.t;
        }
        e.out0 = w;
        e.a0 = simm(1.0);
        if (shift != 0.0) {
            e.u0 = src;
            e.b0 = sscaled(-shift, sig);
        }
        return spmv(e, check);
    }

    // Flexible form: z = p(A) (scale * src) is written to zdst (the preconditioned basis column of the
    // iteration) and w = A z.  When the product form ends with a real root, the last update
    // z = y + t P rides on the SpMV's gather as in poly_then_A, and the SpMV's second output writes
    // that z (the same fused value the gather used) to zdst.
    ppg_status poly_then_A_flex(VecRef src, const double *sig, VecRef zdst, VecRef w, char *const tmp[4], int check,
                                double shift = 0.0)
    {
        chain_begin();
        PPG_TRY(poly_then_A_flex_links(src, sig, zdst, w, tmp, check, shift));
        return chain_end();
    }
    // (shift: w = A z - shift * (scale * src), on the last SpMV's epilogue, for the s-step Newton basis)
    ppg_status poly_then_A_flex_links(VecRef src, const double *sig, VecRef zdst, VecRef w, char *const tmp[4],
                                      int check, double shift)
    {
        char *t3[3] = {tmp[1], tmp[2], tmp[3]};
        const int k = c->degree + 1;
        const bool defer = c->basis == PPG_BASIS_ROOTS && k >= 2 && c->roots[2 * (k - 1) + 1] == 0.0;
        const VecRef acc = defer ? vfix(tmp[0]) : zdst;
        Deferred d;
        PPG_TRY(poly_apply_links(src, sig, acc, t3, check, defer ? &d : nullptr));
        SpmvEpi e = epi_none();
        e.x = acc;
        e.out0 = w;
        e.a0 = simm(1.0);
        if (d.active) {
            e.x2 = d.P;
            e.s2 = d.t;
            e.out1 = zdst;
            e.a1 = simm(0.0);
            e.u1 = acc;
            e.b1 = simm(1.0);
            e.w1 = d.P;
            e.c1 = d.t;
        } else if (defer) {  // the chain did not leave the last root to the SpMV: z is the accumulator
            SpmvEpi cpy = epi_none();
            cpy.out0 = zdst;
            cpy.u0 = acc;
            cpy.b0 = simm(1.0);
            PPG_TRY(axpy(cpy, check));
            e.x = zdst;
        }
        if (shift != 0.0) {
            e.u0 = src;
            e.b0 = sscaled(-shift, sig);
        }
        return spmv(e, check);
    }

    // number of SpMVs in one application of p(A)
    int poly_spmvs() const
    {
        if (!c->has_poly) return 0;
        if (c->basis == PPG_BASIS_POWER) return c->degree;
        return c->degree;  // d+1 roots, the last one needs no SpMV
    }
};

// One Arnoldi iteration for A p(A): w = A p(A) v_j, then the three Gram-Schmidt passes.
struct Iter {
    Exec *x;
    const Layout *L;
    int maxcols;  // restart + 1: bound on the columns a cycle-end combination uses
    bool flex = false;  // flexible float32 form: z_j = p(A) v_j kept in L->zbasis, x += Z y
    bool sstep = false; // s-step blocks: the flexible form keeps P (Z = P M) and transforms y first

    // U: the basis the pass streams (null: the Krylov basis V); w: its vector input (null: vec[0])
    ppg_status gs(int op, int from_k, void *out, int out_follow, int kcols, const void *U = nullptr,
                  void *w = nullptr)
    {
        GsArgs a{};
        a.U = U ? U : L->basis;
        a.ldu = x->c->ld;
        a.w = w ? w : L->vec[0];
        a.out = out;
        a.out_follow = out_follow;
        a.op = op;
        a.kcols_from_k = from_k;
        a.partials = L->partials;
        a.rev = (x->c->gs_alternate && op == kGsUpdDot) ? 1 : 0;
        x->c->launches++;
        PPG_CK(launch_gs(x->prec, kcols, x->c->ld, x->c->num_sms, a, x->c->st, x->s));
        // bytes: k columns read, w read (except when combining), one vector written (passes 2-4);
        // at the cycle end k is known only after the cycle (kcol_bytes is scaled by it then)
        const double col = (double)x->A->n * (x->prec == kF64 ? 8.0 : 4.0);
        double fixed = col * ((op != kGsCombine ? 1.0 : 0.0) + (op != kGsDot ? 1.0 : 0.0));
        if (op == kGsProj) fixed = 2.0 * col;  // w and the extra column v_k
        if (from_k)
            prof_add(x->c, fixed, col);
        else
            prof_add(x->c, fixed + col * kcols, 0.0);
        return PPG_OK;
    }

    // x += Z y (flexible form): k columns of Z read, x read and written in float64
    ppg_status combine_x(double *xsol, int skip_if_stop)
    {
        x->c->launches++;
        PPG_CK(launch_combine_x(x->prec, L->zbasis, x->c->ld, x->A->n, xsol, x->c->st, skip_if_stop,
                                x->c->num_sms, x->s));
        prof_add(x->c, 16.0 * x->A->n, (double)x->A->n * (x->prec == kF64 ? 8.0 : 4.0));
        return PPG_OK;
    }

    // iteration j of the cycle (the device state carries the same j; kernels of a cycle
    // that ended early return at once)
    ppg_status iteration(int j)
    {
        ppg_ctx *c = x->c;
        c->prof_j = j;
        char *tmp[4] = {L->vec[1], L->vec[2], L->vec[3], L->vec[4]};
        prof_open(c, x->s, 0);
        if (flex)
            PPG_TRY(x->poly_then_A_flex(vcol(L->basis, c->ld, 0), c->st->sigma, vcol(L->zbasis, c->ld, 0),
                                        vfix(L->vec[0]), tmp, kSkipIfDone));
        else
            PPG_TRY(x->poly_then_A(vcol(L->basis, c->ld, 0), c->st->sigma, vfix(L->vec[0]), tmp, kSkipIfDone));
        prof_close(c, x->s);
        prof_open(c, x->s, 1);
        PPG_TRY(gs(kGsDot, 0, nullptr, 0, j + 1));
        PPG_TRY(gs(kGsUpdDot, 0, nullptr, 0, j + 1));
        PPG_TRY(gs(kGsUpdNorm, 0, nullptr, 1, j + 1));
        prof_close(c, x->s);
        return PPG_OK;
    }

    // One s-step block: sb Newton vectors (B - theta I) from basis column k into columns k + 1 ..
    // k + sb, then the three block passes (the reductions of the first two finish the block on the
    // device; the third forms (Z - Q C2) R^{-1}).
    // The device's j equals k whenever the block does work (every block of a live cycle advances j by
    // its size); once the cycle has ended every kernel returns at once.
    ppg_status block(int k, int sb, double theta, double tau)
    {
        ppg_ctx *c = x->c;
        c->prof_j = k;
        char *tmp[4] = {L->vec[1], L->vec[2], L->vec[3], L->vec[4]};
        prof_open(c, x->s, 0);
        for (int i = 0; i < sb; ++i) {  // columns follow the device's j (= k): j + i -> j + i + 1
            if (flex)  // the flexible form keeps P_i = p(A) u_i in column j + i of Z
                PPG_TRY(x->poly_then_A_flex(vcol(L->basis, c->ld, i), i == 0 ? c->st->sigma : nullptr,
                                            vcol(L->zbasis, c->ld, i), vcol(L->basis, c->ld, i + 1), tmp,
                                            kSkipIfDone, theta));
            else
                PPG_TRY(x->poly_then_A(vcol(L->basis, c->ld, i), i == 0 ? c->st->sigma : nullptr,
                                       vcol(L->basis, c->ld, i + 1), tmp, kSkipIfDone, theta));
        }
        prof_close(c, x->s);
        prof_open(c, x->s, 1);
        BgsArgs a{};
        a.U = L->basis;
        a.ld = c->ld;
        a.n = x->A->n;
        a.k = k;
        a.sb = sb;
        a.theta = theta;
        a.tau = tau;
        a.partials = c->d_bgs_partials;
        a.pld = c->bgs_pld;
        a.nblk = bgs_max_blocks(c->num_sms);
        a.flex = flex ? 1 : 0;
        const double col = (double)x->A->n * (x->prec == kF64 ? 8.0 : 4.0);
        for (int op : {kBgsDot, kBgsUpdDot, kBgsUpdTri}) {
            a.op = op;
            c->launches += op == kBgsUpdTri ? 1 : 2;
            PPG_CK(launch_bgs(x->prec, a, c->st, c->d_sstep, c->num_sms, x->s));
            // k + 1 basis columns and the block read; the block written by passes 2 and 3
            prof_add(c, col * (k + 1 + sb + (op == kBgsDot ? 0 : sb)), 0.0);
        }
        prof_close(c, x->s);
        return PPG_OK;
    }

    // Iteration j, replayed from a CUDA graph when use_graph is set (captured on first use, and
    // again whenever the signature of what its launches depend on has changed).
    bool use_graph = false;

    void signature(std::vector<double> &sig) const
    {
        const ppg_ctx *c = x->c;
        auto put = [&](unsigned long long v) {
            double d;
            memcpy(&d, &v, sizeof d);
            sig.push_back(d);
        };
        put((unsigned long long)(uintptr_t)L->basis);
        put((unsigned long long)(uintptr_t)L->partials);
        put((unsigned long long)(uintptr_t)(flex ? L->zbasis : nullptr));
        put((unsigned long long)c->ld);
        put((unsigned long long)((c->A.format << 8) | (c->fuse << 4) | (c->has_poly << 2) | c->basis));
        put((unsigned long long)c->degree);
        if (c->has_poly) {
            sig.insert(sig.end(), c->coef.begin(), c->coef.end());
            sig.insert(sig.end(), c->roots.begin(), c->roots.end());
            sig.insert(sig.end(), c->table.begin(), c->table.end());
        }
    }

    ppg_status run(int j)
    {
        ppg_ctx *c = x->c;
        if (!use_graph || c->prof || c->graphs_broken || j >= kKmax || c->ilu_on) return iteration(j);
        const size_t form = flex ? 2 : (x->prec == kF64 ? 1 : 0);
        const size_t slot = (size_t)j + (size_t)kKmax * (size_t)(2 * form + (c->has_poly ? 1 : 0));
        if (c->igraphs.size() < (size_t)(6 * kKmax)) c->igraphs.resize(6 * kKmax);
        ppg_ctx::IterGraph &g = c->igraphs[slot];
        std::vector<double> sig;
        signature(sig);
        if (!g.exec || g.sig != sig) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            // capture only once the same iteration comes round again: a one-off solve launches directly
            if (g.sig != sig) {
                g.sig.swap(sig);
                return iteration(j);
            }
            if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                c->graphs_broken = true;
                return iteration(j);
            }
            cudaStream_t keep = x->s;
            x->s = c->cap_stream;
            const long long l0 = c->launches;
            cudaGraph_t graph = nullptr;
            ppg_status st = PPG_ERR_CUDA;
            if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                st = iteration(j);
                if (cudaStreamEndCapture(c->cap_stream, &graph) != cudaSuccess) st = PPG_ERR_CUDA;
            }
            x->s = keep;
            const long long captured = c->launches - l0;  // kernels iteration j enqueued into the graph
            c->launches = l0;
            cudaGraphExec_t exec = nullptr;
            if (st >= 0 && graph && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
            if (graph) cudaGraphDestroy(graph);
            if (!exec) {  // this iteration cannot be captured here: launch directly from now on
                cudaGetLastError();
                c->graphs_broken = true;
                return iteration(j);
            }
            g.exec = exec;
            g.launches = captured;
            g.sig.swap(sig);
        }
        PPG_CK(cudaGraphLaunch(g.exec, x->s));
        c->launches += g.launches;
        return PPG_OK;
    }

    // x += p(A) V y with the coefficients the last pass-3 finalisation left in coef (flexible form:
    // x += Z y with the y it left, in float64).
    ppg_status cycle_end(double *xsol)
    {
        x->c->prof_j = -2;
        if (flex) {
            prof_open(x->c, x->s, 1);
            if (sstep) {
                x->c->launches++;
                PPG_CK(launch_sstep_flex_y(x->c->st, x->c->d_sstep, 0, x->s));
            }
            PPG_TRY(combine_x(xsol, 0));
            prof_close(x->c, x->s);
            return PPG_OK;
        }
        char *z = L->vec[5], *e = L->vec[6];
        prof_open(x->c, x->s, 1);
        PPG_TRY(gs(kGsCombine, 1, z, 0, maxcols));
        prof_close(x->c, x->s);
        const void *corr = z;
        if (x->c->has_poly) {
            char *t3[3] = {L->vec[1], L->vec[2], L->vec[3]};
            prof_open(x->c, x->s, 0);
            PPG_TRY(x->poly_apply(vfix(z), nullptr, vfix(e), t3, kSkipIfNoCols));
            prof_close(x->c, x->s);
            corr = e;
        }
        x->c->launches++;
        PPG_CK(launch_xupdate(x->A->n, x->prec, corr, xsol, x->c->st, x->s));
        return PPG_OK;
    }

    // Flexible form, before a restart: r = b - A x (float64, kept in float32 in vec[7]); unless the
    // solve stops there, y = argmin ||H y - V^T r|| over the finished cycle's space and x += Z y.
    // The residual that follows starts the next cycle.
    ppg_status restart_projection(const double *b, double *xsol)
    {
        ppg_ctx *c = x->c;
        c->prof_j = -2;
        c->launches++;
        PPG_CK(launch_residual(c->A, x->prec, b, xsol, L->vec[7], c->st, L->partials, x->s, 1));
        prof_open(c, x->s, 1);
        PPG_TRY(gs(kGsProj, 1, nullptr, 0, maxcols, L->basis, L->vec[7]));
        if (sstep) {
            c->launches++;
            PPG_CK(launch_sstep_flex_y(c->st, c->d_sstep, 1, x->s));
        }
        PPG_TRY(combine_x(xsol, 1));
        prof_close(c, x->s);
        return PPG_OK;
    }
};

ppg_status init_cycle_state(ppg_ctx *c, int mode, int m, long long maxit, double tol, double inner)
{
    Cycle *h = c->h_st;
    memset(h, 0, kCycleHeader);
    h->mode = mode;
    h->m = m;
    h->maxit = maxit;
    h->tol = tol;
    h->inner_rtol = inner;
    h->cycle_done = 1;
    h->prog = c->d_prog;
    PPG_CK(cudaMemcpyAsync(c->st, h, kCycleHeader, cudaMemcpyHostToDevice, c->stream));
    PPG_CK(cudaMemsetAsync(c->st->ticket, 0, sizeof(c->st->ticket), c->stream));
    return PPG_OK;
}

ppg_status read_state(ppg_ctx *c)
{
    PPG_CK(cudaMemcpyAsync(c->h_st, c->st, kCycleHeader, cudaMemcpyDeviceToHost, c->stream));
    PPG_CK(cudaStreamSynchronize(c->stream));
    if (c->h_st->error & kErrTimeout) {
        int d[8] = {0};
        if (c->d_rounds) {  // read and clear the two-step kernel's record of the wait that gave up
            cudaMemcpy(d, c->d_rounds + kMaxRounds + 8, sizeof d, cudaMemcpyDeviceToHost);
            cudaMemset(c->d_rounds + kMaxRounds + 8, 0, sizeof d);
        }
        if (d[0])
            return fail(PPG_ERR_TIMEOUT,
                        "a bounded device wait expired (two-step SpMV: %s wait, CTA %d of %d, iteration %d, round %d, "
                        "have %d need %d)",
                        d[0] == 1 ? "stage" : "round", d[1], d[6], d[2], d[3], d[4], d[5]);
        int row = 0;
        if (c->ilu_on && c->d_ilu_abort) cudaMemcpy(&row, c->d_ilu_abort, sizeof row, cudaMemcpyDeviceToHost);
        if (row > 0)
            return fail(PPG_ERR_TIMEOUT,
                        "a bounded device wait expired (ILU(0) triangular solve: the wait on the rows that row %d "
                        "depends on)",
                        row - 1);
        return fail(PPG_ERR_TIMEOUT, "a bounded device wait expired");
    }
    return PPG_OK;
}

// Runs `steps` Arnoldi iterations of A p(A) (current polynomial) from v (float64, n) in float64 with
// the solver's kernels; the Hessenberg matrix stays in c->st.  v may be null when the start vector is
// already in basis column 0.  Returns the number of steps completed in *done.
ppg_status run_arnoldi(ppg_ctx *c, const double *v, int steps, const Layout &L, int *done)
{
    Exec ex{c, &c->A, kF64, c->stream};
    Iter it{&ex, &L, steps + 1};
    PPG_TRY(init_cycle_state(c, 0, steps, steps, 0.0, 0.0));
    c->launches++;
    PPG_CK(launch_norm_start(c->A.n, kF64, v ? v : (const double *)L.basis, v ? (void *)L.basis : nullptr, 1, c->st,
                             L.partials, c->A.resid_blocks, c->stream));
    it.use_graph = true;
    for (int j = 0; j < steps; ++j) PPG_TRY(it.run(j));
    PPG_TRY(read_state(c));
    if (c->h_st->error & kErrNonfinite) return fail(PPG_ERR_NONFINITE, "non-finite value in the Arnoldi run");
    *done = c->h_st->j;
    return PPG_OK;
}

ppg_status build_power(ppg_ctx *c, int deg, const Layout &L, int *used, int *info)
{
    const long long ld = c->ld;
    Exec ex{c, &c->A, kF64, c->stream};
    for (int i = 1; i <= deg + 1; ++i) {
        SpmvEpi e = epi_none();
        e.x = vfix(L.basis + (size_t)(i - 1) * ld * sizeof(double));
        e.out0 = vfix(L.basis + (size_t)i * ld * sizeof(double));
        e.a0 = simm(1.0);
        PPG_TRY(ex.spmv(e, kNoCheck));
    }
    PPG_TRY(init_cycle_state(c, 0, 1, 1, 0.0, 0.0));
    c->launches++;
    PPG_CK(launch_gram_cholesky(c->A.n, ld, (const double *)L.basis, deg, L.partials, gram_grid(c->num_sms),
                                c->d_small, c->d_info, c->st, c->stream));
    PPG_CK(cudaMemcpyAsync(c->h_small, c->d_small, sizeof(double) * (deg + 1), cudaMemcpyDeviceToHost, c->stream));
    PPG_CK(cudaMemcpyAsync(c->h_info, c->d_info, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
    PPG_TRY(read_state(c));
    *info = c->h_info[0];
    *used = c->h_info[1];
    if (*used < 0) return fail(PPG_ERR_POLY_BREAKDOWN, "the Gram matrix of Eq. 1 is not positive at degree 0");
    if (!c->h_info[2]) return fail(PPG_ERR_POLY_BREAKDOWN, "non-finite polynomial coefficients");
    c->basis = PPG_BASIS_POWER;
    c->degree = *used;
    c->coef.assign(c->h_small, c->h_small + *used + 1);
    c->roots.clear();
    c->table.clear();
    c->poly_resid = NAN;
    c->has_poly = 1;
    return PPG_OK;
}

ppg_status build_roots(ppg_ctx *c, int deg, const Layout &L, int *used)
{
    // Arnoldi with A alone from v0 (already in basis column 0)
    const int had = c->has_poly;
    c->has_poly = 0;
    int done = 0;
    ppg_status s = run_arnoldi(c, nullptr, deg + 1, L, &done);
    c->has_poly = had;
    if (s < 0) return s;
    const int k = done;  // harmonic Ritz problem size; degree k - 1
    if (k < 1) return fail(PPG_ERR_POLY_BREAKDOWN, "the generating vector is zero");
    c->launches++;
    PPG_CK(launch_roots(c->st, k, c->d_small, c->d_small + 2 * kKmax, c->d_info, c->stream));
    PPG_CK(cudaMemcpyAsync(c->h_small, c->d_small, sizeof(double) * 4 * kKmax, cudaMemcpyDeviceToHost, c->stream));
    PPG_CK(cudaMemcpyAsync(c->h_info, c->d_info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PPG_CK(cudaStreamSynchronize(c->stream));
    if (c->h_info[0] != 0)
        return fail(PPG_ERR_POLY_BREAKDOWN, "roots of the residual polynomial failed (status %d)", c->h_info[0]);
    c->basis = PPG_BASIS_ROOTS;
    c->degree = k - 1;
    c->roots.assign(c->h_small, c->h_small + 2 * k);
    c->table.assign(c->h_small + 2 * kKmax, c->h_small + 2 * kKmax + 2 * k);
    c->coef.clear();
    c->poly_resid = c->h_st->est;
    c->has_poly = 1;
    *used = k - 1;
    return PPG_OK;
}

// Profiling: after a cycle's launches, read how many iterations really ran (later launches of
// the cycle returned at once) and how many columns the cycle end combined, and mark records.
ppg_status prof_close_cycle(ppg_ctx *c)
{
    PPG_TRY(read_state(c));
    const int done = c->h_st->j, k = c->h_st->k;
    for (size_t i = c->rec_first; i < c->recs.size(); ++i) {
        ppg_ctx::ProfRec &r = c->recs[i];
        if (r.j >= 0) {
            r.valid = r.j < done;
        } else {
            r.valid = k > 0;
            if (r.cls == 1) r.bytes += r.kcol_bytes * k;
        }
    }
    c->rec_first = c->recs.size();
    return PPG_OK;
}

// Profiling of a restart projection (flexible form): its launches did work when the device
// counted a projection; k is still the finished cycle's (the next residual resets it).
ppg_status prof_close_proj(ppg_ctx *c, long long nproj_before)
{
    PPG_TRY(read_state(c));
    const bool ran = c->h_st->nproj > nproj_before;
    const int k = c->h_st->k;
    for (size_t i = c->rec_first; i < c->recs.size(); ++i) {
        ppg_ctx::ProfRec &r = c->recs[i];
        r.valid = ran;
        r.bytes += r.kcol_bytes * k;
    }
    c->rec_first = c->recs.size();
    return PPG_OK;
}

void prof_collect(ppg_ctx *c, ppg_stats *st)
{
    for (const ppg_ctx::ProfRec &r : c->recs) {
        if (!r.valid || !r.b) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
        if (r.cls == 0) {
            st->spmv_ms += ms;
            st->spmv_bytes += r.bytes;
            st->spmv_segments += 1;
        } else {
            st->gs_ms += ms;
            st->gs_bytes += r.bytes;
            st->gs_segments += 1;
        }
    }
}

// Iterations kept queued on the stream beyond the last one the device has finished.  The
// device publishes its progress after every iteration (Cycle::prog); once a cycle ends
// (convergence, breakdown, restart length or iteration limit) the host enqueues nothing
// more for it, so at most this many launched iterations return without work.
int launch_ahead()
{
    static const int v = [] {
        const char *e = getenv("PPG_LAUNCH_AHEAD");
        const int a = e ? atoi(e) : 0;
        return a > 0 ? a : 2;
    }();
    return v;
}

// Enqueues the iterations of one restart cycle.  The host waits (yielding) while `ahead`
// iterations are queued; the wait also ends when the stream has drained, which a cycle whose
// kernels returned early (an error flag) can cause: the caller reads the state next.
// The wait is bounded too (c->waits.ns without any progress by the device): when it runs out the
// host enqueues nothing more, lets the work already queued finish (every device wait is bounded) and
// reports PPG_ERR_TIMEOUT.
ppg_status run_cycle(ppg_ctx *c, Iter &it, int restart)
{
    volatile int *prog = c->h_prog;
    *prog = 0;
    const int ahead = launch_ahead();
    for (int j = 0; j < restart; ++j) {
        auto t0 = std::chrono::steady_clock::now();
        int seen = *prog & 0xffff;
        for (int spin = 0;; ++spin) {
            const int p = *prog;
            if (p >> 16) return PPG_OK;
            if (j - (p & 0xffff) < ahead) break;
            if ((p & 0xffff) != seen) {  // progress: the limit counts from the last step the device made
                seen = p & 0xffff;
                t0 = std::chrono::steady_clock::now();
            }
            if ((spin & 63) == 63) {
                const cudaError_t q = cudaStreamQuery(c->stream);
                if (q == cudaSuccess) {
                    if (*prog >> 16) return PPG_OK;
                    break;
                }
                if (q != cudaErrorNotReady) PPG_CK(q);
            }
            const long long waited =
                std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
            if ((unsigned long long)waited > c->waits.ns) {
                // the device's own record first: a device wait that ran out explains the delay
                PPG_TRY(read_state(c));
                return fail(PPG_ERR_TIMEOUT,
                            "the host's wait for the device's progress ran out after %lld us (iteration %d queued, "
                            "device at iteration %d of the cycle)",
                            waited / 1000, j, *prog & 0xffff);
            }
            std::this_thread::yield();
        }
        PPG_TRY(it.run(j));
    }
    return PPG_OK;
}

// Enqueues the blocks of one s-step restart cycle, paced like run_cycle: at most launch_ahead()
// blocks beyond the one the device is working on.
ppg_status run_cycle_sstep(ppg_ctx *c, Iter &it, int restart, int s, double theta, double tau)
{
    volatile int *prog = c->h_prog;
    *prog = 0;
    const int ahead = launch_ahead();
    for (int k = 0; k < restart;) {
        const int sb = std::min(s, restart - k);
        auto t0 = std::chrono::steady_clock::now();
        int seen = *prog & 0xffff;
        for (int spin = 0;; ++spin) {
            const int p = *prog;
            if (p >> 16) return PPG_OK;
            if (k - (p & 0xffff) < ahead * s) break;
            if ((p & 0xffff) != seen) {
                seen = p & 0xffff;
                t0 = std::chrono::steady_clock::now();
            }
            if ((spin & 63) == 63) {
                const cudaError_t q = cudaStreamQuery(c->stream);
                if (q == cudaSuccess) {
                    if (*prog >> 16) return PPG_OK;
                    break;
                }
                if (q != cudaErrorNotReady) PPG_CK(q);
            }
            const long long waited =
                std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
            if ((unsigned long long)waited > c->waits.ns) {
                PPG_TRY(read_state(c));
                return fail(PPG_ERR_TIMEOUT,
                            "the host's wait for the device's progress ran out after %lld us (block at column %d "
                            "queued, device at column %d of the cycle)",
                            waited / 1000, k, *prog & 0xffff);
            }
            std::this_thread::yield();
        }
        PPG_TRY(it.block(k, sb, theta, tau));
        k += sb;
    }
    return PPG_OK;
}

ppg_status ensure_sstep(ppg_ctx *c)
{
    if (c->d_sstep) return PPG_OK;
    const int nblk = bgs_max_blocks(c->num_sms);
    const int pld = (nblk + 1) & ~1;
    // one slot per (sum, CTA): at most (k + 1) s inner products plus s (s + 1) / 2 Gram entries per pass
    const size_t slots = (size_t)(kSMax * kSColsMax + kSMax * (kSMax + 1) / 2) * (size_t)pld;
    if (cudaMalloc(&c->d_bgs_partials, slots * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->d_bgs_partials = nullptr;
        return fail(PPG_ERR_OOM, "cannot allocate the s-step passes' partial sums");
    }
    if (cudaMalloc(&c->d_sstep, sizeof(SStep)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->d_bgs_partials);
        c->d_bgs_partials = nullptr;
        c->d_sstep = nullptr;
        return fail(PPG_ERR_OOM, "cannot allocate the s-step state");
    }
    PPG_CK(cudaMemsetAsync(c->d_sstep, 0, sizeof(SStep), c->stream));
    c->bgs_pld = pld;
    return PPG_OK;
}

ppg_status solve_impl(ppg_ctx *c, const double *b, double *x, double tol, int restart, int maxit,
                      const ppg_opts *opts, ppg_stats *stats)
{
    if (!b || !x) return fail(PPG_ERR_INVALID_ARG, "null b or x");
    if (restart < 1 || restart > kKmax - 1) return fail(PPG_ERR_INVALID_ARG, "restart must be in [1, %d]", kKmax - 1);
    if (maxit < 0 || !(tol >= 0.0)) return fail(PPG_ERR_INVALID_ARG, "bad tol or maxit");
    const int prec = opts ? opts->precision : PPG_F64;
    if (prec != PPG_F64 && prec != PPG_F32) return fail(PPG_ERR_INVALID_ARG, "unknown precision");
    const int form = opts ? opts->f32_form : PPG_F32_FLEXIBLE;
    if (form != PPG_F32_FLEXIBLE && form != PPG_F32_STANDARD) return fail(PPG_ERR_INVALID_ARG, "unknown f32_form");
    // s-step blocks (Section VII's combination): sstep vectors per orthogonalisation, shift theta
    const int sstep = opts ? opts->sstep : 0;
    const double theta = opts ? opts->sstep_shift : 0.0;
    if (sstep < 0 || sstep > kSMax) return fail(PPG_ERR_INVALID_ARG, "sstep must be in [0, %d]", kSMax);
    if (sstep > 0) {
        if (restart > kSColsMax) return fail(PPG_ERR_INVALID_ARG, "s-step solves take restart <= %d", kSColsMax);
        if (c->ilu_on) return fail(PPG_ERR_INVALID_ARG, "s-step solves do not take ILU(0) on the left");
        if (!std::isfinite(theta)) return fail(PPG_ERR_INVALID_ARG, "the s-step shift must be finite");
    }
    // the flexible form keeps z_j = p(A) v_j; with no polynomial (or a scalar one) z_j is v_j itself
    // (with ILU(0) on the left the standard form runs: its operator is M^{-1} A throughout).  s-step
    // solves keep the chains' p(A) u_i instead and combine them through M (Z = P M)
    const bool flex = prec == PPG_F32 && form == PPG_F32_FLEXIBLE && c->has_poly &&
                      !(c->basis == PPG_BASIS_POWER && c->degree == 0) && !c->ilu_on;
    // limits of the software waits for this solve (the context keeps the defaults otherwise)
    c->waits = WaitCfg{};
    if (opts && opts->wait_limit_us > 0 && opts->wait_limit_us < 1000000)
        c->waits.ns = 1000ull * (unsigned long long)opts->wait_limit_us;
    if (opts && opts->test_unreachable_wait) c->waits.extra_need = 1;
    struct Restore {
        ppg_ctx *c;
        ~Restore() { c->waits = WaitCfg{}; }
    } restore{c};
    double inner = 0.0;
    if (prec == PPG_F32) {
        inner = (opts && opts->inner_rtol > 0.0) ? opts->inner_rtol : (flex ? 1e-7 : 1e-6);
        PPG_TRY(ensure_f32(c));
    }
    const size_t es = prec == PPG_F64 ? 8 : 4;
    const int ncols = restart + 1;
    Layout L;
    PPG_TRY(get_layout(c, ncols, es, &L));
    if (sstep > 0) PPG_TRY(ensure_sstep(c));
    // dependence test of the block's Cholesky QR: a pivot below tau ||z||^2 (float64: the Arnoldi
    // breakdown level; float32: the level to which a float32 block's Gram matrix resolves it)
    const double tau = prec == PPG_F64 ? 1e-14 : 1e-6;
    const long long launches0 = c->launches;
    PPG_CK(cudaEventRecord(c->ev0, c->stream));

    Exec ex{c, &c->A, prec, c->stream};
    Iter it{&ex, &L, ncols};
    it.flex = flex;
    it.sstep = sstep > 0;
    it.use_graph = !opts || opts->use_graph != 0;
    c->prof = opts && opts->profile;
    c->prof_open = false;
    c->recs.clear();
    c->rec_first = 0;
    c->evnext = 0;
    c->prof_j = -1;

    PPG_TRY(init_cycle_state(c, 0, restart, maxit, tol, inner));
    c->launches++;
    PPG_CK(launch_norm_start(c->A.n, kF64, b, nullptr, 0, c->st, L.partials, c->A.resid_blocks, c->stream));
    // ILU(0) on the left (Section VI): the estimate is relative to ||M^{-1} b||, and every cycle starts
    // from the preconditioned residual M^{-1} (b - A x) while the stopping test stays on b - A x
    double *ilu_r = c->ilu_on ? reinterpret_cast<double *>(ex.ilu_v(3)) : nullptr;
    double *ilu_rm = c->ilu_on ? reinterpret_cast<double *>(ex.ilu_v(4)) : nullptr;
    auto start_cycle = [&]() -> ppg_status {
        c->launches++;
        if (!c->ilu_on) {
            PPG_CK(launch_residual(c->A, prec, b, x, L.basis, c->st, L.partials, c->stream));
            return PPG_OK;
        }
        PPG_CK(launch_residual(c->A, kF64, b, x, ilu_r, c->st, L.partials, c->stream, 1));
        PPG_TRY(ex.ilu_apply64(ilu_r, ilu_rm));
        c->launches++;
        PPG_CK(launch_norm_start(c->A.n, prec, ilu_rm, L.basis, 3, c->st, L.partials, c->A.resid_blocks,
                                 c->stream));
        return PPG_OK;
    };
    if (c->ilu_on) {
        PPG_CK(cudaMemsetAsync(c->d_ilu_abort, 0, sizeof(int), c->stream));
        PPG_TRY(ex.ilu_apply64(b, ilu_rm));
        c->launches++;
        PPG_CK(launch_norm_start(c->A.n, kF64, ilu_rm, nullptr, 2, c->st, L.partials, c->A.resid_blocks,
                                 c->stream));
    }
    PPG_TRY(read_state(c));
    if (c->h_st->bnorm == 0.0) {
        PPG_CK(cudaMemsetAsync(x, 0, sizeof(double) * c->A.n, c->stream));
        c->h_st->converged = 1;
        c->h_st->relres = 0.0;
    } else {
        PPG_TRY(start_cycle());
        PPG_TRY(read_state(c));
        while (!c->h_st->stop) {
            if (sstep > 0)
                PPG_TRY(run_cycle_sstep(c, it, restart, sstep, theta, tau));
            else
                PPG_TRY(run_cycle(c, it, restart));
            PPG_TRY(it.cycle_end(x));
            if (c->prof) PPG_TRY(prof_close_cycle(c));
            if (flex) {
                const long long np = c->h_st->nproj;
                PPG_TRY(it.restart_projection(b, x));
                if (c->prof) PPG_TRY(prof_close_proj(c, np));
            }
            PPG_TRY(start_cycle());
            PPG_TRY(read_state(c));
        }
    }
    PPG_CK(cudaEventRecord(c->ev1, c->stream));
    PPG_CK(cudaEventSynchronize(c->ev1));
    const Cycle &h = *c->h_st;
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        memset(stats, 0, sizeof *stats);
        stats->iterations = h.iters;
        stats->restarts = h.cycles;
        // per iteration p(A) and A; per cycle end p(A) once (not in the flexible form); every
        // true residual; dots: three per iteration (Section III), a norm per residual, and one block
        // inner product per restart projection
        const int ps = ex.poly_spmvs();
        if (sstep > 0) {  // per block: its Newton vectors' chains and three reductions
            stats->spmvs = h.nnewton * (long long)(ps + 1) + h.cycles * (long long)ps + h.nres;
            stats->dots = 3 * h.nblocks + h.nres;
        } else {
            stats->spmvs = h.iters * (long long)(ps + 1) + (flex ? 0 : h.cycles * (long long)ps) + h.nres;
            stats->dots = 3 * h.iters + h.nres + h.nproj;
        }
        stats->kernel_launches = c->launches - launches0;
        stats->relres_true = h.relres;
        stats->relres_est = h.est;
        stats->degree_used = c->has_poly ? c->degree : 0;
        stats->converged = h.converged;
        stats->breakdowns = h.n_breakdowns;
        stats->time_ms = ms;
        if (c->prof) prof_collect(c, stats);
    }
    c->prof = false;
    if (h.error & kErrNonfinite) return fail(PPG_ERR_NONFINITE, "non-finite value in a reduction");
    return h.converged ? PPG_OK : PPG_ERR_NOT_CONVERGED;
}

ppg_status check_ctx(const ppg_ctx *c)
{
    if (!c) return fail(PPG_ERR_INVALID_ARG, "null context");
    return PPG_OK;
}

ppg_status set_device(const ppg_ctx *c)
{
    PPG_CK(cudaSetDevice(c->device));
    return PPG_OK;
}

}  // namespace

// =================================================================== batched solves

namespace {

// Per-device state of ppg_solve_batched: workspace, descriptors, the tuned cluster size and the
// captured launch, kept between calls.
struct BatchCache {
    char *ws = nullptr;
    size_t ws_bytes = 0;
    BatchSys *sys_d = nullptr;
    int *order_d = nullptr;
    BatchOut *out_d = nullptr;
    int cap_sys = 0;
    cudaStream_t stream = nullptr, stream2 = nullptr;  // stream2: the small systems' launch of a split batch
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr, ev_fork = nullptr, ev_join = nullptr;
    // autotuner: per batch shape (the sorted (n, nnz) list, degree and restart), the cluster size, and
    // optionally a split: systems with at least big_rows rows run in clusters of `cluster`, the others in
    // clusters of `cluster2` (a second launch, concurrent with the first); and the SpMV's threads per row
    // of each class of rows per CTA
    struct Tuned {
        int cluster = 0;
        int cluster2 = 0;
        long long big_rows = 0;  // 0: one launch, every system in clusters of `cluster`
        int threads = 256;       // threads per CTA of the (large systems') first launch
        int lanes[3] = {1, 1, 1};
    };
    std::map<std::vector<long long>, Tuned> tuned;
    int cluster = 0;  // the current call's
    BatchSys *tune_d = nullptr;  // descriptors of the tuning runs (x in scratch memory)
    int *tune_order_d = nullptr;
    int cap_tune = 0;
    // captured launch
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> exec_key;
    bool configured = false;
};

BatchCache g_batch[64];
std::mutex g_batch_mu;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

ppg_status batch_setup(BatchCache &bc, int nsys)
{
    if (!bc.configured) {
        PPG_CK(batch_configure());
        PPG_CK(cudaStreamCreateWithFlags(&bc.stream, cudaStreamNonBlocking));
        PPG_CK(cudaStreamCreateWithFlags(&bc.stream2, cudaStreamNonBlocking));
        PPG_CK(cudaEventCreateWithFlags(&bc.ev_in, cudaEventDisableTiming));
        PPG_CK(cudaEventCreateWithFlags(&bc.ev_out, cudaEventDisableTiming));
        PPG_CK(cudaEventCreateWithFlags(&bc.ev_fork, cudaEventDisableTiming));
        PPG_CK(cudaEventCreateWithFlags(&bc.ev_join, cudaEventDisableTiming));
        PPG_CK(cudaEventCreate(&bc.t0));
        PPG_CK(cudaEventCreate(&bc.t1));
        bc.configured = true;
    }
    if (nsys > bc.cap_tune) {
        cudaFree(bc.tune_d);
        cudaFree(bc.tune_order_d);
        bc.tune_d = nullptr;
        bc.tune_order_d = nullptr;
        bc.cap_tune = 0;
        PPG_CK(cudaMalloc(&bc.tune_d, sizeof(BatchSys) * nsys));
        PPG_CK(cudaMalloc(&bc.tune_order_d, sizeof(int) * nsys));
        bc.cap_tune = nsys;
    }
    if (nsys > bc.cap_sys) {
        cudaFree(bc.sys_d);
        cudaFree(bc.order_d);
        cudaFree(bc.out_d);
        bc.sys_d = nullptr;
        bc.order_d = nullptr;
        bc.out_d = nullptr;
        bc.cap_sys = 0;
        PPG_CK(cudaMalloc(&bc.sys_d, sizeof(BatchSys) * nsys));
        PPG_CK(cudaMalloc(&bc.order_d, sizeof(int) * nsys));
        PPG_CK(cudaMalloc(&bc.out_d, sizeof(BatchOut) * nsys));
        bc.cap_sys = nsys;
    }
    return PPG_OK;
}

}  // namespace

// =================================================================== allocation-free apply

// Device scratch for ppg_apply_poly_noalloc: the input copy, the output and three working
// vectors of at most kNoAllocMaxN entries each, in one file-scope array that every GPU
// loading the library keeps until the process exits.
namespace {
constexpr long long kNoAllocMaxN = 65536;
constexpr int kNoAllocVecs = 5;
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocVecs * kNoAllocMaxN];

namespace {

// Device address of g_noalloc_scratch on `device` (which must be current).  In host code the
// symbol's name only stands for the device array, so the address is looked up once per device
// with cudaGetSymbolAddress and cached.
ppg_status noalloc_scratch(int device, char **out)
{
    static std::mutex mu;
    static void *addr[256] = {};
    if (device < 0 || device >= 256) return fail(PPG_ERR_INVALID_ARG, "device ordinal %d out of range", device);
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(PPG_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch): %s", cudaGetErrorString(e));
        addr[device] = p;
    }
    *out = static_cast<char *>(addr[device]);
    return PPG_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

const char *ppg_version(void) { return "ppg 0.1 (sm_103a)"; }

const char *ppg_last_error(void) { return g_last_error.c_str(); }

const char *ppg_status_string(ppg_status s)
{
    switch (s) {
    case PPG_OK: return "ok";
    case PPG_WARN_DEGREE_CLAMPED: return "degree clamped (Cholesky of the power-basis Gram matrix failed)";
    case PPG_ERR_NOT_CONVERGED: return "not converged";
    case PPG_ERR_INVALID_ARG: return "invalid argument";
    case PPG_ERR_CUDA: return "CUDA error";
    case PPG_ERR_POLY_BREAKDOWN: return "polynomial breakdown";
    case PPG_ERR_NONFINITE: return "non-finite value";
    case PPG_ERR_TIMEOUT: return "device wait timed out";
    case PPG_ERR_OOM: return "out of device memory";
    case PPG_ERR_NO_POLY: return "no polynomial";
    }
    return "unknown status";
}

ppg_status ppg_create(ppg_ctx **out, int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                      const double *vals, void *stream)
{
    g_last_error.clear();
    if (!out) return fail(PPG_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    if (n <= 0 || nnz < 0 || n >= (1LL << 31) - 256 || nnz >= (1LL << 31) - 64)
        return fail(PPG_ERR_INVALID_ARG, "bad sizes n=%lld nnz=%lld", (long long)n, (long long)nnz);
    if (!rowptr || (nnz > 0 && (!colidx || !vals))) return fail(PPG_ERR_INVALID_ARG, "null CSR pointer");
    ppg_ctx *c = new (std::nothrow) ppg_ctx();
    if (!c) return fail(PPG_ERR_OOM, "host allocation failed");
    struct Guard {
        ppg_ctx **c;
        ~Guard()
        {
            if (*c) ppg_destroy(*c);
        }
    } guard{&c};

    PPG_CK(cudaGetDevice(&c->device));
    PPG_CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    c->stream = (cudaStream_t)stream;
    c->A.n = (int)n;
    c->A.nnz = nnz;
    c->A.num_sms = c->num_sms;
    c->A.resid_blocks = c->num_sms * 8;
    c->ld = round_up(n, kLdPad);
    PPG_CK(cudaMalloc(&c->d_rowptr, sizeof(int) * (n + 1 + 16)));
    PPG_CK(cudaMemsetAsync(c->d_rowptr, 0, sizeof(int) * (n + 1 + 16), c->stream));
    PPG_CK(cudaMalloc(&c->d_colidx, sizeof(int) * (nnz + 16)));
    PPG_CK(cudaMalloc(&c->d_vals, sizeof(double) * (nnz + 8)));
    PPG_CK(cudaMemcpyAsync(c->d_rowptr, rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, c->stream));
    PPG_CK(cudaMemsetAsync(c->d_colidx, 0, sizeof(int) * (nnz + 16), c->stream));
    PPG_CK(cudaMemsetAsync(c->d_vals, 0, sizeof(double) * (nnz + 8), c->stream));
    if (nnz > 0) {
        PPG_CK(cudaMemcpyAsync(c->d_colidx, colidx, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, c->stream));
        PPG_CK(cudaMemcpyAsync(c->d_vals, vals, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, c->stream));
    }
    c->A.rowptr = c->d_rowptr;
    c->A.colidx = c->d_colidx;
    c->A.vals64 = c->d_vals;

    PPG_CK(cudaMalloc(&c->st, sizeof(Cycle)));
    PPG_CK(cudaMemsetAsync(c->st, 0, sizeof(Cycle), c->stream));
    PPG_CK(cudaMalloc(&c->d_small, sizeof(double) * 4 * kKmax));
    PPG_CK(cudaMalloc(&c->d_info, sizeof(int) * 16));
    PPG_CK(cudaMallocHost(&c->h_st, kCycleHeader));
    PPG_CK(cudaMallocHost(&c->h_info, sizeof(int) * 16));
    PPG_CK(cudaMallocHost(&c->h_small, sizeof(double) * 4 * kKmax));
    PPG_CK(cudaHostAlloc(&c->h_prog, 64, cudaHostAllocMapped));
    PPG_CK(cudaHostGetDevicePointer((void **)&c->d_prog, c->h_prog, 0));
    PPG_CK(cudaEventCreate(&c->ev0));
    PPG_CK(cudaEventCreate(&c->ev1));

    // validate on the device
    PPG_CK(cudaMemsetAsync(c->d_info, 0, sizeof(int), c->stream));
    PPG_CK(launch_validate((int)n, nnz, c->d_rowptr, c->d_colidx, c->d_info, c->stream));
    PPG_CK(cudaMemcpyAsync(c->h_info, c->d_info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PPG_CK(cudaStreamSynchronize(c->stream));
    if (c->h_info[0] != 0) return fail(PPG_ERR_INVALID_ARG, "invalid CSR (validation flags 0x%x)", c->h_info[0]);

    // int16 column offsets halve the index traffic of the SpMV where every entry lies within 32767
    // of its row (all banded / stencil matrices of moderate bandwidth)
    PPG_CK(cudaMalloc(&c->d_coloff, sizeof(short) * (nnz + 16)));
    PPG_CK(cudaMemsetAsync(c->d_coloff, 0, sizeof(short) * (nnz + 16), c->stream));
    PPG_CK(cudaMemsetAsync(c->d_info, 0, 2 * sizeof(int), c->stream));
    if (nnz > 0) PPG_CK(launch_make_coloff((int)n, c->d_rowptr, c->d_colidx, c->d_coloff, c->d_info, c->stream));
    PPG_CK(cudaMemcpyAsync(c->h_info, c->d_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PPG_CK(cudaStreamSynchronize(c->stream));
    if (c->h_info[0] != 0) {
        cudaFree(c->d_coloff);
        c->d_coloff = nullptr;
    }
    c->A.coloff = c->d_coloff;
    c->A.bw = c->h_info[1];
    // round counters and ticket of the two-step chain kernel
    PPG_CK(cudaMalloc(&c->d_rounds, sizeof(int) * (kMaxRounds + 16)));
    PPG_CK(cudaMemsetAsync(c->d_rounds, 0, sizeof(int) * (kMaxRounds + 16), c->stream));

    // tiling: rows per tile from the mean row length, staging capacity from the largest tile
    const double avg = n > 0 ? (double)nnz / (double)n : 0.0;
    int R = 256;
    if (avg > 10) R = 128;
    if (avg > 20) R = 64;
    if (avg > 40) R = 32;
    if (avg > 80) R = 8;
    const int G = kThreads / R;  // lanes per row
    R *= spmv_rows_per_thread();
    std::vector<int> hrp(n + 1);
    PPG_CK(cudaMemcpy(hrp.data(), c->d_rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
    long long maxtile = 0;
    for (long long r0 = 0; r0 < n; r0 += R) {
        const long long r1 = std::min<long long>(n, r0 + R);
        maxtile = std::max<long long>(maxtile, hrp[r1] - hrp[r0]);
    }
    const long long cap = std::min<long long>(spmv_cap_max(), round_up(maxtile + 8, 16));
    c->A.rows_per_tile = R;
    c->A.lanes_per_row = G;
    c->A.cap64 = (int)std::max<long long>(cap, 64);
    c->A.cap32 = (int)std::max<long long>(cap, 64);

    // x windows per tile for the staged kernels: the tile's sorted distinct columns are grouped into
    // ranges (columns closer than kXGap share one), each widened to 16-byte boundaries and kept
    // inside [0, n rounded down to 4); a tile needing more than maxw ranges or kXCap entries keeps
    // global gathers (lengths 0).  desc: [tiles][2 maxw] (starts, lengths); lidx: per entry, its
    // index in the tile's concatenated windows; returns the number of covered tiles and the longest
    // window total.
    auto make_windows = [&](const std::vector<int> &hcol, long long Rt, int maxw, std::vector<int> &desc,
                            std::vector<short> &lidx, long long *xmax) -> long long {
        const long long ntiles = (n + Rt - 1) / Rt;
        const long long n4 = n & ~3LL;
        desc.assign(ntiles * 2 * maxw, 0);
        lidx.assign(nnz + 16, 0);
        std::vector<int> cols;
        long long windowed = 0;
        *xmax = 0;
        for (long long t = 0; t < ntiles; ++t) {
            const long long r0 = t * Rt, r1 = std::min<long long>(n, r0 + Rt);
            cols.assign(hcol.begin() + hrp[r0], hcol.begin() + hrp[r1]);
            if (cols.empty()) continue;
            std::sort(cols.begin(), cols.end());
            int lo[kEWin], hi[kEWin], nw = 0;
            bool ok = true;
            long long lw = cols[0], hw = cols[0];
            for (size_t q = 1; q <= cols.size() && ok; ++q) {
                if (q < cols.size() && cols[q] <= hw + kXGap) {
                    hw = std::max<long long>(hw, cols[q]);
                    continue;
                }
                const long long a = lw & ~3LL, b = (hw + 4) & ~3LL;  // [a, b) covers [lw, hw]
                if (nw == maxw || a < 0 || b > n4) ok = false;
                else {
                    lo[nw] = (int)a;
                    hi[nw] = (int)b;
                    ++nw;
                }
                if (q < cols.size()) lw = hw = cols[q];
            }
            long long total = 0;
            for (int w = 0; w < nw; ++w) total += hi[w] - lo[w];
            if (!ok || total > kXCap) continue;
            *xmax = std::max(*xmax, total);
            int off[kEWin];
            for (int w = 0, o = 0; w < nw; ++w) {
                desc[t * 2 * maxw + w] = lo[w];
                desc[t * 2 * maxw + maxw + w] = hi[w] - lo[w];
                off[w] = o;
                o += hi[w] - lo[w];
            }
            for (long long k = hrp[r0]; k < hrp[r1]; ++k) {
                const int col = hcol[k];
                int w = 0;
                while (w + 1 < nw && col >= lo[w + 1]) ++w;
                lidx[k] = (short)(off[w] + col - lo[w]);
            }
            ++windowed;
        }
        return windowed;
    };
    if (nnz > 0 && R <= 256) {
        std::vector<int> hcol(nnz);
        PPG_CK(cudaMemcpy(hcol.data(), c->d_colidx, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
        const long long ntiles = (n + R - 1) / R;
        std::vector<int> desc;
        std::vector<short> lidx;
        long long xmax = 0;
        const long long windowed = make_windows(hcol, R, kXWin, desc, lidx, &xmax);
        if (windowed * 10 >= ntiles * 9) {  // worth a kernel of its own when nearly every tile is covered
            PPG_CK(cudaMalloc(&c->d_twin, sizeof(int) * desc.size()));
            PPG_CK(cudaMemcpy(c->d_twin, desc.data(), sizeof(int) * desc.size(), cudaMemcpyHostToDevice));
            PPG_CK(cudaMalloc(&c->d_lidx, sizeof(short) * lidx.size()));
            PPG_CK(cudaMemcpy(c->d_lidx, lidx.data(), sizeof(short) * lidx.size(), cudaMemcpyHostToDevice));
            c->A.twin = c->d_twin;
            c->A.lidx = c->d_lidx;
        }
        // tile-ELL copy, one thread per row, for tiles of kThreads rows whose windows (up to kEWin
        // ranges each) all exist: tile t is a dense kThreads x w_t block (entry k of row l at
        // k kThreads + l) of float32 values and window indices, padded with value 0 and the index
        // exmax (the longest window total) of a zero kept after the windows.  w_t is the tile's longest
        // row rounded up to a multiple of the row-block kernel's lanes per row G: the thread sums
        // entries k = g mod G apart and combines the G sums in the lanes' shuffle order, so both
        // kernels give the same bits.
        const int G = c->A.lanes_per_row;
        const long long RE = kThreads;
        const long long etiles = (n + RE - 1) / RE;
        const char *ell_env = getenv("PPG_SPMV_ELL");  // 0: no tile-ELL copy (the windowed CSR kernel runs)
        const bool ell_on = !ell_env || atoi(ell_env) != 0;
        // L2 reuse between consecutive passes over the same data (0 turns each off)
        const char *alt_env = getenv("PPG_SPMV_ALTERNATE");
        c->spmv_alternate = alt_env ? atoi(alt_env) : 1;
        const char *galt_env = getenv("PPG_GS_ALTERNATE");
        c->gs_alternate = galt_env ? atoi(galt_env) : 1;
        std::vector<int> edesc;
        std::vector<short> elidx;
        long long exmax = 0, ewindowed = -1;
        if (ell_on && (G == 1 || G == 2 || G == 4) && spmv_rows_per_thread() == 1)
            ewindowed = make_windows(hcol, RE, kEWin, edesc, elidx, &exmax);
        if (ewindowed == etiles) {
            std::vector<double> hval(nnz);
            PPG_CK(cudaMemcpy(hval.data(), c->d_vals, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
            std::vector<int> toff(etiles + 1, 0);
            int wmax = 0;
            for (long long t = 0; t < etiles; ++t) {
                const long long r0 = t * RE, r1 = std::min<long long>(n, r0 + RE);
                int wt = 0;
                for (long long r = r0; r < r1; ++r) wt = std::max(wt, hrp[r + 1] - hrp[r]);
                wt = (wt + G - 1) / G * G;
                wmax = std::max(wmax, wt);
                if ((long long)toff[t] + RE * wt >= (1LL << 31) - 64) {
                    wmax = -1;
                    break;
                }
                toff[t + 1] = toff[t] + (int)(RE * wt);
            }
            if (wmax > 0 && wmax <= kEllWidthMax) {
                const size_t total = (size_t)toff[etiles];
                std::vector<float> ev(total + 16, 0.0f);
                std::vector<double> ev64(total + 16, 0.0);
                std::vector<short> ei(total + 16, (short)exmax);
                for (long long t = 0; t < etiles; ++t) {
                    const long long r0 = t * RE, r1 = std::min<long long>(n, r0 + RE);
                    for (long long r = r0; r < r1; ++r)
                        for (int k = 0; k < hrp[r + 1] - hrp[r]; ++k) {
                            const size_t e = (size_t)toff[t] + (size_t)k * RE + (size_t)(r - r0);
                            ev[e] = (float)hval[hrp[r] + k];
                            ev64[e] = hval[hrp[r] + k];
                            ei[e] = elidx[hrp[r] + k];
                        }
                }
                // float32 values and their indices in one allocation (one L2 residency window)
                const size_t vbytes = (size_t)round_up((long long)(sizeof(float) * ev.size()), 256);
                const size_t ebytes = vbytes + sizeof(short) * ei.size();
                char *blk = nullptr;
                PPG_CK(cudaMalloc(&blk, ebytes));
                c->d_evals = reinterpret_cast<float *>(blk);
                c->d_eidx = reinterpret_cast<short *>(blk + vbytes);
                PPG_CK(cudaMemcpy(c->d_evals, ev.data(), sizeof(float) * ev.size(), cudaMemcpyHostToDevice));
                PPG_CK(cudaMemcpy(c->d_eidx, ei.data(), sizeof(short) * ei.size(), cudaMemcpyHostToDevice));
                PPG_CK(cudaMalloc(&c->d_evals64, sizeof(double) * ev64.size()));
                PPG_CK(cudaMemcpy(c->d_evals64, ev64.data(), sizeof(double) * ev64.size(), cudaMemcpyHostToDevice));
                l2_residency(c, blk, ebytes);
                PPG_CK(cudaMalloc(&c->d_toff, sizeof(int) * toff.size()));
                PPG_CK(cudaMemcpy(c->d_toff, toff.data(), sizeof(int) * toff.size(), cudaMemcpyHostToDevice));
                PPG_CK(cudaMalloc(&c->d_etwin, sizeof(int) * edesc.size()));
                PPG_CK(cudaMemcpy(c->d_etwin, edesc.data(), sizeof(int) * edesc.size(), cudaMemcpyHostToDevice));
                c->A.etwin = c->d_etwin;
                c->A.evals = c->d_evals;
                c->A.evals64 = c->d_evals64;
                c->A.eidx = c->d_eidx;
                c->A.toff = c->d_toff;
                c->A.ewmax = wmax;
                c->A.excap = (int)exmax;
            }
        }
    }
    PPG_CK(spmv_configure(&c->A));
    // the allocation-free apply's scratch: its module data is mapped here, where the context allocates
    // anyway, so that ppg_apply_poly_noalloc itself maps nothing
    if (n <= kNoAllocMaxN) PPG_TRY(noalloc_scratch(c->device, &c->noalloc_base));

    // sliced ELL copy: 32-row slices padded to their longest row (selectable with ppg_spmv_format)
    {
        const long long ns = (n + 31) / 32;
        std::vector<int> hsp(ns + 1, 0);
        long long pos = 0;
        bool fits = true;
        for (long long sl = 0; sl < ns; ++sl) {
            int w = 0;
            for (long long r = sl * 32; r < std::min<long long>(n, sl * 32 + 32); ++r) w = std::max(w, hrp[r + 1] - hrp[r]);
            pos += 32LL * w;
            if (pos >= (1LL << 31) - 64) {
                fits = false;
                break;
            }
            hsp[sl + 1] = (int)pos;
        }
        if (fits && nnz > 0) {
            PPG_CK(cudaMalloc(&c->d_sptr, sizeof(int) * (ns + 1)));
            PPG_CK(cudaMemcpy(c->d_sptr, hsp.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice));
            PPG_CK(cudaMalloc(&c->d_svals64, sizeof(double) * std::max<long long>(pos, 1)));
            if (c->d_coloff)
                PPG_CK(cudaMalloc(&c->d_soff, sizeof(short) * std::max<long long>(pos, 1)));
            else
                PPG_CK(cudaMalloc(&c->d_scol, sizeof(int) * std::max<long long>(pos, 1)));
            PPG_CK(launch_sell_fill((int)n, (int)ns, c->d_rowptr, c->d_colidx, c->d_vals, c->d_sptr, c->d_soff,
                                    c->d_scol, c->d_svals64, c->stream));
            c->A.nslices = (int)ns;
            c->A.sptr = c->d_sptr;
            c->A.soff = c->d_soff;
            c->A.scol = c->d_scol;
            c->A.svals64 = c->d_svals64;
            c->A.spadded = pos;
        }
        c->A.format = (c->A.twin || c->A.evals) ? kFmtCsrStaged : kFmtCsr;
    }
    PPG_CK(gs_configure());
    PPG_CK(gram_configure());

    *out = c;
    c = nullptr;  // release from the guard
    return PPG_OK;
}

void ppg_destroy(ppg_ctx *c)
{
    if (!c) return;
    if (c->tctx) ppg_destroy(c->tctx);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    cudaFree(c->d_rowptr);
    cudaFree(c->d_colidx);
    cudaFree(c->d_coloff);
    cudaFree(c->d_vals);
    cudaFree(c->d_vals32);
    for (ppg_ctx::IterGraph &g : c->igraphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    cudaFree(c->d_rounds);
    cudaFree(c->d_twin);
    cudaFree(c->d_lidx);
    cudaFree(c->d_evals);  // also holds d_eidx
    cudaFree(c->d_lu64);
    cudaFree(c->d_lu32);
    cudaFree(c->d_ilu_diag);
    cudaFree(c->d_ilu_rd64);
    cudaFree(c->d_ilu_rd32);
    cudaFree(c->d_lorder);
    cudaFree(c->d_uorder);
    cudaFree(c->d_ilu_abort);
    cudaFree(c->ilu_vec);
    cudaFree(c->d_toff);
    cudaFree(c->d_etwin);
    cudaFree(c->d_evals64);
    cudaFree(c->d_sptr);
    cudaFree(c->d_soff);
    cudaFree(c->d_scol);
    cudaFree(c->d_svals64);
    cudaFree(c->d_svals32);
    cudaFree(c->st);
    cudaFree(c->d_sstep);
    cudaFree(c->d_bgs_partials);
    cudaFree(c->d_small);
    cudaFree(c->d_info);
    if (c->ws_owned) cudaFree(c->ws);
    cudaFreeHost(c->h_st);
    cudaFreeHost(c->h_info);
    cudaFreeHost(c->h_small);
    cudaFreeHost(c->h_prog);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
    delete c;
}

ppg_status ppg_spmv_format(ppg_ctx *c, int request, int *in_effect)
{
    g_last_error.clear();
    if (!c) return fail(PPG_ERR_INVALID_ARG, "null context");
    switch (request) {
    case PPG_SPMV_QUERY: break;
    case PPG_SPMV_AUTO: c->A.format = (c->A.twin || c->A.evals) ? kFmtCsrStaged : kFmtCsr; break;
    case PPG_SPMV_CSR: c->A.format = kFmtCsr; break;
    case PPG_SPMV_SELL:
        if (c->A.nslices == 0) return fail(PPG_ERR_INVALID_ARG, "no sliced ELL copy for this matrix");
        c->A.format = kFmtSell;
        break;
    case PPG_SPMV_STAGED:
        if (!c->A.twin && !c->A.evals) return fail(PPG_ERR_INVALID_ARG, "no x windows for this matrix");
        c->A.format = kFmtCsrStaged;
        break;
    default: return fail(PPG_ERR_INVALID_ARG, "unknown SpMV format request %d", request);
    }
    if (in_effect)
        *in_effect = c->A.format == kFmtSell ? PPG_SPMV_SELL : c->A.format == kFmtCsrStaged ? PPG_SPMV_STAGED : PPG_SPMV_CSR;
    return PPG_OK;
}

ppg_status ppg_chain_fusion(ppg_ctx *c, int request, int *in_effect)
{
    g_last_error.clear();
    if (!c) return fail(PPG_ERR_INVALID_ARG, "null context");
    if (request != -1 && request != 0 && request != 1) return fail(PPG_ERR_INVALID_ARG, "request must be -1, 0 or 1");
    if (request >= 0) c->fuse = request;
    if (in_effect) *in_effect = (c->fuse && chain_pairs(c->A, kF32, c->d_rounds != nullptr)) ? 1 : 0;
    return PPG_OK;
}

ppg_status ppg_set_stream(ppg_ctx *c, void *stream)
{
    PPG_TRY(check_ctx(c));
    c->stream = (cudaStream_t)stream;
    if (c->tctx) c->tctx->stream = c->stream;
    return PPG_OK;
}

ppg_status ppg_workspace_bytes(const ppg_ctx *c, int restart, int degree, int precision, size_t *bytes)
{
    (void)precision;
    PPG_TRY(check_ctx(c));
    if (!bytes || restart < 1 || restart > kKmax - 1 || degree < -1 || degree > kSmallMax - 2)
        return fail(PPG_ERR_INVALID_ARG, "bad restart, degree or null output");
    const int d = degree < 0 ? 30 : degree;
    *bytes = layout_bytes(c, std::max(restart + 1, d + 2));
    return PPG_OK;
}

ppg_status ppg_set_workspace(ppg_ctx *c, void *ws, size_t bytes)
{
    PPG_TRY(check_ctx(c));
    PPG_TRY(set_device(c));
    if (c->ws_owned && c->ws) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->ws);
    }
    if (ws) {
        if (((uintptr_t)ws & 255) != 0) return fail(PPG_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        c->ws = (char *)ws;
        c->ws_bytes = bytes;
        c->ws_owned = false;
    } else {
        c->ws = nullptr;
        c->ws_bytes = 0;
        c->ws_owned = true;
    }
    return PPG_OK;
}

ppg_status ppg_spmv(ppg_ctx *c, const void *x, void *y, int precision)
{
    PPG_TRY(check_ctx(c));
    if (!x || !y) return fail(PPG_ERR_INVALID_ARG, "null vector");
    if (precision != PPG_F64 && precision != PPG_F32) return fail(PPG_ERR_INVALID_ARG, "unknown precision");
    PPG_TRY(set_device(c));
    if (precision == PPG_F32) PPG_TRY(ensure_f32(c));
    Exec ex{c, &c->A, precision, c->stream};
    ex.plain = true;  // A itself, also with ILU(0) on
    SpmvEpi e = epi_none();
    e.x = vfix(x);
    e.out0 = vfix(y);
    e.a0 = simm(1.0);
    return ex.spmv(e, kNoCheck);
}

ppg_status ppg_build_poly(ppg_ctx *c, int degree, int basis, const double *v0, uint64_t seed, int *degree_used)
{
    PPG_TRY(check_ctx(c));
    if (degree < -1 || degree > kSmallMax - 2) return fail(PPG_ERR_INVALID_ARG, "degree must be in [-1, 62]");
    if (basis != PPG_BASIS_POWER && basis != PPG_BASIS_ROOTS) return fail(PPG_ERR_INVALID_ARG, "unknown basis");
    PPG_TRY(set_device(c));
    if (c->ilu_on) PPG_CK(cudaMemsetAsync(c->d_ilu_abort, 0, sizeof(int), c->stream));
    const bool autodeg = degree < 0;
    int deg = autodeg ? 30 : degree;
    Layout L;
    PPG_TRY(get_layout(c, std::max(deg + 2, 2), sizeof(double), &L));
    double *b0 = (double *)L.basis;
    if (v0) {
        PPG_CK(launch_copy_in(c->A.n, kF64, v0, b0, c->stream));
    } else {
        PPG_CK(launch_fill_uniform(b0, c->A.n, seed, c->stream));
    }
    c->launches++;
    ppg_status status = PPG_OK;
    int used = 0, info = 0;
    if (basis == PPG_BASIS_POWER || autodeg) {
        PPG_TRY(build_power(c, deg, L, &used, &info));
        if (!autodeg && used < deg) status = PPG_WARN_DEGREE_CLAMPED;
        deg = used;
    }
    if (basis == PPG_BASIS_ROOTS) {
        if (autodeg) {  // the power build overwrote nothing but columns 1..; column 0 still holds v0
        }
        PPG_TRY(build_roots(c, deg, L, &used));
    }
    if (degree_used) *degree_used = used;
    return status;
}

ppg_status ppg_set_poly(ppg_ctx *c, int basis, int degree, const double *coef_h)
{
    PPG_TRY(check_ctx(c));
    if (degree < 0 || degree > kSmallMax - 2 || !coef_h) return fail(PPG_ERR_INVALID_ARG, "bad degree or null data");
    if (basis == PPG_BASIS_POWER) {
        for (int i = 0; i <= degree; ++i)
            if (!std::isfinite(coef_h[i])) return fail(PPG_ERR_POLY_BREAKDOWN, "non-finite coefficient");
        c->coef.assign(coef_h, coef_h + degree + 1);
        c->roots.clear();
        c->table.clear();
    } else if (basis == PPG_BASIS_ROOTS) {
        const int k = degree + 1;
        std::vector<double> r(coef_h, coef_h + 2 * k), t(2 * k, 0.0);
        for (int i = 0; i < k; ++i) {
            const double re = r[2 * i], im = r[2 * i + 1];
            if (!std::isfinite(re) || !std::isfinite(im) || (re == 0.0 && im == 0.0))
                return fail(PPG_ERR_POLY_BREAKDOWN, "zero or non-finite root");
            if (im != 0.0) {
                if (i + 1 >= k || r[2 * i + 2] != re || r[2 * i + 3] != -im || im < 0.0)
                    return fail(PPG_ERR_INVALID_ARG, "a complex root (im > 0) must be followed by its conjugate");
                ++i;  // the conjugate partner was checked with it
            }
        }
        PPG_TRY(set_device(c));
        PPG_CK(cudaMemcpyAsync(c->d_small, r.data(), sizeof(double) * 2 * k, cudaMemcpyHostToDevice, c->stream));
        PPG_CK(launch_root_table(k, c->d_small, c->d_small + 2 * kKmax, c->d_info, c->stream));
        PPG_CK(cudaMemcpyAsync(c->h_small, c->d_small + 2 * kKmax, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost,
                               c->stream));
        PPG_CK(cudaMemcpyAsync(c->h_info, c->d_info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PPG_CK(cudaStreamSynchronize(c->stream));
        if (c->h_info[0]) return fail(PPG_ERR_POLY_BREAKDOWN, "zero or non-finite root");
        t.assign(c->h_small, c->h_small + 2 * k);
        c->roots = r;
        c->table = t;
        c->coef.clear();
    } else {
        return fail(PPG_ERR_INVALID_ARG, "unknown basis");
    }
    c->basis = basis;
    c->degree = degree;
    c->poly_resid = NAN;
    c->has_poly = 1;
    return PPG_OK;
}

ppg_status ppg_get_poly(ppg_ctx *c, int *basis, int *degree, double *coef_h, int cap, double *resid_h)
{
    PPG_TRY(check_ctx(c));
    if (!c->has_poly) return fail(PPG_ERR_NO_POLY, "no polynomial has been built or set");
    if (basis) *basis = c->basis;
    if (degree) *degree = c->degree;
    if (resid_h) *resid_h = c->poly_resid;
    if (coef_h) {
        const std::vector<double> &v = c->basis == PPG_BASIS_POWER ? c->coef : c->roots;
        if ((size_t)cap < v.size()) return fail(PPG_ERR_INVALID_ARG, "capacity %d < %zu", cap, v.size());
        std::copy(v.begin(), v.end(), coef_h);
    }
    return PPG_OK;
}

ppg_status ppg_set_left_ilu0(ppg_ctx *c, int enable, double *lu_out)
{
    PPG_TRY(check_ctx(c));
    PPG_TRY(set_device(c));
    if (enable && !c->d_lu64) {
        const long long n = c->A.n, nnz = c->A.nnz;
        std::vector<int> rp(n + 1), ci(nnz > 0 ? nnz : 1);
        PPG_CK(cudaMemcpy(rp.data(), c->d_rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
        if (nnz > 0) PPG_CK(cudaMemcpy(ci.data(), c->d_colidx, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
        // the pattern: sorted rows, every diagonal present; levels of the two triangles' dependencies
        std::vector<int> diag(n), llev(n, 0), ulev(n, 0);
        int lmax = 0, umax = 0;
        for (long long i = 0; i < n; ++i) {
            diag[i] = -1;
            int lv = 0;
            for (int t = rp[i]; t < rp[i + 1]; ++t) {
                if (t > rp[i] && ci[t] <= ci[t - 1])
                    return fail(PPG_ERR_INVALID_ARG, "ILU(0) needs the columns of every row sorted (row %lld)", i);
                if (ci[t] == i) diag[i] = t;
                if (ci[t] < i) lv = std::max(lv, llev[ci[t]] + 1);
            }
            if (diag[i] < 0) return fail(PPG_ERR_INVALID_ARG, "ILU(0) needs every diagonal entry (row %lld)", i);
            llev[i] = lv;
            lmax = std::max(lmax, lv);
        }
        for (long long i = n - 1; i >= 0; --i) {
            int lv = 0;
            for (int t = diag[i] + 1; t < rp[i + 1]; ++t) lv = std::max(lv, ulev[ci[t]] + 1);
            ulev[i] = lv;
            umax = std::max(umax, lv);
        }
        auto sort_by = [&](const std::vector<int> &lev, int nl, std::vector<int> &order, std::vector<int> &start) {
            start.assign(nl + 2, 0);
            for (long long i = 0; i < n; ++i) start[lev[i] + 1]++;
            for (int l = 0; l <= nl; ++l) start[l + 1] += start[l];
            std::vector<int> fill(start.begin(), start.end() - 1);
            order.resize(n);
            for (long long i = 0; i < n; ++i) order[fill[lev[i]]++] = (int)i;
        };
        std::vector<int> lorder, lstart, uorder, ustart;
        sort_by(llev, lmax, lorder, lstart);
        sort_by(ulev, umax, uorder, ustart);
        PPG_CK(cudaMalloc(&c->d_lu64, sizeof(double) * (nnz + 1)));
        PPG_CK(cudaMalloc(&c->d_lu32, sizeof(float) * (nnz + 1)));
        PPG_CK(cudaMalloc(&c->d_ilu_diag, sizeof(int) * n));
        PPG_CK(cudaMalloc(&c->d_lorder, sizeof(int) * n));
        PPG_CK(cudaMalloc(&c->d_uorder, sizeof(int) * n));
        PPG_CK(cudaMalloc(&c->d_ilu_abort, sizeof(int)));
        PPG_CK(cudaMalloc(&c->ilu_vec, sizeof(double) * 5 * c->ld));
        PPG_CK(cudaMemcpy(c->d_ilu_diag, diag.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        PPG_CK(cudaMemcpy(c->d_lorder, lorder.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        PPG_CK(cudaMemcpy(c->d_uorder, uorder.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        PPG_CK(cudaMemset(c->d_ilu_abort, 0, sizeof(int)));
        PPG_CK(cudaMemset(c->ilu_vec, 0, sizeof(double) * 5 * c->ld));
        // factorisation on the device, one launch per level of the lower triangle
        if (nnz > 0) PPG_CK(cudaMemcpyAsync(c->d_lu64, c->d_vals, sizeof(double) * nnz, cudaMemcpyDeviceToDevice,
                                            c->stream));
        for (int l = 0; l <= lmax; ++l)
            PPG_CK(launch_ilu0_level(c->d_lorder + lstart[l], lstart[l + 1] - lstart[l], c->d_rowptr, c->d_colidx,
                                     c->d_ilu_diag, c->d_lu64, c->stream));
        if (nnz > 0) PPG_CK(launch_ilu_cast(c->d_lu64, c->d_lu32, nnz, c->stream));
        // pivots: U's diagonal must be finite and non-zero
        std::vector<double> lu(nnz > 0 ? nnz : 1);
        if (nnz > 0)
            PPG_CK(cudaMemcpyAsync(lu.data(), c->d_lu64, sizeof(double) * nnz, cudaMemcpyDeviceToHost, c->stream));
        PPG_CK(cudaStreamSynchronize(c->stream));
        std::vector<double> rd64(n);
        std::vector<float> rd32(n);
        for (long long i = 0; i < n; ++i) {
            const double d = lu[diag[i]];
            if (!(d != 0.0) || !std::isfinite(d)) {
                cudaFree(c->d_lu64);
                c->d_lu64 = nullptr;
                return fail(PPG_ERR_POLY_BREAKDOWN, "ILU(0) breaks down: pivot %lld is %g", i, d);
            }
            rd64[i] = 1.0 / d;
            rd32[i] = (float)rd64[i];
        }
        PPG_CK(cudaMalloc(&c->d_ilu_rd64, sizeof(double) * n));
        PPG_CK(cudaMalloc(&c->d_ilu_rd32, sizeof(float) * n));
        PPG_CK(cudaMemcpy(c->d_ilu_rd64, rd64.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        PPG_CK(cudaMemcpy(c->d_ilu_rd32, rd32.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
        int longest = 1;
        for (long long i = 0; i < n; ++i) longest = std::max(longest, rp[i + 1] - rp[i]);
        c->ilu_red = 1;
        while (c->ilu_red < longest && c->ilu_red < 32) c->ilu_red *= 2;
    }
    const int on = enable ? 1 : 0;
    if (on != c->ilu_on) {
        c->ilu_on = on;
        c->has_poly = 0;  // a polynomial belongs to its operator (A, or M^{-1} A): build it again
    }
    if (lu_out && c->d_lu64)
        PPG_CK(cudaMemcpyAsync(lu_out, c->d_lu64, sizeof(double) * c->A.nnz, cudaMemcpyDeviceToDevice, c->stream));
    PPG_CK(cudaStreamSynchronize(c->stream));
    return PPG_OK;
}

ppg_status ppg_apply_poly(ppg_ctx *c, const void *v, void *out, int precision)
{
    PPG_TRY(check_ctx(c));
    if (!v || !out) return fail(PPG_ERR_INVALID_ARG, "null vector");
    if (precision != PPG_F64 && precision != PPG_F32) return fail(PPG_ERR_INVALID_ARG, "unknown precision");
    if (!c->has_poly) return fail(PPG_ERR_NO_POLY, "no polynomial has been built or set");
    PPG_TRY(set_device(c));
    if (precision == PPG_F32) PPG_TRY(ensure_f32(c));
    if (c->ilu_on) PPG_CK(cudaMemsetAsync(c->d_ilu_abort, 0, sizeof(int), c->stream));
    const size_t es = precision == PPG_F64 ? 8 : 4;
    Layout L;
    PPG_TRY(get_layout(c, 1, es, &L));
    PPG_TRY(init_cycle_state(c, 0, 1, 1, 0.0, 0.0));
    PPG_CK(launch_copy_in(c->A.n, precision, v, L.vec[0], c->stream));
    Exec ex{c, &c->A, precision, c->stream};
    char *tmp[3] = {L.vec[2], L.vec[3], L.vec[4]};
    PPG_TRY(ex.poly_apply(vfix(L.vec[0]), nullptr, vfix(L.vec[1]), tmp, kNoCheck));
    PPG_CK(launch_copy_in(c->A.n, precision, L.vec[1], out, c->stream));
    return PPG_OK;
}

ppg_status ppg_apply_poly_noalloc(ppg_ctx *c, const void *v, void *out, int precision)
{
    PPG_TRY(check_ctx(c));
    if (!v || !out) return fail(PPG_ERR_INVALID_ARG, "null vector");
    if (precision != PPG_F64 && precision != PPG_F32) return fail(PPG_ERR_INVALID_ARG, "unknown precision");
    if (!c->has_poly) return fail(PPG_ERR_NO_POLY, "no polynomial has been built or set");
    if (c->ilu_on)
        return fail(PPG_ERR_INVALID_ARG, "ppg_apply_poly_noalloc does not apply ILU(0): turn it off or use ppg_apply_poly");
    if (c->A.n > kNoAllocMaxN)
        return fail(PPG_ERR_INVALID_ARG,
                    "ppg_apply_poly_noalloc handles at most %lld rows (n = %d); use ppg_apply_poly", kNoAllocMaxN,
                    c->A.n);
    if (precision == PPG_F32 && !c->d_vals32)
        return fail(PPG_ERR_INVALID_ARG,
                    "the float32 copy of the matrix does not exist yet and this call may not allocate it: make one "
                    "float32 ppg_spmv, ppg_apply_poly or ppg_solve call first");
    PPG_TRY(set_device(c));
    char *base = c->noalloc_base;  // looked up by ppg_create
    if (!base) PPG_TRY(noalloc_scratch(c->device, &base));
    char *vec[kNoAllocVecs];
    for (int i = 0; i < kNoAllocVecs; ++i) vec[i] = base + (size_t)i * kNoAllocMaxN * sizeof(double);
    PPG_CK(launch_copy_in(c->A.n, precision, v, vec[0], c->stream));
    Exec ex{c, &c->A, precision, c->stream};
    char *tmp[3] = {vec[2], vec[3], vec[4]};
    PPG_TRY(ex.poly_apply(vfix(vec[0]), nullptr, vfix(vec[1]), tmp, kNoCheck));
    PPG_CK(launch_copy_in(c->A.n, precision, vec[1], out, c->stream));
    return PPG_OK;
}

ppg_status ppg_solve_batched(int nsys, const ppg_batch_system *sys_h, int degree, double tol, int restart,
                             int maxit, uint64_t seed, void *stream, ppg_stats *per_sys)
{
    g_last_error.clear();
    if (nsys < 1 || !sys_h) return fail(PPG_ERR_INVALID_ARG, "need at least one system");
    if (restart < 1 || restart > kBatchMaxRestart)
        return fail(PPG_ERR_INVALID_ARG, "batched restart must be in [1, %d]", kBatchMaxRestart);
    if (degree < 0 || degree > kBatchMaxDegree)
        return fail(PPG_ERR_INVALID_ARG, "batched degree must be in [0, %d]", kBatchMaxDegree);
    if (maxit < 0 || !(tol >= 0.0)) return fail(PPG_ERR_INVALID_ARG, "bad tol or maxit");
    for (int i = 0; i < nsys; ++i) {
        const ppg_batch_system &q = sys_h[i];
        if (q.n < 1 || q.n >= (1LL << 31) - 256 || q.nnz < 0 || !q.rowptr || !q.b || !q.x ||
            (q.nnz > 0 && (!q.colidx || !q.vals)))
            return fail(PPG_ERR_INVALID_ARG, "system %d: bad sizes or null pointers", i);
    }
    int dev = 0;
    PPG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(PPG_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchCache &bc = g_batch[dev];
    PPG_TRY(batch_setup(bc, nsys));
    cudaStream_t us = (cudaStream_t)stream;

    // workspace: float32 values, float32 basis and work vectors, float64 construction basis
    std::vector<size_t> off(nsys);
    size_t total = 0;
    long long total_nnz = 0, total_n = 0;
    for (int i = 0; i < nsys; ++i) {
        const long long n = sys_h[i].n, nnz = sys_h[i].nnz;
        off[i] = total;
        total += align256(sizeof(float) * (nnz + 8)) + align256(sizeof(float) * n * (restart + 1)) +
                 align256(sizeof(float) * n * restart) + align256(sizeof(float) * n * 6) +
                 align256(sizeof(double) * n * (degree + 2)) + align256(sizeof(double) * n) +
                 align256(sizeof(double) * n);
        total_nnz += nnz;
        total_n += n;
    }
    if (total > bc.ws_bytes) {
        cudaFree(bc.ws);
        bc.ws = nullptr;
        bc.ws_bytes = 0;
        PPG_CK(cudaMalloc(&bc.ws, total));
        bc.ws_bytes = total;
    }
    std::vector<BatchSys> hs(nsys);
    std::vector<double *> xscratch(nsys);
    for (int i = 0; i < nsys; ++i) {
        const ppg_batch_system &q = sys_h[i];
        BatchSys &d = hs[i];
        char *p = bc.ws + off[i];
        d.n = (int)q.n;
        d.nnz = (int)q.nnz;
        d.rowptr = q.rowptr;
        d.colidx = q.colidx;
        d.vals64 = q.vals;
        d.b = q.b;
        d.x = q.x;
        d.vals32 = reinterpret_cast<float *>(p);
        p += align256(sizeof(float) * (q.nnz + 8));
        d.V = reinterpret_cast<float *>(p);
        p += align256(sizeof(float) * q.n * (restart + 1));
        d.Z = reinterpret_cast<float *>(p);
        p += align256(sizeof(float) * q.n * restart);
        d.fw = reinterpret_cast<float *>(p);
        p += align256(sizeof(float) * q.n * 6);
        d.V64 = reinterpret_cast<double *>(p);
        p += align256(sizeof(double) * q.n * (degree + 2));
        d.dw = reinterpret_cast<double *>(p);
        p += align256(sizeof(double) * q.n);
        xscratch[i] = reinterpret_cast<double *>(p);  // x of the tuning runs
        d.lanes = 1;
    }
    // largest systems first: the hardware then fills idle SMs with the smaller ones
    std::vector<int> order(nsys);
    for (int i = 0; i < nsys; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sys_h[a].nnz > sys_h[b].nnz; });

    PPG_CK(cudaEventRecord(bc.ev_in, us));
    PPG_CK(cudaStreamWaitEvent(bc.stream, bc.ev_in, 0));
    PPG_CK(cudaMemcpyAsync(bc.sys_d, hs.data(), sizeof(BatchSys) * nsys, cudaMemcpyHostToDevice, bc.stream));
    PPG_CK(cudaMemcpyAsync(bc.order_d, order.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, bc.stream));
    PPG_CK(launch_batch_cast(bc.sys_d, nsys, bc.stream));

    // flexible float32 form with the restart projection (as ppg_solve's default), inner tolerance 1e-7
    BatchParams prm{degree, restart, (long long)maxit, tol, 1e-7, (unsigned long long)seed, 1};

    // autotuner, once per batch shape, on this very batch with x in scratch memory: the cluster size
    // (CTAs per system, i.e. the rows of each CTA) by timing whole solves -- the launch ends with its
    // slowest system, whose iterations a short run does not show -- then, per size class of rows per
    // CTA, the SpMV's threads per row by timing short solves (construction and half a cycle)
    std::vector<long long> shape;
    {
        std::vector<std::pair<long long, long long>> sh(nsys);
        for (int i = 0; i < nsys; ++i) sh[i] = {sys_h[i].n, sys_h[i].nnz};
        std::sort(sh.begin(), sh.end());
        for (const auto &q : sh) {
            shape.push_back(q.first);
            shape.push_back(q.second);
        }
        shape.push_back(degree);
        shape.push_back(restart);
    }
    auto cls_of = [](long long n, int cluster) {
        const long long rpc = (n + cluster - 1) / cluster;
        return rpc < kThreads ? 0 : (rpc < 8 * kThreads ? 1 : 2);
    };
    auto cluster_of = [&](int i, const BatchCache::Tuned &t) {
        return (t.big_rows > 0 && sys_h[i].n < t.big_rows) ? t.cluster2 : t.cluster;
    };
    // the systems of ord with the large ones (>= big_rows) first, each part in ord's order; returns
    // how many are large
    auto arrange = [&](const std::vector<int> &ord, long long big_rows, std::vector<int> &out) {
        out.clear();
        if (big_rows <= 0) {
            out = ord;
            return (int)ord.size();
        }
        for (int i : ord)
            if (sys_h[i].n >= big_rows) out.push_back(i);
        const int split = (int)out.size();
        for (int i : ord)
            if (sys_h[i].n < big_rows) out.push_back(i);
        return split;
    };
    // the launch(es) of a batch arranged as above: the first `split` systems in clusters of c1 on s1, the
    // rest in clusters of c2 on the second stream, joined back into s1
    auto launch_arranged = [&](const BatchSys *sysd, const int *ordd, int cnt, int split, int c1, int c2,
                               const BatchParams &pp, cudaStream_t s1, int t1) -> cudaError_t {
        if (split >= cnt) return launch_batch(sysd, ordd, cnt, c1, pp, bc.out_d, s1, t1);
        if (split <= 0) return launch_batch(sysd, ordd, cnt, c2, pp, bc.out_d, s1);
        cudaError_t e = cudaEventRecord(bc.ev_fork, s1);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(bc.stream2, bc.ev_fork, 0);
        if (e == cudaSuccess) e = launch_batch(sysd, ordd, split, c1, pp, bc.out_d, s1, t1);
        if (e == cudaSuccess) e = launch_batch(sysd, ordd + split, cnt - split, c2, pp, bc.out_d, bc.stream2);
        if (e == cudaSuccess) e = cudaEventRecord(bc.ev_join, bc.stream2);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s1, bc.ev_join, 0);
        return e;
    };
    // PPG_BATCH_CONFIG="cluster,cluster2,big_rows[,threads]" in the environment fixes the configuration
    // (threads per row: 2 for fewer than 256 rows per CTA, else 1) instead of tuning it; for tests and
    // measurements
    BatchCache::Tuned forced;
    if (const char *env = getenv("PPG_BATCH_CONFIG")) {
        long long c1 = 0, c2 = 0, big = 0, nt = 256;
        const int got = sscanf(env, "%lld,%lld,%lld,%lld", &c1, &c2, &big, &nt);
        auto size_ok = [](long long c) { return c == 1 || c == 2 || c == 4 || c == 8 || c == 16; };
        if (got < 3 || !size_ok(c1) || !size_ok(c2) || big < 0 || (nt != 256 && nt != 512))
            return fail(PPG_ERR_INVALID_ARG, "PPG_BATCH_CONFIG must be \"cluster,cluster2,big_rows[,threads]\" "
                                             "with cluster sizes 1, 2, 4, 8 or 16 and 256 or 512 threads");
        forced.cluster = (int)c1;
        forced.cluster2 = big > 0 ? (int)c2 : (int)c1;
        forced.big_rows = big;
        forced.threads = (int)nt;
        for (int c = 0; c < 3; ++c) forced.lanes[c] = c == 0 ? 2 : 1;
    }
    auto it_t = forced.cluster ? bc.tuned.end() : bc.tuned.find(shape);
    if (!forced.cluster && it_t == bc.tuned.end()) {
        BatchCache::Tuned tb;
        std::vector<BatchSys> ht = hs;
        for (int i = 0; i < nsys; ++i) ht[i].x = xscratch[i];
        BatchParams tp = prm;
        const long long short_maxit = std::max(1, std::min(maxit, std::max(1, restart / 2)));
        // one timed solve of the systems listed in ord (x reset to the caller's x0 first) in the
        // configuration t, with the threads per row already set in ht
        std::vector<int> arranged;
        auto timed = [&](const std::vector<int> &ord, const BatchCache::Tuned &t, int reps, float *ms) -> ppg_status {
            const int split = arrange(ord, t.big_rows, arranged);
            PPG_CK(cudaMemcpyAsync(bc.tune_d, ht.data(), sizeof(BatchSys) * nsys, cudaMemcpyHostToDevice, bc.stream));
            PPG_CK(cudaMemcpyAsync(bc.tune_order_d, arranged.data(), sizeof(int) * arranged.size(),
                                   cudaMemcpyHostToDevice, bc.stream));
            float best = 0.f;
            for (int rep = 0; rep < reps; ++rep) {  // short runs: the first one also warms caches
                for (int i : ord)
                    PPG_CK(cudaMemcpyAsync(xscratch[i], sys_h[i].x, sizeof(double) * sys_h[i].n,
                                           cudaMemcpyDeviceToDevice, bc.stream));
                PPG_CK(cudaEventRecord(bc.t0, bc.stream));
                PPG_CK(launch_arranged(bc.tune_d, bc.tune_order_d, (int)arranged.size(), split, t.cluster, t.cluster2,
                                       tp, bc.stream, t.threads));
                PPG_CK(cudaEventRecord(bc.t1, bc.stream));
                PPG_CK(cudaEventSynchronize(bc.t1));
                PPG_CK(cudaEventElapsedTime(&best, bc.t0, bc.t1));
            }
            *ms = best;
            return PPG_OK;
        };
        // candidates: every system in clusters of 4, 8 or 16; or the systems of at least 16384 / 65536
        // rows in clusters of 16 and the others, in a concurrent launch, in clusters of 4 or 8
        std::vector<BatchCache::Tuned> cands;
        for (int cl : {4, 8, 16}) {
            BatchCache::Tuned t;
            t.cluster = t.cluster2 = cl;
            cands.push_back(t);
        }
        // (small systems in clusters of 1 or 2 CTAs synchronise with cheaper barriers)
        for (long long big : {4096LL, 16384LL, 65536LL}) {
            int nbig = 0;
            for (int i = 0; i < nsys; ++i) nbig += sys_h[i].n >= big ? 1 : 0;
            if (nbig == 0 || nbig == nsys) continue;
            for (int c2 : {1, 2, 4, 8})
                for (int t1 : {256, 512}) {  // 512: twice the warps per large system, half the CTAs per SM
                    if (t1 == 512 && big != 65536) continue;
                    BatchCache::Tuned t;
                    t.cluster = 16;
                    t.cluster2 = c2;
                    t.big_rows = big;
                    t.threads = t1;
                    cands.push_back(t);
                }
        }
        float best_ms = 0.f;
        tp.maxit = maxit;
        for (const BatchCache::Tuned &t : cands) {
            if (batch_max_clusters(t.cluster, t.threads) < 1 || batch_max_clusters(t.cluster2) < 1) continue;
            for (int i = 0; i < nsys; ++i) ht[i].lanes = cls_of(sys_h[i].n, cluster_of(i, t)) == 0 ? 2 : 1;
            float ms = 0.f;
            PPG_TRY(timed(order, t, 1, &ms));
            if (!tb.cluster || ms < best_ms) {
                tb = t;
                best_ms = ms;
            }
        }
        if (!tb.cluster) return fail(PPG_ERR_CUDA, "no cluster size is launchable for the batched solver");
        for (int i = 0; i < nsys; ++i) ht[i].lanes = cls_of(sys_h[i].n, cluster_of(i, tb)) == 0 ? 2 : 1;
        tp.maxit = short_maxit;
        for (int c = 0; c < 3; ++c) {
            std::vector<int> sub;
            for (int i : order)
                if (cls_of(sys_h[i].n, cluster_of(i, tb)) == c) sub.push_back(i);
            if (sub.empty()) continue;
            float cbest = 0.f;
            for (int lanes : {1, 2, 4, 8}) {
                if (c == 2 && lanes > 2) continue;  // long row blocks: one or two threads per row
                for (int i : sub) ht[i].lanes = lanes;
                float ms = 0.f;
                PPG_TRY(timed(sub, tb, 2, &ms));
                if (lanes == 1 || ms < cbest) {
                    tb.lanes[c] = lanes;
                    cbest = ms;
                }
            }
            for (int i : sub) ht[i].lanes = tb.lanes[c];
        }
        it_t = bc.tuned.emplace(shape, tb).first;
    }
    const BatchCache::Tuned &tb = forced.cluster ? forced : it_t->second;
    bc.cluster = tb.cluster;
    for (int i = 0; i < nsys; ++i) hs[i].lanes = tb.lanes[cls_of(sys_h[i].n, cluster_of(i, tb))];
    std::vector<int> arranged_final;
    const int split = arrange(order, tb.big_rows, arranged_final);
    PPG_CK(cudaMemcpyAsync(bc.sys_d, hs.data(), sizeof(BatchSys) * nsys, cudaMemcpyHostToDevice, bc.stream));
    PPG_CK(cudaMemcpyAsync(bc.order_d, arranged_final.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, bc.stream));

    // the solve itself: one launch, captured once as a graph and replayed
    std::vector<long long> key = {(long long)(uintptr_t)bc.sys_d, nsys, tb.cluster, tb.cluster2, tb.big_rows,
                                  tb.threads, split, degree, restart, maxit, (long long)seed};
    double tolbits;
    memcpy(&tolbits, &tol, sizeof tol);
    key.push_back((long long)tolbits);
    if (!bc.exec || key != bc.exec_key) {
        if (bc.exec) cudaGraphExecDestroy(bc.exec);
        bc.exec = nullptr;
        cudaGraph_t graph = nullptr;
        PPG_CK(cudaStreamBeginCapture(bc.stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t le = launch_arranged(bc.sys_d, bc.order_d, nsys, split, tb.cluster, tb.cluster2, prm,
                                               bc.stream, tb.threads);
        const cudaError_t ce = cudaStreamEndCapture(bc.stream, &graph);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(PPG_ERR_CUDA, "capturing the batched launch: %s / %s", cudaGetErrorString(le),
                        cudaGetErrorString(ce));
        }
        const cudaError_t ie = cudaGraphInstantiate(&bc.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return fail(PPG_ERR_CUDA, "instantiating the batched graph: %s", cudaGetErrorString(ie));
        bc.exec_key = key;
    }
    PPG_CK(cudaEventRecord(bc.t0, bc.stream));
    PPG_CK(cudaGraphLaunch(bc.exec, bc.stream));
    PPG_CK(cudaEventRecord(bc.t1, bc.stream));
    PPG_CK(cudaEventRecord(bc.ev_out, bc.stream));
    PPG_CK(cudaStreamWaitEvent(us, bc.ev_out, 0));
    std::vector<BatchOut> ho(nsys);
    PPG_CK(cudaMemcpyAsync(ho.data(), bc.out_d, sizeof(BatchOut) * nsys, cudaMemcpyDeviceToHost, bc.stream));
    PPG_CK(cudaStreamSynchronize(bc.stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, bc.t0, bc.t1);
    ppg_status worst = PPG_OK;
    long long t_first = ho.empty() ? 0 : ho[0].t_start;
    for (const BatchOut &o : ho) t_first = std::min(t_first, o.t_start);
    for (int i = 0; i < nsys; ++i) {
        const BatchOut &o = ho[i];
        if (per_sys) {
            ppg_stats &st = per_sys[i];
            memset(&st, 0, sizeof st);
            st.iterations = o.iters;
            st.restarts = o.cycles;
            st.spmvs = o.spmvs;
            st.dots = 3 * o.iters + o.cycles + 1;
            st.kernel_launches = (i == 0) ? 1 : 0;
            st.relres_true = o.relres;
            st.relres_est = o.est;
            st.degree_used = o.degree;
            st.converged = o.converged;
            st.breakdowns = o.breakdowns;
            st.ctas_per_system = cluster_of(i, tb);
            st.spmv_lanes = hs[i].lanes;
            st.time_ms = ms;
            st.spmv_ms = (double)(o.t_end - o.t_start) * 1e-6;  // this system's own time on the device
            st.gs_ms = (double)(o.t_start - t_first) * 1e-6;     // when its cluster started in the launch
        }
        if (o.status == 2 && worst >= 0) worst = fail(PPG_ERR_NONFINITE, "system %d: non-finite value", i);
        if (o.status == 3 && worst >= 0) worst = fail(PPG_ERR_POLY_BREAKDOWN, "system %d: no usable polynomial", i);
        if (o.status == 0 && !o.converged && worst == PPG_OK) worst = PPG_ERR_NOT_CONVERGED;
    }
    return worst;
}

ppg_status ppg_solve(ppg_ctx *c, const double *b, double *x, double tol, int restart, int maxit,
                     const ppg_opts *opts, ppg_stats *stats)
{
    PPG_TRY(check_ctx(c));
    PPG_TRY(set_device(c));
    return solve_impl(c, b, x, tol, restart, maxit, opts, stats);
}

ppg_status ppg_solve_transpose(ppg_ctx *c, const double *g, double *lambda, double tol, int restart, int maxit,
                               const ppg_opts *opts, ppg_stats *stats)
{
    PPG_TRY(check_ctx(c));
    PPG_TRY(set_device(c));
    if (c->ilu_on)
        return fail(PPG_ERR_INVALID_ARG, "the transposed solve does not compose with ILU(0): turn it off first");
    if (!c->tctx) {
        int *rpT = nullptr, *ciT = nullptr, *work = nullptr;
        double *vaT = nullptr;
        const long long n = c->A.n, nnz = c->A.nnz;
        PPG_CK(cudaMalloc(&rpT, sizeof(int) * (n + 1)));
        PPG_CK(cudaMalloc(&ciT, sizeof(int) * (nnz + 1)));
        PPG_CK(cudaMalloc(&vaT, sizeof(double) * (nnz + 1)));
        PPG_CK(cudaMalloc(&work, sizeof(int) * (n + 1)));
        PPG_CK(launch_transpose(c->A, rpT, ciT, vaT, work, c->stream));
        PPG_CK(cudaStreamSynchronize(c->stream));
        ppg_status s = ppg_create(&c->tctx, n, nnz, rpT, ciT, vaT, c->stream);
        cudaFree(rpT);
        cudaFree(ciT);
        cudaFree(vaT);
        cudaFree(work);
        if (s < 0) return s;
    }
    ppg_ctx *t = c->tctx;
    t->stream = c->stream;
    // p(A^T) = p(A)^T: the same polynomial, whatever its representation
    t->has_poly = c->has_poly;
    t->basis = c->basis;
    t->degree = c->degree;
    t->coef = c->coef;
    t->roots = c->roots;
    t->table = c->table;
    t->poly_resid = c->poly_resid;
    return solve_impl(t, g, lambda, tol, restart, maxit, opts, stats);
}

ppg_status ppg_csr_outer(ppg_ctx *c, const double *u, const double *v, double alpha, double *out)
{
    PPG_TRY(check_ctx(c));
    if (!u || !v || !out) return fail(PPG_ERR_INVALID_ARG, "null vector");
    PPG_TRY(set_device(c));
    c->launches++;
    PPG_CK(launch_csr_outer(c->A, u, v, alpha, out, c->stream));
    return PPG_OK;
}

ppg_status ppg_arnoldi(ppg_ctx *c, const double *v, int k, double *V, double *H_h, int *steps)
{
    PPG_TRY(check_ctx(c));
    if (!v || k < 1 || k > kKmax - 1) return fail(PPG_ERR_INVALID_ARG, "bad start vector or k");
    PPG_TRY(set_device(c));
    Layout L;
    PPG_TRY(get_layout(c, k + 1, sizeof(double), &L));
    int done = 0;
    PPG_TRY(run_arnoldi(c, v, k, L, &done));
    if (steps) *steps = done;
    if (V) {
        Exec ex{c, &c->A, kF64, c->stream};
        for (int col = 0; col <= done; ++col) {
            SpmvEpi e = epi_none();
            e.out0 = vfix(V + (size_t)col * c->A.n);
            e.u0 = vfix(L.basis + (size_t)col * c->ld * sizeof(double));
            e.b0 = Scalar{1.0, c->st->sigma, col, 0, nullptr, 0, 0};
            PPG_TRY(ex.axpy(e, kNoCheck));
        }
    }
    if (H_h) {
        PPG_CK(cudaMemcpy2DAsync(H_h, sizeof(double) * (k + 1), c->st->H, sizeof(double) * kLdH,
                                 sizeof(double) * (k + 1), k, cudaMemcpyDeviceToHost, c->stream));
    }
    PPG_CK(cudaStreamSynchronize(c->stream));
    return PPG_OK;
}

ppg_status ppg_hessenberg_eigs(ppg_ctx *c, int k, const double *H, int ld, double *wr, double *wi)
{
    PPG_TRY(check_ctx(c));
    if (k < 1 || k > kSmallMax || ld < k || !H || !wr || !wi) return fail(PPG_ERR_INVALID_ARG, "bad arguments");
    PPG_TRY(set_device(c));
    PPG_CK(launch_hess_eigs(k, H, ld, wr, wi, c->d_info, c->stream));
    PPG_CK(cudaMemcpyAsync(c->h_info, c->d_info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PPG_CK(cudaStreamSynchronize(c->stream));
    if (c->h_info[0]) return fail(PPG_ERR_POLY_BREAKDOWN, "QR iteration did not converge");
    return PPG_OK;
}

ppg_status ppg_gram_solve(ppg_ctx *c, int degree, const double *G_h, const double *r_h, double *coef_h, int *info,
                          int *degree_used)
{
    PPG_TRY(check_ctx(c));
    if (degree < 0 || degree > kSmallMax - 2 || !G_h || !r_h || !coef_h)
        return fail(PPG_ERR_INVALID_ARG, "bad arguments (0 <= degree <= %d, non-null G, r, coef)", kSmallMax - 2);
    PPG_TRY(set_device(c));
    const int kk = degree + 1;
    double *d = nullptr;
    PPG_CK(cudaMalloc(&d, sizeof(double) * (size_t)(kk * kk + 2 * kk)));
    struct Free {
        double *p;
        ~Free() { cudaFree(p); }
    } guard{d};
    PPG_CK(cudaMemcpyAsync(d, G_h, sizeof(double) * kk * kk, cudaMemcpyHostToDevice, c->stream));
    PPG_CK(cudaMemcpyAsync(d + kk * kk, r_h, sizeof(double) * kk, cudaMemcpyHostToDevice, c->stream));
    PPG_CK(launch_gram_solve(d, d + kk * kk, degree, d + kk * kk + kk, c->d_info, c->stream));
    PPG_CK(cudaMemcpyAsync(coef_h, d + kk * kk + kk, sizeof(double) * kk, cudaMemcpyDeviceToHost, c->stream));
    PPG_CK(cudaMemcpyAsync(c->h_info, c->d_info, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
    PPG_CK(cudaStreamSynchronize(c->stream));
    if (info) *info = c->h_info[0];
    if (degree_used) *degree_used = c->h_info[1];
    if (c->h_info[1] < 0) return fail(PPG_ERR_POLY_BREAKDOWN, "the Gram matrix is not positive at degree 0");
    return c->h_info[0] ? PPG_WARN_DEGREE_CLAMPED : PPG_OK;
}

ppg_status ppg_fill_uniform(ppg_ctx *c, double *out, int64_t n, uint64_t seed)
{
    PPG_TRY(check_ctx(c));
    if (!out || n < 0) return fail(PPG_ERR_INVALID_ARG, "bad output");
    PPG_TRY(set_device(c));
    PPG_CK(launch_fill_uniform(out, n, seed, c->stream));
    return PPG_OK;
}

}  // extern "C"
