// ppg_internal.h -- host-side launch interface between the library's translation units.
#pragma once

#include "ppg_common.cuh"

#include <utility>

namespace ppg {

enum Prec : int { kF64 = 0, kF32 = 1 };

// Whether solve-path kernels are launched with programmatic stream serialization (on by
// default; PPG_NO_PDL=1 in the environment turns it off, for comparisons).
bool pdl_enabled();

// Launches kernel<<<grid, block, smem, s>>>(args...) with programmatic stream serialization
// allowed when pdl_enabled().
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// As launch_pdl, and when win_bytes > 0 the launch's global accesses to [win_base, win_base +
// win_bytes) are marked persisting in L2 for a fraction win_hit of the window (the rest streaming),
// so that data read by every launch of a chain (the float32 matrix blocks) can stay in L2 between
// launches while the vectors stream through.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_l2(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          const void *win_base, size_t win_bytes, float win_hit, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (win_bytes > 0) {
        attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[1].val.accessPolicyWindow.base_ptr = const_cast<void *>(win_base);
        attr[1].val.accessPolicyWindow.num_bytes = win_bytes;
        attr[1].val.accessPolicyWindow.hitRatio = win_hit;
        attr[1].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[1].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        cfg.numAttrs = 2;
    }
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// A launch whose CTAs wait on one another: cooperative, so that the whole grid is resident at
// once (the launch fails rather than starting part of the grid).
template <typename... KArgs, typename... Args>
cudaError_t launch_coop(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Persistent grid and pipeline depth of a tile-ELL kernel (one value type).
struct EllLaunch {
    int blocks, nst;        // one input
    int blocks_x2, nst_x2;  // with a second staged input (A (x + s2 x2))
};

// The context's device copy of the CSR matrix and the tiling chosen for it.
struct DevMatrix {
    int n;
    long long nnz;
    const int *rowptr;   // n + 1
    const int *colidx;   // nnz (+ 16 bytes of padding)
    const short *coloff; // int16 column offsets col - row (+ padding), or null when some |col - row| > 32767
    const double *vals64;
    const float *vals32;  // may be null until first needed
    int rows_per_tile;    // rows of one SpMV tile (R); R * lanes_per_row == kThreads * rows per thread
    int lanes_per_row;    // G
    int cap64, cap32;     // non-zeros one tile can stage in shared memory
    int num_sms;
    int resid_blocks;     // grid of the persistent residual / norm kernels
    int spmv_blocks64;    // persistent SpMV grids
    int spmv_blocks32;
    int spmv2_blocks64;   // persistent grids of the two-step kernel
    int spmv2_blocks32;
    int bw;               // bandwidth max |col - row|
    // x windows per tile (float32 staged kernel): kXWin (lo, len) pairs covering every column the
    // tile's rows reference, or lengths 0 when the tile's columns do not fit kXCap entries
    const int *twin;      // [ntiles][2 kXWin], or null
    const short *lidx;    // per entry: index of its column in the tile's concatenated windows
    // tile-ELL copy (one thread per row, tiles of kThreads rows, every tile windowed): tile t holds
    // entries toff[t] .. toff[t+1]-1, entry k of row l at toff[t] + k kThreads + l; padding has value 0
    // and index excap
    const float *evals;
    const short *eidx;
    const int *toff;      // tiles of kThreads rows + 1
    const int *etwin;     // x windows of those tiles: [tiles][2 kEWin] (starts, then lengths)
    int ewmax;            // widest tile (entries per row)
    int excap;            // longest window total over the tiles (the padding's zero sits at this index)
    const double *evals64; // the same blocks' values in float64 (float64 solves and the construction)
    // L2 residency of the float32 blocks (values and indices, one allocation): float32 tile-ELL launches
    // mark this window persisting for a fraction l2_hit of it; l2_bytes = 0: off
    const void *l2_base;
    size_t l2_bytes;
    float l2_hit;
    EllLaunch ell[2];     // tile-ELL grid and stages: [0] float32, [1] float64
    int spmvw_blocks32;   // persistent grid of the staged kernel
    // sliced ELL copy (slices of 32 rows; entry k of row 32 s + l at sptr[s] + 32 k + l, slices padded
    // to their longest row with a sentinel index), used by the SpMV when format == kFmtSell
    int format;           // kFmtCsr or kFmtSell
    int nslices;          // 0 when no sliced copy exists
    const int *sptr;      // nslices + 1 entry offsets
    const short *soff;    // int16 col - row, sentinel kSellPadOff; or null (then scol)
    const int *scol;      // int32 columns, sentinel -1
    const double *svals64;
    const float *svals32;  // may be null until first needed
    long long spadded;     // sptr[nslices]
};

constexpr int kFmtCsr = 0;
constexpr int kFmtSell = 1;
constexpr int kFmtCsrStaged = 2;  // row-block CSR with the tile's x windows and row operands staged by TMA
constexpr int kXWin = 4;          // x windows per tile
constexpr int kEWin = 8;          // x windows per tile of the tile-ELL kernel
constexpr int kXCap = 2048;       // x entries per tile
constexpr int kEllWidthMax = 32;  // widest tile-ELL tile (entries per row, rounded to lanes per row)
constexpr int kXGap = 64;         // columns closer than this share a window
constexpr short kSellPadOff = -32768;  // outside the int16 offsets a row may use (|col - row| <= 32767)

// Fused SpMV epilogue (one row r, Ax = (A (x + s2 x2))[r], x2 optional):
//   out0[r] = a0 * Ax + b0 * u0[r] + c0 * w0[r]
//   out1[r] = a1 * Ax + b1 * u1[r] + c1 * w1[r]      (when out1 is set)
// Null vectors drop their term.  out may alias its own u/w (same row is read then
// written) but never x or x2.
struct SpmvEpi {
    VecRef x, x2;
    VecRef out0, u0, w0;
    VecRef out1, u1, w1;
    Scalar a0, b0, c0, a1, b1, c1, s2;
    int rev;  // 1: the launch visits its row tiles last to first (tile-ELL kernel)
};

// Gram-Schmidt / basis kernels over the column-major basis U (ld entries per column).
enum GsOp : int {
    kGsDot = 1,        // h1 = sigma .* (U^T w), ||w||^2          -> finalize pass 1
    kGsUpdDot = 2,     // w -= U coef; h2 = sigma .* (U^T w), ||w||^2 -> finalize pass 2 and the Hessenberg
                       // column (||v_{j+1}||^2 = ||w||^2 - ||h2||^2)
    kGsUpdNorm = 3,    // out = w - U (h2 .* sigma) into column j + 1 (pass 3: update only, no reduction)
    kGsCombine = 4,    // out = -U coef (cycle end: z = V y)
    kGsProj = 6,       // c = sigma .* (U^T w) over the finished cycle's k + 1 columns, then y = the least-
                       // squares solution of H y ~ c with the cycle's rotations and R (restart projection)
};

struct GsArgs {
    const void *U;
    long long ldu;
    void *w;          // input vector (kGsDot, kGsUpdDot: updated in place)
    void *out;        // kGsUpdNorm / kGsCombine output (VecRef-like, column follows j when out_follow)
    int out_follow;   // 1: out = U + k * ldu (k the pass's column count, i.e. column j + 1)
    int op;
    int kcols_from_k; // 1: number of columns is Cycle::k (cycle end), else Cycle::j + 1
    long long ntiles;
    double *partials;
    int nblk;
    int kstage;   // columns one pipeline stage holds (>= the columns used); set by launch_gs
    int nstages;  // pipeline depth; set by launch_gs
    int use_tmap; // 1: a tile's kstage basis columns arrive by one 2-D tensor copy (set by launch_gs)
    int rev;      // 1: the pass visits its row tiles last to first
};

// ---- s-step GMRES with the polynomial (Section VII's combination)
// A block of sb <= kSMax basis vectors is built from the last orthonormal column q_k of the basis U
// (column k): the raw Newton vectors z_1 = (B - theta I) q_k, z_{i+1} = (B - theta I) z_i with B =
// A p(A) go to columns k + 1 .. k + sb; block classical Gram-Schmidt twice against columns 0 .. k
// and Cholesky QR turn them into orthonormal columns, and the block's Hessenberg columns follow
// from the change of basis.
constexpr int kSMax = 8;       // largest block
constexpr int kSColsMax = 64;  // columns 0 .. k a block pass combines (restart <= 64)
enum BgsOp : int {
    kBgsDot = 0,     // P = U^T W and the squared norms of the raw Newton vectors W
    kBgsUpdDot = 1,  // W -= U coef; P = U^T W and G = W^T W, then the block's finalisation
    kBgsUpdTri = 2,  // W -= U coef, then W R^{-1} into the block's columns (no reduction)
};
// Device state of the block being built (one per context).
struct SStep {
    double C[kSMax][kSColsMax];     // C[i][c] = q_c . z_i, summed over both Gram-Schmidt passes
    double coef[kSMax][kSColsMax];  // the next update's coefficients of the stored columns
    double w0[kSMax];               // ||z_i||^2 before the projections
    double red[kSMax * kSColsMax + kSMax * (kSMax + 1) / 2];  // the last pass's reduced sums
    double tinv[kSMax * kSMax];     // R^{-1} (column-major, upper), for the triangular pass
    // flexible float32 form: the preconditioned basis is Z = P M, P the chains' p(A) u_i (stored where
    // the flexible form keeps Z), M upper triangular, column j at M[j][0 .. j]
    double M[kSColsMax][kSColsMax];
    int tri_cols;                   // columns the triangular pass turns into Z R^{-1} (0: none)
    int tri_base;                   // the first of them
    unsigned int ticket[4];
};
struct BgsArgs {
    const void *U;     // the basis (column-major, ld entries per column)
    long long ld;
    int n;
    int k;             // columns 0 .. k are the orthonormal basis; the block is columns k + 1 .. k + sb
    int sb;
    int op;            // BgsOp
    double theta;      // the Newton shift
    double tau;        // Cholesky pivot threshold relative to ||z_i||^2 (the dependence test)
    double *partials;  // per-CTA sums: slot o of CTA b at o * pld + b
    int pld;
    int nblk;
    long long ntiles;
    int flex;          // 1: flexible float32 form (the finalisation extends M)
};
// One pass over the block (nblk CTAs); for kBgsDot and kBgsUpdDot the reduction of its sums follows
// and, after kBgsUpdDot, the block's finalisation: Cholesky, Hessenberg columns, Givens rotations and
// the cycle's tests.  The passes return at once when the cycle has ended before the block (kBgsUpdTri:
// when the finalisation left no columns to form).
cudaError_t launch_bgs(int prec, BgsArgs a, Cycle *st, SStep *ss, int num_sms, cudaStream_t s);
int bgs_max_blocks(int num_sms);
// Flexible s-step form, before x += Z y: y <- M y over the cycle's k columns (Z = P M), so that the
// combination of the stored p(A) u_i with y gives x's correction.  Returns at once when k = 0 or
// (skip_if_stop) the solve has stopped, like the combination.
cudaError_t launch_sstep_flex_y(Cycle *st, SStep *ss, int skip_if_stop, cudaStream_t s);

// ---- ILU(0) on the left (Section VI)
// One level of the row-by-row ILU(0) factorisation (rows: the level's rows): lu holds A's values on
// entry (A's sorted pattern, diag: each row's diagonal position) and L (unit diagonal not stored)
// and U on exit, level by level.
cudaError_t launch_ilu0_level(const int *rows, int count, const int *rp, const int *ci, const int *diag, double *lu,
                              cudaStream_t s);
cudaError_t launch_ilu_cast(const double *in, float *out, long long count, cudaStream_t s);
// A triangular solve with the factors: lower: y = L^{-1} x (unit diagonal); upper: y = U^{-1} x.
// order: the rows sorted by their level for this triangle; y (n entries of the solve's type) is set
// to a pending pattern by the launch and each entry, once written, marks its row final.  The epilogue
// e (its x, x2 unused)
// is applied per row to y: out0 = a0 y + b0 u0 + c0 w0, out1 likewise.  abort: one int, zero; a wait
// that runs out stores there 1 + the row it was computing (the first such row wins) and stops the cycle.
struct IluSolveArgs {
    int n;
    const int *rp, *ci;
    const void *lu;     // factors in the solve's value type
    const int *order;
    int *abort;
    VecRef x;           // input
    void *y;            // the solution (also read by later rows)
    SpmvEpi e;
    Cycle *st;
    int check;          // Check
    const void *rdiag;  // 1 / u_ii in the solve's value type (upper solve)
    int red;            // a power of two <= 32 and >= the longest row: lanes a row's sum is reduced over
    unsigned long long wait_ns;  // limit of one wait on a row the row depends on
    int unreachable;    // tests of the failure path: 1 makes every such wait treat the row as not ready
};
cudaError_t launch_ilu_solve(int prec, bool lower, const IluSolveArgs &a, int num_sms, cudaStream_t s);

// x += U y (float64 x and y = Cycle::y, k = Cycle::k columns of U; flexible cycle end and restart
// projection, U = the preconditioned basis Z); rows n..ld-1 of U are not read.  skip_if_stop: return
// at once when the solve has stopped.
cudaError_t launch_combine_x(int prec, const void *U, long long ld, long long n, double *x, Cycle *st,
                             int skip_if_stop, int num_sms, cudaStream_t s);

cudaError_t launch_validate(int n, long long nnz, const int *rowptr, const int *colidx, int *flag, cudaStream_t s);
cudaError_t launch_cast_f32(const double *in, float *out, long long count, cudaStream_t s);
// check: 0 always run; kSkipIfDone: return when the cycle is done (iteration kernels);
// kSkipIfNoCols: return when the finished cycle has no columns to combine (cycle-end kernels).
enum Check : int { kNoCheck = 0, kSkipIfDone = 1, kSkipIfNoCols = 2, kSkipIfStop = 3 };
cudaError_t launch_spmv(const DevMatrix &A, int prec, const SpmvEpi &e, Cycle *st, int check, cudaStream_t s);
cudaError_t launch_axpy(int n, int prec, const SpmvEpi &e, Cycle *st, int check, cudaStream_t s);
// r = b - A x in float64 written as prec into out (column 0 of the basis); ||r|| finalises the
// start of a restart cycle in st.
// proj = 1: the residual before a restart projection: out = r unscaled; the convergence, iteration-
// limit and finiteness tests as above, but a solve that goes on keeps the finished cycle's state
// (k, the rotations, R) for the projection and the next residual starts the cycle.
cudaError_t launch_residual(const DevMatrix &A, int out_prec, const double *b, const double *x, void *out,
                            Cycle *st, double *partials, cudaStream_t s, int proj = 0);
// ||v||: mode 0 stores ||v|| in st->bnorm; mode 1 starts an Arnoldi run from v (beta, sigma_0, copy into out)
cudaError_t launch_norm_start(int n, int out_prec, const double *v, void *out, int mode, Cycle *st,
                              double *partials, int nblk, cudaStream_t s);
cudaError_t launch_xupdate(int n, int prec, const void *e, double *x, Cycle *st, cudaStream_t s);
cudaError_t launch_copy_in(int n, int prec, const void *src, void *dst, cudaStream_t s);
cudaError_t launch_fill_uniform(double *out, long long n, unsigned long long seed, cudaStream_t s);
cudaError_t launch_csr_outer(const DevMatrix &A, const double *u, const double *v, double alpha, double *out,
                             cudaStream_t s);
cudaError_t launch_transpose(const DevMatrix &A, int *rpT, int *ciT, double *vaT, int *work, cudaStream_t s);

// Gram-Schmidt passes (TMA-staged basis tiles).  kcols: an upper bound on the number of basis
// columns the launch will combine (it selects the tile-shape bucket); ld a multiple of 1024.
cudaError_t launch_gs(int prec, int kcols, long long ld, int num_sms, GsArgs a, Cycle *st, cudaStream_t s);
int gs_max_blocks(int num_sms);

// Power-basis Gram matrix of Eq. 1 with Cholesky and the degree clamp (one kernel).
cudaError_t launch_gram_cholesky(int n, long long ld, const double *B, int deg, double *partials, int nblk,
                                 double *coef_out, int *info_out, Cycle *st, cudaStream_t s);
int gram_grid(int num_sms);
// The same Cholesky and solve on a given (deg + 1)^2 Gram matrix G and right-hand side r (device
// pointers); coef_out deg + 1 values, info_out 3 ints as launch_gram_cholesky's.
cudaError_t launch_gram_solve(const double *G, const double *r, int deg, double *coef_out, int *info_out,
                              cudaStream_t s);

// Roots of 1 - z p(z): harmonic Ritz values of the Arnoldi Hessenberg matrix, Leja ordered.
cudaError_t launch_roots(const Cycle *st, int k, double *roots_out /* 2k */, double *table_out, int *status_out,
                         cudaStream_t s);
cudaError_t launch_root_table(int k, const double *roots, double *table_out, int *status_out, cudaStream_t s);
cudaError_t launch_hess_eigs(int k, const double *H, int ld, double *wr, double *wi, int *status_out,
                             cudaStream_t s);
// ---- batched solver (one thread-block cluster per system)
struct BatchSys {
    int n, nnz;
    const int *rowptr, *colidx;
    const double *vals64;
    const float *vals32;  // library-made float32 copy of vals64
    const double *b;
    double *x;
    float *V;     // (restart + 1) columns of n entries
    float *Z;     // restart columns of n entries: z_j = p(A) v_j of the flexible form
    float *fw;    // 6 vectors of n entries
    double *V64;  // (degree + 2) columns of n entries
    double *dw;   // 1 vector of n entries
    int lanes;    // threads per row of the system's SpMVs (1, 2, 4 or 8; chosen by the autotuner)
};
struct BatchParams {
    int degree, m;
    long long maxit;
    double tol, inner_rtol;
    unsigned long long seed;
    int flexible;  // 1: flexible float32 form with the restart projection (as ppg_solve's default)
};
struct BatchOut {
    long long iters, cycles, spmvs;
    long long t_start, t_end;  // the system's cluster: global timer (ns) at its start and end
    double relres, est;
    int status, degree, converged, breakdowns;
};
constexpr int kBatchMaxRestart = 40;
constexpr int kBatchMaxDegree = 31;
cudaError_t launch_batch_cast(const BatchSys *sys_d, int nsys, cudaStream_t s);
cudaError_t launch_batch(const BatchSys *sys_d, const int *order_d, int nsys, int cluster, const BatchParams &p,
                         BatchOut *out_d, cudaStream_t s, int threads = 256);
int batch_max_clusters(int cluster, int threads = 256);
cudaError_t batch_configure();

// one-time kernel attribute setup (dynamic shared memory limits)
cudaError_t spmv_configure(DevMatrix *A);
// fills the sliced ELL copy (entries and padding; sptr given) from the CSR arrays
cudaError_t launch_sell_fill(int n, int nslices, const int *rowptr, const int *colidx, const double *vals,
                             const int *sptr, short *soff, int *scol, double *svals, cudaStream_t s);
// Two consecutive links of a chain in one launch: e2.x (and e2.x2) are outputs of e1, and e2
// writes none of its own inputs x, x2.  Requires the bandwidth to span at most as many tiles
// as the launch has CTAs (spmv2_tiles_ok); round_done (zero on entry, left zero) holds one int
// per round of the persistent grid, ticket one unsigned int (zero), diag 8 ints (zero) where a
// wait that gives up records itself.
// Limits of the library's software waits: the round-counter waits of the two-step kernel give up
// after ns; extra_need (tests of the failure path only) makes a round need that many CTAs more than
// the launch has, so that those waits run out.
struct WaitCfg {
    unsigned long long ns = kWaitLimitNs;
    int extra_need = 0;
};
cudaError_t launch_spmv2(const DevMatrix &A, int prec, const SpmvEpi &e1, const SpmvEpi &e2, Cycle *st, int check_done,
                         int *round_done, unsigned int *ticket, int *diag, const WaitCfg &wc, cudaStream_t s);
cudaError_t launch_make_coloff(int n, const int *rowptr, const int *colidx, short *out, int *flag, cudaStream_t s);
int spmv_cap_max();
int spmv_rows_per_thread();
cudaError_t gs_configure();
cudaError_t gram_configure();

}  // namespace ppg
