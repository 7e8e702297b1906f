/*
 * ppg.h -- C ABI of the GB300 polynomial-preconditioned GMRES library (libppg.so).
 *
 * The method is the GMRES minimum-residual polynomial preconditioner of Loe,
 * Thornquist and Boman, "Polynomial Preconditioned GMRES to Reduce
 * Communication in Parallel Computing" (arXiv 1907.00072):
 *
 *   - p is the degree-d polynomial minimising ||v0 - A p(A) v0||_2 for a
 *     generating vector v0 (Section II, Eq. 1);
 *   - p(A) = y_{d+1} A^d + ... + y_2 A + y_1 (Eq. 2) is applied as a right
 *     preconditioner: A p(A) u = b, x = p(A) u (Section I);
 *   - the outer solver is restarted GMRES(m) with two passes of classical
 *     Gram-Schmidt (Section III) and a relative residual stopping test
 *     ||b - A x|| / ||b|| <= tol (Section III).
 *
 * Conventions for every entry point:
 *   - Matrix and vector pointers are DEVICE pointers unless a name ends in _h
 *     (host).  The caller owns them; the library never frees them.
 *   - A context owns its own copy of the CSR matrix (made by ppg_create), its
 *     CUDA stream (borrowed, may be NULL for the legacy default stream) and a
 *     workspace (library-allocated unless the caller provides one with
 *     ppg_set_workspace).
 *   - Calls enqueue work on the context's stream.  Calls that return host data
 *     (degree_used, stats, ppg_get_poly, ppg_create's validation) synchronise
 *     that stream before returning.
 *   - No C++ exception crosses this boundary.  Every call returns a
 *     ppg_status; ppg_last_error() gives a one-line explanation of the most
 *     recent failure on the calling thread.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef PPG_H
#define PPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ppg_ctx ppg_ctx;

typedef enum {
    PPG_OK = 0,
    PPG_WARN_DEGREE_CLAMPED = 1, /* power basis: the Gram matrix of Eq. 1 failed Cholesky at the
                                    requested degree; the highest degree that factors is used (Section IV) */
    PPG_ERR_NOT_CONVERGED = 2,   /* maxit reached; x holds the last iterate */
    PPG_ERR_INVALID_ARG = -1,    /* bad sizes, null pointers, CSR with rowptr not monotone or colidx out of range */
    PPG_ERR_CUDA = -2,           /* a CUDA runtime call failed (see ppg_last_error) */
    PPG_ERR_POLY_BREAKDOWN = -3, /* no usable polynomial: degree 0 fails, non-finite coefficients or roots */
    PPG_ERR_NONFINITE = -4,      /* NaN or Inf in a reduction (residual, inner product or norm) */
    PPG_ERR_TIMEOUT = -5,        /* a bounded device wait expired */
    PPG_ERR_OOM = -6,            /* device allocation failed or the caller's workspace is too small */
    PPG_ERR_NO_POLY = -7         /* apply requested before a polynomial was built or set */
} ppg_status;

/* polynomial representations */
enum {
    PPG_BASIS_POWER = 0, /* coefficients y_1..y_{d+1} of Eq. 2, from the normal equations of Eq. 1 */
    PPG_BASIS_ROOTS = 1  /* the d+1 roots theta_i of 1 - z p(z), i.e. p(z) = (1 - prod(1 - z/theta_i)) / z */
};

/* arithmetic of the Krylov basis, p(A) and the SpMVs inside them */
enum {
    PPG_F64 = 0, /* float64 throughout */
    PPG_F32 = 1  /* float32 p(A) and Arnoldi; float64 true residual, Hessenberg least squares and updates of x */
};

/* form of the float32 inner solve (ppg_opts.f32_form) */
enum {
    PPG_F32_FLEXIBLE = 0, /* default: the preconditioned vectors z_j = p(A) v_j are kept (float32) and x += Z y
                             at the end of a cycle (flexible GMRES, the same iterates as right-preconditioned
                             GMRES in exact arithmetic), and before a restart the float64 true residual is
                             projected onto the finished cycle's space (x += Z u, u the least-squares solution
                             of H u ~ V^T r, zero in exact arithmetic) */
    PPG_F32_STANDARD = 1  /* x += p(A) V y with p(A) applied in float32, no projection */
};

typedef struct {
    int precision;     /* PPG_F64 (default) or PPG_F32 */
    double inner_rtol; /* PPG_F32 only: a restart cycle also ends when its residual estimate has dropped by
                          this factor (iterative refinement step); <= 0 selects the default of the form
                          (flexible: 1e-7, about the accuracy one float32 cycle attains; standard: 1e-6) */
    int use_graph;     /* 1: replay each Arnoldi iteration (the p(A) chain and the three Gram-Schmidt
                          passes) from a CUDA graph, captured the second time an iteration index comes
                          round with the same polynomial, workspace, precision and storage format (the
                          first time it launches directly) and kept while those stay the same; kernels of
                          a cycle that has ended still return at once on the device.  0: enqueue the
                          kernels one by one; < 0: library default (graphs) */
    int profile;       /* 1: time every SpMV and Gram-Schmidt launch with CUDA events and report their
                          device time and algorithmic bytes in ppg_stats (adds a sync per cycle) */
    int f32_form;      /* PPG_F32 only: PPG_F32_FLEXIBLE (0, default) or PPG_F32_STANDARD */
    int wait_limit_us; /* limit of the library's software waits, in microseconds: the two-step kernel's waits on
                          its round counters (ppg_chain_fusion), the ILU(0) triangular solves' waits on the rows
                          a row depends on, and the host's wait for the device's progress between enqueued
                          iterations.  <= 0 or >= 10^6: 1 s.  A wait that runs out ends the solve
                          with PPG_ERR_TIMEOUT once the work already queued has finished (every device wait is
                          bounded; waits on TMA copies keep their 1 s limit), and ppg_last_error() says where */
    int test_unreachable_wait; /* tests of the failure path only (0 otherwise): 1 makes every round of the
                          two-step kernel need one CTA more than its launch has, and every ILU(0) triangular
                          solve treat the rows it waits on as never ready, so that those waits run out after
                          wait_limit_us */
    int sstep;         /* 0 (default): one basis vector per orthogonalisation.  1..8: s-step blocks (Section VII's
                          combination of the polynomial with an s-step method): sstep vectors of the Newton basis
                          (A p(A) - sstep_shift I)^i q_k are built by SpMV chains alone, then orthogonalised
                          together by block classical Gram-Schmidt twice and Cholesky QR, three global
                          reductions per block; the block's Hessenberg columns follow from the change of
                          basis, so the iterates are GMRES's in exact arithmetic.  Requires restart <= 64 and no
                          ILU(0).  float32 solves take f32_form: the flexible form keeps each chain's p(A) u_i and
                          the block's preconditioned columns as their combination Z = P M (M from the same change
                          of basis), so x += Z y as without blocks.  A block whose Newton vector
                          is numerically dependent (Cholesky pivot below 1e-14 (float64) or 1e-6 (float32)
                          of its squared norm) ends the cycle with a lucky breakdown.  The first s-step solve of a
                          context allocates the blocks' device state and per-CTA sums (about 45 KB + 13 KB per SM
                          of the GPU), outside the workspace */
    double sstep_shift; /* the Newton shift theta (sstep > 0): a point inside the spectrum of A p(A); a
                          minimum-residual polynomial clusters that spectrum around 1 */
} ppg_opts;

typedef struct {
    int64_t iterations;  /* GMRES iterations (basis vectors built) */
    int64_t restarts;    /* restart cycles started */
    int64_t spmvs;       /* sparse matrix-vector products, counted as in Section III */
    int64_t dots;        /* 2 block inner products + 1 norm per iteration (Section III) and 1 norm per cycle; s-step
                            solves: 3 global reductions per block and 1 per cycle */
    int64_t kernel_launches;
    double relres_true;  /* ||b - A x|| / ||b|| of the returned x, computed in float64 */
    double relres_est;   /* last in-cycle Givens estimate |g_{j+1}| / ||b|| */
    int degree_used;     /* degree of the polynomial applied */
    int converged;       /* 1 if relres_true <= tol */
    int breakdowns;      /* cycles ended by a (lucky) Arnoldi breakdown */
    int ctas_per_system; /* ppg_solve_batched: CTAs (cluster size) per system; 0 otherwise */
    int spmv_lanes;      /* ppg_solve_batched: threads per row of the system's SpMV (tuned); 0 otherwise */
    double time_ms;      /* wall time of the call on the device stream (CUDA events) */
    /* filled when ppg_opts.profile = 1, for launches that did work: device time and algorithmic
       bytes of the SpMV chain (p(A) steps and the SpMV that applies A) and of the Gram-Schmidt
       passes (block inner products, updates, norms, cycle-end combination).  Each run of
       consecutive launches of one kind (one iteration's SpMV chain, its three passes, ...) is
       timed by one pair of CUDA events; *_segments counts those runs.  Bytes are algorithmic:
       matrix values and indices once, every vector read or written once per launch. */
    double spmv_ms, spmv_bytes;
    int64_t spmv_segments;
    double gs_ms, gs_bytes;
    int64_t gs_segments;
} ppg_stats;

/* ------------------------------------------------------------------ context */

/* Creates a context for the n x n CSR matrix (int32 rowptr[n+1] and colidx[nnz], float64 vals[nnz],
 * device pointers, zero-based).  The matrix is copied into library-owned device memory and validated
 * on the device (rowptr[0] = 0, rowptr non-decreasing, rowptr[n] = nnz, 0 <= colidx < n); columns within
 * a row need not be sorted.  stream is a cudaStream_t (NULL: legacy default stream).  Synchronises.
 * Errors: PPG_ERR_INVALID_ARG (n <= 0, nnz < 0, null pointer, invalid CSR), PPG_ERR_OOM, PPG_ERR_CUDA. */
ppg_status ppg_create(ppg_ctx **ctx, int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                      const double *vals, void *stream);

/* Frees everything the context allocated (not a caller-provided workspace).  NULL is a no-op. */
void ppg_destroy(ppg_ctx *ctx);

/* Changes the stream later calls enqueue on. */
ppg_status ppg_set_stream(ppg_ctx *ctx, void *stream);

/* Bytes of device workspace needed by solves with this restart length, polynomial degree and
 * precision (also enough for ppg_build_poly at that degree and ppg_apply_poly). */
ppg_status ppg_workspace_bytes(const ppg_ctx *ctx, int restart, int degree, int precision, size_t *bytes);

/* Hands the context a caller-owned device workspace (at least 256-byte aligned).  The library then
 * allocates no workspace of its own while this one is large enough; a call that needs more returns
 * PPG_ERR_OOM.  Passing NULL returns to library-managed allocation.  The buffer must outlive its use. */
ppg_status ppg_set_workspace(ppg_ctx *ctx, void *ws, size_t bytes);

/* ------------------------------------------------------------------ kernels */

/* y = A x (Section II's SpMV).  precision PPG_F64: x, y are float64[n]; PPG_F32: float32[n] with the
 * float32 copy of the values.  x and y must not overlap. */
ppg_status ppg_spmv(ppg_ctx *ctx, const void *x, void *y, int precision);

/* Sparse storage the SpMV kernels read.  The paper stores A in CSR (Epetra, Section II); this library
 * keeps the CSR arrays and, at ppg_create, also
 *   - a sliced ELL copy: slices of 32 consecutive rows, each padded to its longest row and stored entry
 *     index by entry index, so one warp reads a slice with coalesced loads (PPG_SPMV_SELL);
 *   - for each tile of rows, up to four contiguous ranges of x covering every column the tile's rows
 *     reference (banded matrices), and per entry its index into those ranges: with PPG_SPMV_STAGED the
 *     float32 kernel copies the ranges into shared memory along with the matrix tile, so that each x
 *     gather is one shared-memory load (available when 90 % of the tiles are covered).  When every
 *     256-row tile's columns fit eight such ranges and rows have at most 32 entries (mean row length
 *     <= 40), the matrix is also stored tile by tile as dense 256 x w blocks of float32 values and
 *     window indices (w = the tile's longest row, padding pointing at a zero), and a float64 copy of
 *     them, which STAGED then reads instead in float32 and float64: one thread per row, no row
 *     pointers, w shared-memory multiply-adds per row.
 * The windows end on 16-byte boundaries inside x, so when n is not a multiple of 4 the last tile has
 * none and no dense blocks are built.  STAGED is available when either copy exists; PPG_SPMV_AUTO then
 * selects it, and the row-block CSR kernel otherwise (measured per SpMV: 7-point 128^3 25.2 us with CSR,
 * 16.6 us STAGED; 27-point 100^3 44.4 and 28.5 us; SELL slower than both).  PPG_SPMV_CSR, PPG_SPMV_SELL
 * and PPG_SPMV_STAGED force one (STAGED applies to float32 links, and to float64 and two-input links
 * w = A (x + s x2) where the dense blocks exist; others run as CSR).
 * Every result is the same sum; CSR and STAGED give identical bits.  request = PPG_SPMV_QUERY changes
 * nothing; *in_effect (host, may be NULL) receives the format now used.
 * Errors: PPG_ERR_INVALID_ARG (unknown request, or a format whose copy was not built). */
enum {
    PPG_SPMV_QUERY = -1,
    PPG_SPMV_AUTO = 0,
    PPG_SPMV_CSR = 1,
    PPG_SPMV_SELL = 2,
    PPG_SPMV_STAGED = 3
};
ppg_status ppg_spmv_format(ppg_ctx *ctx, int request, int *in_effect);

/* Pairing of the p(A) chain's links (Eq. 2 applied link by link: each link is one SpMV with a fused
 * vector update), in the spirit of the matrix powers kernel Section VII points to.  When on, two
 * consecutive links share one cooperative launch: every tile of rows staged in shared memory serves
 * the first link and, two rounds of the persistent grid later (once all rows within the matrix
 * bandwidth have their first-link result, counted per round), the second, so the matrix crosses HBM
 * once per two links.  Applies to the row-block CSR kernel when the bandwidth max |col - row| spans
 * no more tiles than the launch has CTAs; otherwise links run one per launch.  Results are
 * bit-identical either way (same tiles, same per-row arithmetic).  Off by default: on the 128^3
 * stencil a paired launch took 124 us against 2 x 28.8 us for two single ones (the per-round waits
 * cost more than the saved matrix traffic).  request: 1 on, 0 off, -1 query; *in_effect (host, may
 * be NULL) receives 1 when float32 chains of this matrix are paired.  Errors: PPG_ERR_INVALID_ARG. */
ppg_status ppg_chain_fusion(ppg_ctx *ctx, int request, int *in_effect);

/* ------------------------------------------------------------------ polynomial */

/* Builds the minimum-residual polynomial of the given degree from the generating vector v0
 * (float64[n] device pointer, or NULL for v0 uniform in [-1, 1] from the counter-based SplitMix64
 * stream `seed`, as Section V recommends a random vector).
 *   PPG_BASIS_POWER: the paper's construction (Eq. 1): d+1 SpMVs give AV = [A v0, ..., A^{d+1} v0],
 *     G = (AV)^T AV and r = (AV)^T v0 are formed in one pass, G y = r is solved by Cholesky.  If the
 *     Cholesky pivot of order j is not positive, the degree is clamped to j-2 (Section IV) and
 *     PPG_WARN_DEGREE_CLAMPED is returned.
 *   PPG_BASIS_ROOTS: the same polynomial represented by the roots of 1 - z p(z) (the harmonic Ritz
 *     values of a (d+1)-step Arnoldi run from v0), applied as a product in Leja order; stable at the
 *     high degrees where the power basis fails (Sections II and VIII point to such constructions).
 * degree = -1 selects the degree automatically by Section IV's rule: the highest degree whose power-
 * basis Gram matrix still factors (searched up to 30).  degree_used (host, may be NULL) receives the
 * degree built.  Synchronises.  0 <= degree <= 62.
 * Errors: PPG_ERR_INVALID_ARG, PPG_ERR_POLY_BREAKDOWN, PPG_ERR_NONFINITE, PPG_ERR_OOM, PPG_ERR_CUDA. */
ppg_status ppg_build_poly(ppg_ctx *ctx, int degree, int basis, const double *v0, uint64_t seed, int *degree_used);

/* Sets the polynomial from host data instead of building it.
 *   PPG_BASIS_POWER: coef_h[0..degree] with coef_h[i] multiplying A^i (y_{i+1} of Eq. 2).
 *   PPG_BASIS_ROOTS: coef_h holds degree+1 roots as (re, im) pairs, applied in the given order;
 *     a complex root must be followed by its conjugate. */
ppg_status ppg_set_poly(ppg_ctx *ctx, int basis, int degree, const double *coef_h);

/* Copies the current polynomial to host: *basis, *degree, and coef_h (capacity cap doubles):
 * degree+1 coefficients (power) or degree+1 (re, im) root pairs in application order (roots).
 * Also returns (resid_h, may be NULL) ||v0 - A p(A) v0|| / ||v0|| as measured during construction
 * (NaN if the polynomial was set). */
ppg_status ppg_get_poly(ppg_ctx *ctx, int *basis, int *degree, double *coef_h, int cap, double *resid_h);

/* out = p(A) v (Eq. 2) with the current polynomial; precision as in ppg_spmv.  v and out are
 * device vectors of length n of the matching type and must not overlap. */
ppg_status ppg_apply_poly(ppg_ctx *ctx, const void *v, void *out, int precision);

/* ILU(0) on the left of the polynomial (Section VI): with enable = 1 the context factors its matrix
 * as M = L U, the incomplete LU with no fill (L U agrees with A on A's sparsity pattern; computed on
 * the device, once), and from then on the operator of ppg_build_poly, ppg_apply_poly and ppg_solve
 * is B = M^{-1} A: the polynomial is the minimum-residual polynomial of B and ppg_solve solves
 * M^{-1} A p(M^{-1} A) u = M^{-1} b with x = p(M^{-1} A) u, each restart cycle starting from the
 * preconditioned residual M^{-1} (b - A x), its estimate relative to ||M^{-1} b||, the stopping test
 * the true ||b - A x|| <= tol ||b||.  The float32 solve runs the standard form (PPG_F32_STANDARD)
 * and no CUDA graphs.  enable = 0 returns to A (the factors are kept).  Changing the setting drops the
 * current polynomial (build it again).  ppg_spmv still computes A x; ppg_solve_transpose and
 * ppg_apply_poly_noalloc refuse to run while ILU(0) is on.  lu_out (device, nnz doubles, may be
 * NULL) receives the factors on A's pattern: L below the diagonal (unit diagonal not stored), U on and
 * above it.  The triangular solves are one cooperative launch each, whose warps wait (bounded: 1 s, or a
 * solve's ppg_opts.wait_limit_us) for the rows they depend on.  Synchronises.
 * Errors: PPG_ERR_INVALID_ARG (a row's columns not sorted, a diagonal entry missing),
 * PPG_ERR_POLY_BREAKDOWN (a zero or non-finite pivot), PPG_ERR_OOM, PPG_ERR_CUDA. */
ppg_status ppg_set_left_ilu0(ppg_ctx *ctx, int enable, double *lu_out);

/* Allocation-free variant of ppg_apply_poly (the paper has no counterpart; this is a service of the
 * library).  For callers that may not allocate device memory at the point of the call -- for example
 * a service that reserves its whole device-memory budget at start-up, or code running where a
 * cudaMalloc could fail or must not happen -- it computes out = p(A) v exactly like ppg_apply_poly
 * but takes its working vectors from a fixed array compiled into the library (one array per GPU that
 * loads the library, kept until the process exits) instead of the context's workspace, and it calls
 * no allocating routine.
 *   - Limit: n <= 65536 rows (5 working vectors of 65536 float64 entries, 2.5 MiB).  Larger
 *     matrices return PPG_ERR_INVALID_ARG; use ppg_apply_poly.
 *   - precision PPG_F32 needs the context's float32 copy of the matrix, which this call does not
 *     create: make one float32 ppg_spmv / ppg_apply_poly / ppg_solve call first (else
 *     PPG_ERR_INVALID_ARG).
 *   - ppg_create, which allocates anyway, looks up the array's device address (once per device) for
 *     every matrix within the limit, so this call maps no memory and allocates nothing.
 *   - Every call uses the same array, which keeps the previous call's contents; calls whose work
 *     overlaps on the GPU (different streams, or concurrent host threads) race with each other.
 *     Calls enqueued on one stream run one after another and are safe.
 * Asynchronous on the context's stream, like ppg_apply_poly. */
ppg_status ppg_apply_poly_noalloc(ppg_ctx *ctx, const void *v, void *out, int precision);

/* ------------------------------------------------------------------ solvers */

/* Solves A x = b by right-preconditioned GMRES(restart) with the current polynomial (the identity if
 * none was built): the Krylov basis is built for A p(A) with two classical Gram-Schmidt passes per
 * iteration, the Hessenberg least-squares problem is solved with Givens rotations on the device, and
 * at each restart x += p(A) V y (the float32 flexible form: x += Z y with the kept Z = p(A) V) followed
 * by a float64 true residual b - A x.  b and x are float64[n]
 * (x: initial guess in, solution out).  Stops when ||b - A x|| / ||b|| <= tol or after maxit
 * iterations.  1 <= restart <= 127.  opts and stats may be NULL.  Synchronises.
 * Returns PPG_OK, PPG_ERR_NOT_CONVERGED, or an error. */
ppg_status ppg_solve(ppg_ctx *ctx, const double *b, double *x, double tol, int restart, int maxit,
                     const ppg_opts *opts, ppg_stats *stats);

/* Solves A^T lambda = g with the same method and the preconditioner p(A^T) = p(A)^T (same
 * polynomial), using a transposed copy of the matrix built on the device at the first call.  Used by
 * the adjoint of x = A^{-1} b: dL/db = lambda and dL/dvals_k = -lambda_{row(k)} x_{col(k)}. */
ppg_status ppg_solve_transpose(ppg_ctx *ctx, const double *g, double *lambda, double tol, int restart, int maxit,
                               const ppg_opts *opts, ppg_stats *stats);

/* out_k = alpha * u_{row(k)} * v_{col(k)} for every stored entry k of the matrix (CSR order of the
 * matrix passed to ppg_create).  u, v float64[n]; out float64[nnz]. */
ppg_status ppg_csr_outer(ppg_ctx *ctx, const double *u, const double *v, double alpha, double *out);

/* k steps of Arnoldi for the operator A p(A) (current polynomial, or A alone if none) from v (float64[n]),
 * with the solver's two-pass classical Gram-Schmidt kernels, in float64.  V (device, may be NULL):
 * n x (k+1) column-major orthonormal basis; H_h (host): (k+1) x k column-major Hessenberg matrix.
 * Returns the number of steps completed (< k on breakdown) in *steps.  1 <= k <= 127. */
ppg_status ppg_arnoldi(ppg_ctx *ctx, const double *v, int k, double *V, double *H_h, int *steps);

/* Eigenvalues of a k x k upper Hessenberg matrix (float64, column-major with leading dimension ld,
 * device pointer) by the device's Francis double-shift QR kernel, the one used for the roots of the
 * polynomial.  wr, wi: device float64[k].  Exposed for testing.  1 <= k <= 64. */
ppg_status ppg_hessenberg_eigs(ppg_ctx *ctx, int k, const double *H, int ld, double *wr, double *wi);

/* Solves the normal equations G y = r of Eq. 1 for a caller-given Gram matrix with the device's Cholesky, the
 * one ppg_build_poly(PPG_BASIS_POWER) runs: column by column with LAPACK POTRF's test (a pivot that is not
 * positive, NaN included, stops the factorisation; *info = its 1-based order, 0 if none), then the solve with
 * the leading block that factored, so that the degree used is degree (info = 0) or info - 2 (Section IV).
 * G_h: (degree+1) x (degree+1) column-major, r_h: degree+1 values, coef_h: degree+1 values out (zero beyond
 * the degree used); all host memory.  info, degree_used (host) may be NULL.  0 <= degree <= 62.  Exposed to
 * test the factorisation and the degree rule on a given G.  Allocates a small device buffer; synchronises.
 * Returns PPG_OK, PPG_WARN_DEGREE_CLAMPED, or an error (PPG_ERR_POLY_BREAKDOWN when degree 0 fails). */
ppg_status ppg_gram_solve(ppg_ctx *ctx, int degree, const double *G_h, const double *r_h, double *coef_h, int *info,
                          int *degree_used);

/* Fills out[i] = uniform in [-1, 1) from the counter-based SplitMix64 stream `seed` (element i is the
 * stream's position i: z = mix(mix(seed) + (i+1) * 0x9E3779B97F4A7C15), u = (z >> 11) * 2^-53).
 * This is the generator ppg_build_poly uses when v0 is NULL. */
ppg_status ppg_fill_uniform(ppg_ctx *ctx, double *out, int64_t n, uint64_t seed);

/* ------------------------------------------------------------------ batched */

/* One system of a batch: a CSR matrix (int32 rowptr[n+1], colidx[nnz], float64 vals[nnz]) and its
 * vectors, all device pointers owned by the caller. */
typedef struct {
    int64_t n, nnz;
    const int32_t *rowptr, *colidx;
    const double *vals;
    const double *b;
    double *x; /* initial guess in, solution out */
} ppg_batch_system;

/* Solves nsys independent systems in one persistent launch (replayed from a CUDA graph).  Each
 * system is owned by one thread-block cluster, which builds the system's minimum-residual polynomial
 * (roots form, the given degree, v0 uniform in [-1, 1] from the SplitMix64 stream seed + i, float64
 * construction) and runs float32 PP-GMRES(restart) cycles in the flexible form of ppg_solve's
 * default (z_j = p(A) v_j kept, x += Z y in float64, the float64 true residual projected onto the
 * finished cycle's space before a restart; a cycle also stops once its residual estimate drops by
 * 1e-7), until ||b - A x|| <= tol ||b|| or maxit iterations.  Systems start largest first.  The first
 * call with a new batch shape (the sorted list of (n, nnz), degree and restart) tunes the launch by
 * timing solves of the batch itself (x in scratch memory, so the caller's x is untouched): the CTAs
 * per system (the rows each CTA owns) -- 4, 8 or 16 for every system, or 16 (CTAs of 256 or 512
 * threads) for the systems of at least 4096, 16384 or 65536 rows and 1, 2, 4 or 8 for the others, the
 * two groups then running as two concurrent launches -- then, per class of rows per CTA (< 256,
 * < 2048, more), the SpMV's threads per row (1, 2, 4 or 8); the choice is cached for the shape.
 * per_sys (host, nsys entries, may be NULL) receives each system's statistics (time_ms: the whole
 * batch; spmv_ms: the system's own time on the device, from its cluster's start to its end; gs_ms:
 * when that cluster started, after the first cluster's start; ctas_per_system: the system's tuned
 * cluster size; spmv_lanes: its SpMV's threads per row).
 * restart <= 40,
 * degree <= 31.  stream as in ppg_create.  Synchronises.  The library keeps one workspace per device
 * for batched calls (not thread-safe across host threads on one device).
 * Returns PPG_OK, PPG_ERR_NOT_CONVERGED if any system missed the tolerance, or an error. */
ppg_status ppg_solve_batched(int nsys, const ppg_batch_system *sys_h, int degree, double tol, int restart, int maxit,
                             uint64_t seed, void *stream, ppg_stats *per_sys);

/* ------------------------------------------------------------------ diagnostics */

const char *ppg_status_string(ppg_status status);

/* One-line description of the last failure on the calling thread ("" if none). */
const char *ppg_last_error(void);

/* Library version string. */
const char *ppg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PPG_H */
