// ppg_ortho.cu -- Gram-Schmidt and Gram-matrix kernels of the GB300 PP-GMRES library.
//
// Arnoldi orthogonalisation is classical Gram-Schmidt applied twice (Loe,
// Thornquist, Boman, Section III: "two steps of Classical Gram Schmidt", two block
// inner products and one norm per iteration).  With w = A p(A) v_j the three
// passes over the basis are
//   pass 1:  h1 = V^T w                         (block inner product, and ||w||^2)
//   pass 2:  w <- w - V h1,  h2 = V^T w         (update fused with the second inner product
//                                                and the norm ||w||^2 of the updated w)
//   pass 3:  v_{j+1} <- w - V h2                (update only)
// Each pass streams the basis once.  The norm of v_{j+1} follows from pass 2 by Pythagoras,
// ||w - V h2||^2 = ||w||^2 - ||h2||^2 for orthonormal V (after one orthogonalisation h2 is tiny
// against w, so the difference is exact to working precision), so an iteration has two global
// reductions, not three.  Tiles of the column-major basis (TR rows x k columns) are staged in
// shared memory with TMA bulk copies, double-buffered across a persistent grid, so the update and
// the inner product of pass 2 read each tile from HBM once.  Per-CTA partial sums go to a
// [column x CTA] buffer and the last CTA to finish reduces them in a fixed order (deterministic
// results) and finalises the Hessenberg column on the device: Givens rotations and the
// convergence test of GMRES never leave the GPU.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include "ppg_cycle.cuh"
#include "ppg_internal.h"

namespace ppg {

// Tile height by basis-width bucket KM (k <= KM columns): a tile of all KM columns would be
// 32 KB.  At run time a stage holds exactly the launch's column bound kst (<= KM) plus w, and
// as many stages as fit the shared-memory budget are used, so that small k still keeps many
// bytes in flight.
#ifndef PPG_GS_SMEM_KB
#define PPG_GS_SMEM_KB 72
#endif
#ifndef PPG_GS_TILE_BYTES
#define PPG_GS_TILE_BYTES 32768  // a full-width stage (KM columns) of one tile
#endif
#ifndef PPG_GS_TILE_BYTES_WIDE
#define PPG_GS_TILE_BYTES_WIDE 65536  // the same for the buckets KM >= 64 (tiles of 256 float32 rows)
#endif
#ifndef PPG_GS_SMEM_KB_WIDE
#define PPG_GS_SMEM_KB_WIDE 132
#endif
#ifndef PPG_GS_STAGES
#define PPG_GS_STAGES 2  // cap on the pipeline depth: more CTAs per SM beat deeper pipelines (measured)
#endif
constexpr int kGsMaxStages = 8;

constexpr int pow2_floor(int v) { return v < 2 ? 1 : 2 * pow2_floor(v / 2); }

template <typename T, int KM>
struct GsCfg {
    static constexpr int kTileBytes = KM >= 64 ? PPG_GS_TILE_BYTES_WIDE : PPG_GS_TILE_BYTES;
    static constexpr int TR = pow2_floor(kTileBytes / (KM * (int)sizeof(T))) > 32
                                  ? pow2_floor(kTileBytes / (KM * (int)sizeof(T)))
                                  : 32;  // rows per tile (divides 1024)
    static constexpr int kSmemBudget = (KM >= 64 ? PPG_GS_SMEM_KB_WIDE : PPG_GS_SMEM_KB) * 1024;  // per CTA
    static_assert(2 * (KM + 1) * TR * (int)sizeof(T) <= kSmemBudget, "two full-width stages must fit");
    static constexpr int RPT = TR >= kThreads ? TR / kThreads : 1;       // rows per thread (update phase)
    static constexpr int TPR = TR >= kThreads ? 1 : kThreads / TR;       // threads per row (update phase)
    static constexpr int RPL = TR / 32;                                  // rows per lane (dot phase, stride 32)
    static constexpr int CPW = (KM + 7) / 8;                             // columns per warp (dot phase)
};

// Accumulator of a warp's column sums: float64 directly, or float32 with Kahan
// compensation (float64 arithmetic is scarce on this GPU; the float32 basis is
// reduced in float32 per lane and in float64 across lanes and CTAs).
template <typename T>
struct Acc {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    // every lane calls these; lane 0 (thread 0) stores the slot
    __device__ __forceinline__ void store_warp_total(double *slot) const
    {
        const double v = warp_sum(s);
        if ((threadIdx.x & 31) == 0) *slot = v;
    }
    __device__ __forceinline__ void store_block_total(double *slot, double *scratch) const
    {
        const double v = block_sum(s, scratch);
        if (threadIdx.x == 0) *slot = v;
    }
    static __device__ __forceinline__ double reduce(const double *slots, int ld, int nblk, int c)
    {
        return reduce_slots_f64(slots, ld, nblk, c);
    }
};
template <>
struct Acc<float> {
    float s = 0.f, c = 0.f;  // the running sum is s - c
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    // across lanes, warps and CTAs with compensated float32 sums (see F2), kept as pairs until
    // the final column sum
    __device__ __forceinline__ void store_warp_total(double *slot) const
    {
        const F2 v = warp_tree_f2(F2{s, -c});
        if ((threadIdx.x & 31) == 0) *reinterpret_cast<float2 *>(slot) = make_float2(v.hi, v.lo);
    }
    __device__ __forceinline__ void store_block_total(double *slot, double *scratch) const
    {
        const F2 v = block_sum_f2_pair(F2{s, -c}, reinterpret_cast<F2 *>(scratch));
        if (threadIdx.x == 0) *reinterpret_cast<float2 *>(slot) = make_float2(v.hi, v.lo);
    }
    static __device__ __forceinline__ double reduce(const double *slots, int ld, int nblk, int c)
    {
        return reduce_slots_f2(slots, ld, nblk, c);
    }
};

// Accumulator of a row of x += U y (kGsCombineX).  Float64 basis: float64 products and sums.
// Float32 basis (float64 y split as yh + yl in float32): each product yh z is kept exactly as
// p + (fma(yh, z, -p)), yl z is added to that error term, and the running sum is a two-sum pair,
// so the row's correction reaches x with float64-level accuracy from float32 arithmetic only.
template <typename T>
struct XAcc {
    double s = 0.0;
    __device__ __forceinline__ void add(T z, T yh, T) { s = fma((double)z, (double)yh, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct XAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float z, float yh, float yl)
    {
        const float p = yh * z;
        const float pe = fmaf(yl, z, fmaf(yh, z, -p));
        const float t = s + p;
        const float bp = t - s;
        c += ((s - (t - bp)) + (p - bp)) + pe;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// ---------------------------------------------------------------- finalisation (last CTA)
//
// The device state lives in global memory, where every dependent access of a serial loop costs
// an L2 round trip; the last CTA therefore does the per-column work with all its threads and
// runs the serial recurrences (Givens rotations, back substitution) on shared-memory copies.

// Pass 3: completes Hessenberg column j, H[0..j, j] = h1 + h2, H[j+1, j] = ||v_{j+1}||.  In GMRES
// mode the previous Givens rotations are applied to the column, a new rotation zeroes H[j+1, j]
// and updates g; the cycle ends on a small estimate |g_{j+1}|, a breakdown, the restart length or
// the iteration limit, and then y = R^{-1} g is formed and the coefficients of the correction
// z = V y are left in coef.  ||v_{j+1}||^2 is the sum of the CTAs' norm slots.  sh: shared
// scratch of sh_bytes (at least 5 (kKmax + 2) doubles).
//
// Float64 instructions are scarce on this GPU, so the serial part is kept short: warp 0 sums the
// norm slots while the other warps stage the column, the rotations and the state's scalars; the
// rotations form the recurrence a_{i+1} = -s_i a_i + c_i b_{i+1} (a_0 = b_0, b = the column as
// built), whose products c_i b_{i+1} and rotated entries c_i a_i + s_i b_{i+1} are formed by all
// threads, leaving one multiply-add per step to thread 0, while warp 1 forms the norm and its
// reciprocal.
template <typename T>
__device__ void cta_finish_pass3(Cycle *st, int j, double wsq, double *sh, size_t sh_bytes, int *s_int)
{
    const int tid = threadIdx.x, nt = blockDim.x, wid = tid >> 5, lane = tid & 31;
    double *col = sh;                // column j as built (j + 1 values)
    double *cs = sh + (kKmax + 2);   // rotations 0 .. j-1
    double *sn = cs + (kKmax + 2);
    double *cb = sn + (kKmax + 2);   // cs[i] col[i+1]
    double *ar = cb + (kKmax + 2);   // a_i, then the rotated column (j + 2 values)
    // [0] ||v||^2  [1] ||v||  [2] sigma_{j+1}  [3] g_j  [4] tol ||b||  [5] inner_rtol beta (or -1)
    // [6] 1 / ||b||  [7] breakdown threshold on ||v||^2  [8] ||w'||^2
    __shared__ double sc[9];
    __shared__ long long s_it[2];  // iters, maxit
    __shared__ int s_m[2];         // restart length, mode
    if (tid == 0) s_int[0] = 0;
    __syncthreads();
    if (wid == 0) {
        // ||v_{j+1}||^2 = ||w'||^2 - ||h2||^2 (h2 = V^T w', written by this CTA before the call)
        double s2 = 0.0;
        for (int i = lane; i <= j; i += 32) {
            const double h = st->h2[i];
            s2 = fma(h, h, s2);
        }
        s2 = warp_sum(s2);
        if (lane == 0) {
            sc[0] = wsq - s2;
            sc[8] = wsq;
        }
    } else {
        if (tid == nt - 1) {
            s_it[0] = st->iters;
            s_it[1] = st->maxit;
            s_m[0] = st->m;
            s_m[1] = st->mode;
            const double bn = st->enorm, irt = st->inner_rtol;
            sc[3] = st->g[j];
            sc[4] = st->tol * bn;
            sc[5] = irt > 0.0 ? irt * st->beta : -1.0;
            sc[6] = 1.0 / bn;
            sc[7] = 1e-28 * st->w0sq;
        }
        for (int i = tid - 32; i <= j; i += nt - 32) {
            const double h = st->h1[i] + st->h2[i];
            col[i] = h;
            st->H[(long long)j * kLdH + i] = h;
            if (!isfinite(h)) s_int[0] = 1;
            if (i < j) {  // used in GMRES mode only
                const double c = st->cs[i], sv = st->sn[i];
                cs[i] = c;
                sn[i] = sv;
                cb[i] = c * (st->h1[i + 1] + st->h2[i + 1]);
            }
        }
    }
    __syncthreads();
    const bool gm = s_m[1] == 0;
    if (tid == 0 && gm) {
        double a = col[0];
        for (int i = 0; i < j; ++i) {
            ar[i] = a;
            a = fma(-sn[i], a, cb[i]);
        }
        ar[j] = a;
    } else if (tid == 32) {
        const double nsq = sc[0];
        // breakdown: v_{j+1} negligible against ||w||, or the second pass removed more than 99 % of w'
        // (then the difference of squares is no longer accurate): either way the cycle ends there
        const bool brk = !(nsq > sc[7]) || !(nsq > 1e-2 * sc[8]);
        const double nrm = !isfinite(nsq) ? nsq : (brk ? 0.0 : sqrt(nsq));  // NaN / Inf stay visible
        sc[1] = nrm;
        sc[2] = brk ? 0.0 : 1.0 / nrm;
        s_int[2] = brk;
    }
    __syncthreads();
    if (gm)
        for (int i = tid; i < j; i += nt) ar[i] = fma(cs[i], ar[i], sn[i] * col[i + 1]);
    if (tid == 0) {
        int kdone = 0;
        const double nrm = sc[1];
        st->H[(long long)j * kLdH + j + 1] = nrm;
        if (s_int[0] || !isfinite(nrm)) {
            st->error |= kErrNonfinite;
            st->stop = 1;
            st->cycle_done = 1;
            st->k = 0;
            st->j = j + 1;
            kdone = -1;
            publish_progress(st, 1, j + 1);
        } else {
            const bool brk = s_int[2] != 0;
            const long long it = s_it[0] + 1;
            st->sigma[j + 1] = sc[2];
            st->iters = it;
            bool done = brk || (j + 1 >= s_m[0]) || (it >= s_it[1]);
            if (gm) {
                const double a = ar[j];
                const double r = sqrt(fma(a, a, nrm * nrm));
                double c = 1.0, s = 0.0;
                if (r != 0.0) {
                    const double ri = 1.0 / r;
                    c = a * ri;
                    s = nrm * ri;
                }
                st->cs[j] = c;
                st->sn[j] = s;
                ar[j] = r;
                ar[j + 1] = 0.0;
                const double gj = sc[3];
                st->g[j] = c * gj;
                st->g[j + 1] = -s * gj;
                const double res = fabs(s * gj);
                st->est = res * sc[6];
                done = done || (res <= sc[4]) || (res <= sc[5]);
            }
            if (brk) {
                st->breakdown = 1;
                st->n_breakdowns += 1;
            }
            st->j = j + 1;
            if (done) {
                st->k = j + 1;
                st->cycle_done = 1;
                kdone = j + 1;
            } else {
                publish_progress(st, 0, j + 1);
            }
        }
        s_int[1] = kdone;
    }
    __syncthreads();
    const int kdone = s_int[1];
    if (kdone >= 0 && gm)
        for (int i = tid; i <= j + 1; i += nt) st->R[(long long)j * kLdH + i] = ar[i];
    if (kdone > 0 && gm) {
        __syncthreads();  // col, cs, sn, ar no longer needed
        cta_solve_r(st, kdone, sh, sh_bytes);
        if (tid == 0) publish_progress(st, 1, j + 1);
    }
}

// Restart projection (flexible float32 solves), by the last CTA of the kGsProj pass: the finished
// cycle left V_{k+1}, its rotations Q and triangle R with H = Q R; the pass summed U^T r for the
// true residual r.  c = V^T r (c_q = sigma_q (U^T r)_q), the least-squares solution of H u ~ c is
// u = R^{-1} (Q^T c)_{0..k-1}, written to y for the following x += Z u.  In exact arithmetic r is
// orthogonal to range(H) and u = 0; in float32 it removes the part of r that the previous Krylov
// space still represents.
template <typename T>
__device__ __noinline__ void cta_finish_proj(Cycle *st, int k, const double *slots, int pld, int nblk, double *sh,
                                size_t sh_bytes)
{
    const int tid = threadIdx.x, nt = blockDim.x, wid = tid >> 5, lane = tid & 31;
    double *c = sh;                   // k + 1 values
    double *cs = sh + (kKmax + 2);    // rotations 0 .. k-1
    double *sn = cs + (kKmax + 2);
    for (int q = wid; q <= k; q += nt / 32) {
        const double sg = lane == 0 ? st->sigma[q] : 0.0;
        const double v = Acc<T>::reduce(slots, pld, nblk, q);
        if (lane == 0) c[q] = sg * v;
    }
    for (int i = tid; i < k; i += nt) {
        cs[i] = st->cs[i];
        sn[i] = st->sn[i];
    }
    __syncthreads();
    if (tid == 0) {
        double a = c[0];
        for (int i = 0; i < k; ++i) {
            const double b = c[i + 1];
            st->g[i] = fma(cs[i], a, sn[i] * b);
            a = fma(-sn[i], a, cs[i] * b);
        }
        st->nproj += 1;
    }
    __syncthreads();
    cta_solve_r(st, k, sh, sh_bytes);
}

// ---------------------------------------------------------------- the pass kernel

// Threads: eight compute warps (kThreads) and one producer warp that issues the stage copies.
constexpr int kGsThreads = kThreads + 32;

template <typename T, int KM>
__global__ void __launch_bounds__(kGsThreads) k_gs(GsArgs a, Cycle *st, const __grid_constant__ CUtensorMap tmap)
{
    using C = GsCfg<T, KM>;
    constexpr int TR = C::TR, TPR = C::TPR, RPT = C::RPT, RPL = C::RPL, CPW = C::CPW;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kGsMaxStages];
    __shared__ T s_wn[TR];
    __shared__ T s_part[TPR > 1 ? TPR : 1][TPR > 1 ? TR : 1];
    __shared__ T s_coef[KM];
    __shared__ double scratch[33];
    __shared__ int s_last;
    __shared__ int s_int[3];
    __shared__ int s_timeout;
    __shared__ double s_wsq;  // pass 2: ||w'||^2

    const int op = a.op;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool prod = wid == kThreads / 32;  // the producer warp
    const T *__restrict__ U = (const T *)a.U;
    T *w = (T *)a.w;
    const bool need_w = (op != kGsCombine);
    T *stage0 = reinterpret_cast<T *>(smem);
    const int nst = a.nstages;                            // pipeline depth (2..kGsMaxStages)
    const long long SS = (long long)(a.kstage + 1) * TR;  // elements per stage: kst columns + w
    const uint32_t colb = TR * (uint32_t)sizeof(T);
    if (tid == 0) {
        for (int q = 0; q < nst; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
        s_timeout = 0;
    }
    __syncthreads();

    // Stage fills, by the lanes of the producer warp.  A stage's barrier completes once lane 0 has arrived
    // (with the w copy) and all bytes have landed, so the basis columns may be requested earlier.
    // With a tensor map (iteration passes) the tile's kc = kstage columns are one box copy;
    // otherwise one bulk copy per column.
    auto issue_cols = [&](long long tile, int stage, int kc) {
        T *sU = stage0 + stage * SS;
        if (lane == 0) mbar_expect_tx(&bars[stage], colb * (uint32_t)kc);
        __syncwarp();
        fence_proxy_async_smem();
        const long long row0 = tile * TR;
        if (a.use_tmap) {
            if (lane == 0) {
                if constexpr (TR <= 256)
                    tma_load_2d(sU, &tmap, (int)row0, 0, &bars[stage]);
                else
                    tma_load_3d(sU, &tmap, 0, (int)(row0 / 256), 0, &bars[stage]);
            }
        } else {
            for (int c = lane; c < kc; c += 32)
                bulk_g2s(sU + c * TR, U + (long long)c * a.ldu + row0, colb, &bars[stage]);
        }
    };
    auto issue_w = [&](long long tile, int stage) {
        if (lane == 0) {
            mbar_arrive_expect_tx(&bars[stage], need_w ? colb : 0u);
            if (need_w) bulk_g2s(stage0 + stage * SS + (long long)a.kstage * TR, w + tile * TR, colb, &bars[stage]);
        }
    };
    // the CTA's q-th tile (q < my_tiles); a reversed pass visits the same tiles last to first, so it
    // starts on the basis rows the previous (forward) pass read last, which are still in L2
    const long long my_tiles = blockIdx.x < a.ntiles ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_of = [&](long long q) {
        return blockIdx.x + (a.rev ? my_tiles - 1 - q : q) * (long long)gridDim.x;
    };

    // Before the wait on the predecessor: the basis columns of the first stages.  For the
    // iteration passes the host's column count is the device's k, and the columns were written
    // at least two launches back (every kernel of the stream releases its dependents only after
    // its own wait, so all launches before the predecessor are complete here).  Pass 2 also
    // takes w early: the SpMV wrote it two launches back and pass 1 only reads it.
    const bool early = !a.kcols_from_k;
    const bool early_w = early && op == kGsUpdDot;
    if (early && prod) {
        for (int q = 0; q < nst - 1; ++q)
            if (q < my_tiles) {
                issue_cols(tile_of(q), q, a.kstage);
                if (early_w) issue_w(tile_of(q), q);
            }
    }

    pdl_wait();
    pdl_trigger();
    bool skip = a.kcols_from_k ? (st->k == 0) : (st->cycle_done != 0);
    if (op == kGsProj) skip = skip || st->stop;
    int k = a.kcols_from_k ? st->k + (op == kGsProj ? 1 : 0) : st->j + 1;
    if (op == kGsUpdNorm) {
        // pass 3 follows the finalisation of its own iteration (done by pass 2, which advanced j to
        // the host's column count); it also runs when that finalisation ended the cycle, since the
        // new basis vector is used by the restart projection
        skip = st->j != a.kstage;
        k = a.kstage;
    }
    // the host's bound must cover k (else refuse rather than overrun a stage)
    const bool bad = !skip && (k > KM || k > a.kstage || (early && k != a.kstage));
    if (skip || bad) {
        if (bad && tid == 0 && blockIdx.x == 0) timeout_stop(st);
        if (early) {  // the copies already requested land before the CTA's shared memory is released
            if (prod && lane == 0 && !early_w)
                for (int q = 0; q < nst - 1; ++q)
                    if (q < my_tiles) mbar_arrive(&bars[q]);
            if (tid == 0)
                for (int q = 0; q < nst - 1; ++q)
                    if (q < my_tiles) mbar_wait_bounded(&bars[q], 0, kWaitLimitNs);
        }
        return;
    }
    T *out = a.out_follow ? (T *)a.U + (long long)k * a.ldu : (T *)a.out;
    // pass 3's coefficients h2 .* sigma are formed here: the finalisation may have replaced coef by
    // the cycle-end combination's
    for (int c = tid; c < KM; c += kThreads)
        s_coef[c] = (c < k && op != kGsDot && op != kGsProj)
                        ? (T)(op == kGsUpdNorm ? st->h2[c] * st->sigma[c] : st->coef[c])
                        : T(0);

    // prologue: the first nst - 1 tiles (their remaining copies); tile it + nst - 1 is issued at
    // the start of iteration it into the stage freed by iteration it - 1
    if (prod) {
        for (int q = 0; q < nst - 1; ++q)
            if (q < my_tiles) {
                if (!early) issue_cols(tile_of(q), q, k);
                if (!early_w) issue_w(tile_of(q), q);
            }
    }
    __syncthreads();

    Acc<T> acc[CPW];
    Acc<T> nrm;  // float32 path: float32 Kahan sum per thread, float64 across threads
    bool timed_out = false;
    int it = 0;
    for (; it < my_tiles; ++it) {
        const long long tile = tile_of(it);
        const int stage = it % nst;
        if (prod) {
            // the producer refills the stage the previous iteration released, then meets the
            // compute warps at the end-of-tile barrier
            if (it + nst - 1 < my_tiles) {
                const long long nt = tile_of(it + nst - 1);
                issue_cols(nt, (it + nst - 1) % nst, k);
                issue_w(nt, (it + nst - 1) % nst);
            }
            __syncthreads();
            if (s_timeout) {
                timed_out = true;
                break;
            }
            continue;
        }
        // every compute thread waits for the stage; they agree on the outcome before any of them
        // enters a barrier the others might not reach
        const bool filled = mbar_wait_bounded(&bars[stage], (it / nst) & 1, kWaitLimitNs);
        if (bar_any(1, kThreads, !filled)) {  // the stage never filled: skip its work
            if (tid == 0) s_timeout = 1;
            __syncthreads();
            timed_out = true;
            break;
        }
        const T *sU = stage0 + stage * SS;
        const T *sw = sU + (long long)a.kstage * TR;
        const long long row0 = tile * TR;
        const T *dotvec = sw;
        if (op != kGsDot && op != kGsProj) {
            // update: wn = w - sum_c U[:, c] coef[c] on this tile
            if constexpr (TPR == 1) {
                T part[RPT];
#pragma unroll
                for (int r = 0; r < RPT; ++r) part[r] = T(0);
                for (int c = 0; c < k; ++c) {
                    const T cc = s_coef[c];
#pragma unroll
                    for (int r = 0; r < RPT; ++r) part[r] = fma(sU[c * TR + tid + r * kThreads], cc, part[r]);
                }
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int row = tid + r * kThreads;
                    const T wn = (op == kGsCombine ? T(0) : sw[row]) - part[r];
                    if (op == kGsUpdDot) {
                        w[row0 + row] = wn;
                        s_wn[row] = wn;
                        nrm.add(wn * wn);
                    } else {
                        out[row0 + row] = wn;
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");  // compute warps only
            } else {
                const int row = tid % TR, q = tid / TR;
                T part = T(0);
                for (int c = q; c < k; c += TPR) part = fma(sU[c * TR + row], s_coef[c], part);
                s_part[q][row] = part;
                asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
                if (tid < TR) {
                    T sum = s_part[0][row];
#pragma unroll
                    for (int p = 1; p < TPR; ++p) sum += s_part[p][row];
                    const T wn = (op == kGsCombine ? T(0) : sw[row]) - sum;
                    if (op == kGsUpdDot) {
                        w[row0 + row] = wn;
                        s_wn[row] = wn;
                        nrm.add(wn * wn);
                    } else {
                        out[row0 + row] = wn;
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
            }
            dotvec = s_wn;
        } else {
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int row = tid + r * kThreads;
                if (row < TR) {
                    const T t = sw[row];
                    nrm.add(t * t);
                }
            }
        }
        if (op == kGsDot || op == kGsUpdDot || op == kGsProj) {
#pragma unroll
            for (int i = 0; i < CPW; ++i) {
                const int c = wid + 8 * i;
                if (c < k) {
                    T s = T(0);
#pragma unroll
                    for (int r = 0; r < RPL; ++r) s = fma(sU[c * TR + r * 32 + lane], dotvec[r * 32 + lane], s);
                    acc[i].add(s);
                }
            }
        }
        __syncthreads();  // every thread is done with this stage before it is refilled
        if (s_timeout) {
            timed_out = true;
            break;
        }
    }
    if (timed_out) {
        if (tid == 0) timeout_stop(st);
        // copies already issued into the stages may still land: wait for them (bounded) first
        for (int q = 0; q < nst - 1; ++q) mbar_wait_bounded(&bars[(it + q) % nst], ((it + q) / nst) & 1, kWaitLimitNs);
        return;
    }

    // per-CTA partial sums: one 8-byte slot per column and CTA (a compensated float32 pair for the
    // float32 basis), column stride pld = nblk rounded up to even so that slots load in pairs
    const int pld = (a.nblk + 1) & ~1;
    const bool want_dots = op == kGsDot || op == kGsUpdDot || op == kGsProj;
    const bool want_norm = op == kGsDot || op == kGsUpdDot;
    if (want_dots && !prod) {
#pragma unroll
        for (int i = 0; i < CPW; ++i) {
            const int c = wid + 8 * i;
            if (c < k) acc[i].store_warp_total(a.partials + (long long)c * pld + blockIdx.x);
        }
    }
    if (want_norm) nrm.store_block_total(a.partials + (long long)kKmax * pld + blockIdx.x, scratch);
    if (op == kGsCombine || op == kGsUpdNorm) return;  // pass 3 is an update only: no reduction

    const int tk = op == kGsProj ? 6 : 2 + op;  // ticket 6 is the plain combination's, which has no last CTA
    if (last_block_done(&st->ticket[tk], &s_last)) {
        if (op == kGsProj) {
            cta_finish_proj<T>(st, k - 1, a.partials, pld, a.nblk, reinterpret_cast<double *>(smem),
                               (size_t)nst * (size_t)SS * sizeof(T));
        } else {
            // passes 1 and 2: each warp sums the slots of its columns and finalises them: the
            // pass's Hessenberg coefficients h = sigma .* sum and the next update's coefficients
            // coef = h .* sigma (sigma is loaded ahead of the sum); the norm is job k (pass 1:
            // ||w||^2, the breakdown scale; pass 2: ||w'||^2 of the once-orthogonalised vector)
            double *h_out = op == kGsDot ? st->h1 : st->h2;
            const int njobs = k + (want_norm ? 1 : 0);
            for (int q = wid; q < njobs; q += kGsThreads / 32) {
                const bool is_norm = q == k;
                const double sg = (!is_norm && lane == 0) ? st->sigma[q] : 0.0;
                const double v = Acc<T>::reduce(a.partials, pld, a.nblk, is_norm ? kKmax : q);
                if (lane == 0) {
                    if (is_norm) {
                        if (op == kGsDot)
                            st->w0sq = v;
                        else
                            s_wsq = v;
                    } else {
                        const double h = sg * v;
                        h_out[q] = h;
                        st->coef[q] = h * sg;
                    }
                }
            }
            if (op == kGsUpdDot) {
                // the Hessenberg column is complete: ||v_{j+1}||^2 = ||w'||^2 - ||h2||^2 (v_{j+1} =
                // w' - V h2 with V orthonormal), so pass 3 needs no reduction of its own
                __syncthreads();
                cta_finish_pass3<T>(st, k - 1, s_wsq, reinterpret_cast<double *>(smem),
                                    (size_t)nst * (size_t)SS * sizeof(T), s_int);
            }
        }
        if (tid == 0) st->ticket[tk] = 0;
    }
}

// ---------------------------------------------------------------- x += Z y (flexible cycle end)

// x[r] += sum_c y_c U[r, c] over the k columns the finished cycle (or the restart projection) left
// coefficients for, r < n: float64 x and y, U float32 (float64 for a float64 basis), accumulated as
// XAcc describes.  Once per cycle; each thread keeps its row's k column loads in flight.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_combine_x(const T *__restrict__ U, long long ld, long long n,
                                                        double *__restrict__ x, Cycle *st, int skip_if_stop)
{
    __shared__ T s_hi[kKmax], s_lo[kKmax];
    pdl_wait();
    pdl_trigger();
    const int k = st->k;
    if (k == 0 || (skip_if_stop && st->stop)) return;
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        const double y = st->y[c];
        const T hi = (T)y;
        s_hi[c] = hi;
        s_lo[c] = (T)(y - (double)hi);
    }
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        XAcc<T> xa;
        int c = 0;
        for (; c + 8 <= k; c += 8) {
            T z[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) z[u] = __ldcs(U + (long long)(c + u) * ld + r);
#pragma unroll
            for (int u = 0; u < 8; ++u) xa.add(z[u], s_hi[c + u], s_lo[c + u]);
        }
        for (; c < k; ++c) xa.add(__ldcs(U + (long long)c * ld + r), s_hi[c], s_lo[c]);
        x[r] += xa.value();
    }
}

cudaError_t launch_combine_x(int prec, const void *U, long long ld, long long n, double *x, Cycle *st,
                             int skip_if_stop, int num_sms, cudaStream_t s)
{
    long long grid = (n + kThreads - 1) / kThreads;
    if (grid > 8LL * num_sms) grid = 8LL * num_sms;
    if (grid < 1) grid = 1;
    if (prec == kF64)
        return launch_pdl(k_combine_x<double>, dim3((unsigned)grid), dim3(kThreads), 0, s, (const double *)U, ld, n,
                          x, st, skip_if_stop);
    return launch_pdl(k_combine_x<float>, dim3((unsigned)grid), dim3(kThreads), 0, s, (const float *)U, ld, n, x, st,
                      skip_if_stop);
}

// ---- host side: bucket selection, occupancy (cached per instantiation), launch

namespace {

// Tensor-map copies of the basis tiles (PPG_GS_TMAP=0 in the environment: one bulk copy per column).
bool gs_tmap_enabled()
{
    static const bool v = [] {
        const char *e = getenv("PPG_GS_TMAP");
        return !(e && atoi(e) == 0);
    }();
    return v;
}

// The driver's tensor-map encoder, looked up once through the runtime (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// Tensor map of the first kcols columns of the column-major basis U (ld elements per column) whose
// box is one tile of a stage, TR rows x kcols columns, laid out column after column as the stage
// keeps it.  A box side holds at most 256 elements, so the rows are a 2-D (row chunk, chunk index)
// pair of 256 x TR/256 when TR > 256: three dimensions (rows in chunk, chunk, column).  The tile at
// row r0 is then the box at (0, r0 / 256, 0), else at (r0, 0).  False when it cannot be made.
template <typename T>
bool basis_tmap(CUtensorMap *m, const void *U, long long ld, int kcols, int TR)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc || kcols < 1 || kcols > 256 || ((uintptr_t)U & 15u) != 0) return false;
    const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r;
    if (TR <= 256) {
        const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)kcols};
        const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(T)};
        const cuuint32_t box[2] = {(cuuint32_t)TR, (cuuint32_t)kcols};
        r = enc(m, dt, 2, const_cast<void *>(U), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        if (TR % 256 != 0 || ld % 256 != 0 || TR / 256 > 256) return false;
        const cuuint64_t dims[3] = {256, (cuuint64_t)(ld / 256), (cuuint64_t)kcols};
        const cuuint64_t strides[2] = {256 * sizeof(T), (cuuint64_t)ld * sizeof(T)};
        const cuuint32_t box[3] = {256, (cuuint32_t)(TR / 256), (cuuint32_t)kcols};
        r = enc(m, dt, 3, const_cast<void *>(U), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    return r == CUDA_SUCCESS;
}

template <typename T, int KM>
struct GsInst {
    static cudaError_t configure()
    {
        cudaError_t e = cudaFuncSetAttribute(k_gs<T, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             GsCfg<T, KM>::kSmemBudget);
        if (e == cudaSuccess)  // one L1 / shared-memory split for the kernels of an iteration
            e = cudaFuncSetAttribute(k_gs<T, KM>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        return e;
    }
    static cudaError_t launch(GsArgs a, int kcols, long long ld, int num_sms, Cycle *st, cudaStream_t s)
    {
        constexpr int TR = GsCfg<T, KM>::TR;
        const size_t stage_bytes = (size_t)(kcols + 1) * TR * sizeof(T);
        int nst = (int)(GsCfg<T, KM>::kSmemBudget / stage_bytes);
        if (nst > kGsMaxStages) nst = kGsMaxStages;
        if (nst > PPG_GS_STAGES) nst = PPG_GS_STAGES;
        if (nst < 2) return cudaErrorInvalidValue;
        a.kstage = kcols;
        a.nstages = nst;
        const size_t smem = (size_t)nst * stage_bytes;
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gs<T, KM>, kGsThreads, smem);
        if (per < 1) per = 1;
        a.ntiles = ld / TR;
        long long g = (long long)per * num_sms;
        if (g > a.ntiles) g = a.ntiles;
        a.nblk = (int)(g > 0 ? g : 1);
        // iteration passes (k = kcols on the device) of buckets whose tile columns are small copies
        CUtensorMap tm;
        memset(&tm, 0, sizeof tm);
        a.use_tmap = (!a.kcols_from_k && gs_tmap_enabled() && basis_tmap<T>(&tm, a.U, ld, kcols, TR)) ? 1 : 0;
        return launch_pdl(k_gs<T, KM>, dim3(a.nblk), dim3(kGsThreads), smem, s, a, st, tm);
    }
};

template <typename T>
cudaError_t gs_launch_t(int kcols, GsArgs a, long long ld, int num_sms, Cycle *st, cudaStream_t s)
{
    if (kcols <= 8) return GsInst<T, 8>::launch(a, kcols, ld, num_sms, st, s);
    if (kcols <= 16) return GsInst<T, 16>::launch(a, kcols, ld, num_sms, st, s);
    if (kcols <= 32) return GsInst<T, 32>::launch(a, kcols, ld, num_sms, st, s);
    if (kcols <= 64) return GsInst<T, 64>::launch(a, kcols, ld, num_sms, st, s);
    return GsInst<T, 128>::launch(a, kcols, ld, num_sms, st, s);
}

template <typename T>
cudaError_t gs_configure_t()
{
    cudaError_t e = GsInst<T, 8>::configure();
    if (e == cudaSuccess) e = GsInst<T, 16>::configure();
    if (e == cudaSuccess) e = GsInst<T, 32>::configure();
    if (e == cudaSuccess) e = GsInst<T, 64>::configure();
    if (e == cudaSuccess) e = GsInst<T, 128>::configure();
    return e;
}

}  // namespace

cudaError_t gs_configure()
{
    cudaError_t e = gs_configure_t<double>();
    if (e == cudaSuccess) e = gs_configure_t<float>();
    return e;
}

int gs_max_blocks(int num_sms) { return 16 * num_sms; }  // 3 CTAs per SM in practice

cudaError_t launch_gs(int prec, int kcols, long long ld, int num_sms, GsArgs a, Cycle *st, cudaStream_t s)
{
    if (kcols < 1 || kcols > kKmax) return cudaErrorInvalidValue;
    if (prec == kF64) return gs_launch_t<double>(kcols, a, ld, num_sms, st, s);
    return gs_launch_t<float>(kcols, a, ld, num_sms, st, s);
}

// ---------------------------------------------------------------- Gram matrix of Eq. 1 and its Cholesky solve

// The normal equations G y = r of Eq. 1 (G = (AV)^T AV, kk = deg + 1, column-major in shared memory,
// overwritten by its Cholesky factor L), by the whole CTA: column-by-column Cholesky with LAPACK
// POTRF's test (a pivot that is not > 0, NaN included, stops the factorisation with info = its 1-based
// order), then forward and back substitution with the leading block that factored.  The degree used is
// deg when info = 0, else info - 2 (the largest degree with no Cholesky failure, Section IV).
// info_out: [0] info, [1] degree used, [2] 1 if the coefficients are finite; coef_out: kk values
// (zero beyond the degree used).  Products and differences are rounded separately (no fused
// multiply-add), so a given G factors to the same bits as a plain IEEE evaluation of the same loops.
__device__ void cta_gram_solve(double *G, const double *r, double *y, int kk, int deg, double *coef_out, int *info_out,
                               int *s_info)
{
    const int tid = threadIdx.x;
    if (tid == 0) *s_info = 0;
    __syncthreads();
    for (int j = 0; j < kk; ++j) {
        if (tid == 0) {
            double d = G[j + j * kk];
            for (int p = 0; p < j; ++p) d = __dsub_rn(d, __dmul_rn(G[j + p * kk], G[j + p * kk]));
            if (!(d > 0.0))
                *s_info = j + 1;
            else
                G[j + j * kk] = sqrt(d);
        }
        __syncthreads();
        if (*s_info) break;
        const double ljj = G[j + j * kk];
        for (int i = j + 1 + tid; i < kk; i += blockDim.x) {
            double s = G[i + j * kk];
            for (int p = 0; p < j; ++p) s = __dsub_rn(s, __dmul_rn(G[i + p * kk], G[j + p * kk]));
            G[i + j * kk] = s / ljj;
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int info = *s_info;
        const int used = info ? info - 2 : deg;
        for (int i = 0; i < kk; ++i) y[i] = 0.0;
        const int m = used + 1;
        for (int i = 0; i < m; ++i) {
            double s = r[i];
            for (int p = 0; p < i; ++p) s = __dsub_rn(s, __dmul_rn(G[i + p * kk], y[p]));
            y[i] = s / G[i + i * kk];
        }
        for (int i = m - 1; i >= 0; --i) {
            double s = y[i];
            for (int p = i + 1; p < m; ++p) s = __dsub_rn(s, __dmul_rn(G[p + i * kk], y[p]));
            y[i] = s / G[i + i * kk];
        }
        bool finite = true;
        for (int i = 0; i < kk; ++i) {
            coef_out[i] = (i < m) ? y[i] : 0.0;
            finite = finite && isfinite(coef_out[i]);
        }
        info_out[0] = info;
        info_out[1] = used;
        info_out[2] = finite ? 1 : 0;
    }
}

// B holds the power basis [v0, A v0, ..., A^{d+1} v0] column-major (ld rows per column,
// rows beyond n zero).  One streaming pass forms every inner product B_a . B_b
// (0 <= a <= b <= d+1) from TMA-staged row tiles; the last CTA reduces them, factors
// G = (AV)^T AV (columns 1..d+1) by Cholesky with LAPACK POTRF's test (a pivot that is
// not > 0, NaN included, stops the factorisation with info = its 1-based order), and
// solves G y = (AV)^T v0 with the leading block that factored.  The degree used is d
// when info = 0, else info - 2 (the largest degree with no Cholesky failure, Section IV).
constexpr int kGramTR = 64;
constexpr int kGramStride = kGramTR + 2;  // padded column stride: 16-byte aligned, spreads banks
constexpr int kGramCols = 64;             // d + 2 <= 64
constexpr int kGramPairsPerThread = (kGramCols * (kGramCols + 1) / 2 + kThreads - 1) / kThreads;

__global__ void __launch_bounds__(kThreads) k_gram_cholesky(int n, long long ld, const double *__restrict__ B,
                                                             int deg, long long ntiles, double *partials,
                                                             double *coef_out, int *info_out, Cycle *st)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_last;
    __shared__ int s_info;
    double *stage0 = reinterpret_cast<double *>(smem);
    const int ncol = deg + 2;
    const int npair = ncol * (ncol + 1) / 2;
    const int tid = threadIdx.x;
    constexpr int TR = kGramTR;
    const long long stage_elems = (long long)kGramCols * kGramStride;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](long long tile, int stage) {
        double *sB = stage0 + stage * stage_elems;
        const uint32_t colb = TR * 8u;
        mbar_arrive_expect_tx(&bars[stage], colb * (uint32_t)ncol);
        for (int c = 0; c < ncol; ++c) bulk_g2s(sB + c * kGramStride, B + c * ld + tile * TR, colb, &bars[stage]);
    };
    if (tid == 0) {
        if (blockIdx.x < ntiles) issue(blockIdx.x, 0);
        if (blockIdx.x + (long long)gridDim.x < ntiles) issue(blockIdx.x + (long long)gridDim.x, 1);
    }
    // pair p -> (a, b), a <= b, row-major over the upper triangle
    int pa[kGramPairsPerThread], pb[kGramPairsPerThread];
    double acc[kGramPairsPerThread];
#pragma unroll
    for (int i = 0; i < kGramPairsPerThread; ++i) {
        int p = tid + i * kThreads;
        int a = 0, b = 0;
        if (p < npair) {
            int rem = p;
            a = 0;
            while (rem >= ncol - a) {
                rem -= ncol - a;
                ++a;
            }
            b = a + rem;
        }
        pa[i] = a;
        pb[i] = b;
        acc[i] = 0.0;
    }
    bool timed_out = false;
    int it = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int stage = it & 1;
        if (!mbar_wait_bounded(&bars[stage], (it >> 1) & 1, kWaitLimitNs)) {
            timed_out = true;
            break;
        }
        const double *sB = stage0 + stage * stage_elems;
#pragma unroll
        for (int i = 0; i < kGramPairsPerThread; ++i) {
            if (tid + i * kThreads < npair) {
                const double *x = sB + pa[i] * kGramStride, *y = sB + pb[i] * kGramStride;
                double s = 0.0;
                for (int r = 0; r < TR; ++r) s = fma(x[r], y[r], s);
                acc[i] += s;
            }
        }
        __syncthreads();
        if (tid == 0) {
            const long long nt = tile + 2LL * gridDim.x;
            if (nt < ntiles) {
                fence_proxy_async_smem();
                issue(nt, stage);
            }
        }
    }
    if (timed_out) {
        if (tid == 0) timeout_stop(st);
        // copies already issued into either stage may still land: wait for them (bounded) first
        mbar_wait_bounded(&bars[it & 1], (it >> 1) & 1, kWaitLimitNs);
        mbar_wait_bounded(&bars[(it + 1) & 1], ((it + 1) >> 1) & 1, kWaitLimitNs);
        return;
    }
#pragma unroll
    for (int i = 0; i < kGramPairsPerThread; ++i) {
        const int p = tid + i * kThreads;
        if (p < npair) partials[(long long)p * gridDim.x + blockIdx.x] = acc[i];
    }
    if (!last_block_done(&st->ticket[7], &s_last)) return;

    // ---- last CTA: reduce, factor, solve
    const int kk = deg + 1;
    double *G = stage0;             // kk x kk, column-major (ld kk)
    double *r = stage0 + kk * kk;   // kk
    double *y = r + kk;             // kk
    const int lane = tid & 31, wid = tid >> 5;
    for (int p = wid; p < npair; p += kThreads / 32) {
        const double v = reduce_partials(partials, gridDim.x, p);
        if (lane == 0) {
            int rem = p, a = 0;
            while (rem >= ncol - a) {
                rem -= ncol - a;
                ++a;
            }
            const int b = a + rem;
            if (a == 0) {
                if (b > 0) r[b - 1] = v;
            } else {
                G[(a - 1) + (b - 1) * kk] = v;
                G[(b - 1) + (a - 1) * kk] = v;
            }
        }
    }
    cta_gram_solve(G, r, y, kk, deg, coef_out, info_out, &s_info);
    if (tid == 0) st->ticket[7] = 0;
}

// Standalone use of the same factorisation and solve on a caller-given Gram matrix (tests).
__global__ void __launch_bounds__(kThreads) k_gram_solve(const double *__restrict__ Gin, const double *__restrict__ rin,
                                                         int deg, double *coef_out, int *info_out)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_info;
    const int kk = deg + 1;
    double *G = reinterpret_cast<double *>(smem);
    double *r = G + kk * kk;
    double *y = r + kk;
    for (int e = threadIdx.x; e < kk * kk; e += blockDim.x) G[e] = Gin[e];
    for (int i = threadIdx.x; i < kk; i += blockDim.x) r[i] = rin[i];
    __syncthreads();
    cta_gram_solve(G, r, y, kk, deg, coef_out, info_out, &s_info);
}

cudaError_t launch_gram_solve(const double *G, const double *r, int deg, double *coef_out, int *info_out,
                              cudaStream_t s)
{
    const int kk = deg + 1;
    const size_t smem = sizeof(double) * (size_t)(kk * kk + 2 * kk);
    k_gram_solve<<<1, kThreads, smem, s>>>(G, r, deg, coef_out, info_out);
    return cudaGetLastError();
}

int gram_grid(int num_sms)
{
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gram_cholesky, kThreads,
                                                  2 * sizeof(double) * kGramCols * kGramStride);
    if (per < 1) per = 1;
    return per * num_sms;
}

cudaError_t gram_configure()
{
    return cudaFuncSetAttribute(k_gram_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * sizeof(double) * kGramCols * kGramStride));
}

cudaError_t launch_gram_cholesky(int n, long long ld, const double *B, int deg, double *partials, int nblk,
                                 double *coef_out, int *info_out, Cycle *st, cudaStream_t s)
{
    const long long ntiles = ld / kGramTR;
    int grid = nblk;
    if (grid > ntiles) grid = (int)ntiles;
    k_gram_cholesky<<<grid, kThreads, 2 * sizeof(double) * kGramCols * kGramStride, s>>>(n, ld, B, deg, ntiles, partials,
                                                                                    coef_out, info_out, st);
    return cudaGetLastError();
}

}  // namespace ppg
