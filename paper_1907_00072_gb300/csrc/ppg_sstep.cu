// ppg_sstep.cu -- s-step GMRES with the polynomial preconditioner (Loe, Thornquist, Boman,
// Section VII: inside an s-step method, orthogonalisation happens once per deg * s SpMVs).
//
// The paper proposes the combination without giving an algorithm; this file takes the standard
// s-step construction.  A block of sb vectors is built from the last orthonormal basis column q_k:
//   Newton vectors   z_1 = (B - theta I) q_k,  z_{i+1} = (B - theta I) z_i      (B = A p(A), raw:
//                    the SpMV chain writes them to basis columns k + 1 .. k + sb, no reductions)
//   pass 1 (dot)      P = Q^T Z, and ||z_i||^2                       (one global reduction)
//   pass 2 (upd+dot)  Z -= Q C1,  C2 = Q^T Z, and Z^T Z                (one global reduction)
//   finalisation      the projected block's Gram matrix G = Z^T Z - C2^T C2 (Pythagoras) = R^T R
//                     (Cholesky), the block's Hessenberg columns
//                     H[:, k .. k+sb-1] = (S T - [H_old S_a; 0]) S_b^{-1}  (S: the change of basis
//                     [q_k, z_1 .. z_sb] = [Q, Q_new] S; T: theta on the diagonal, 1 below), the
//                     Givens rotations and GMRES's tests column by column
//   pass 3 (upd+tri)  Q_new = (Z - Q C2) R^{-1} into the block's columns (no reduction)
// Each pass streams tiles of 256 rows of the k + 1 + sb columns into shared memory with cp.async
// (16-byte copies, no barrier waits) and accumulates per-thread sums; the per-CTA sums are reduced in
// a fixed order by a second kernel whose last CTA finishes the pass, so results are deterministic.
// A Cholesky pivot below tau ||z_j||^2 means z_{j+1} lies in the span already built: the block
// then ends with j + 1 columns, the last one with a zero subdiagonal entry (a lucky breakdown).
// Flexible float32 form: each chain keeps P_i = p(A) u_i (u_0 = q_k, u_i = z_i); the block's
// preconditioned columns (P_blk - Z_old S_a) S_b^{-1} satisfy A Z = [Q, Q_new] H exactly as built, and
// are kept as Z = P M with M extended by the finalisation (y <- M y before x += Z y).
#include <cuda_runtime.h>

#include "ppg_cycle.cuh"
#include "ppg_internal.h"

namespace ppg {

namespace {

constexpr int kTR = 256;      // rows per tile
constexpr int kBT = 512;      // threads of a pass CTA: two per row in the update phase
constexpr int kBW = kBT / 32; // its warps
constexpr int kMaxStages = 8;

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// waits until at most n of this thread's copy groups are pending (n < kMaxStages)
__device__ __forceinline__ void cp_async_wait(int n)
{
    switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;" ::: "memory"); break;
    }
}

// A running sum per thread: float64 directly; float32 with Kahan compensation (the Gram matrix
// decides the Cholesky factor, whose error grows with the square of the block's condition).
template <typename T>
struct KSum {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct KSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// 16-byte vectors of V consecutive rows of one column (float4 / double2)
template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using type = float4;
    static constexpr int V = 4;
    static __device__ __forceinline__ float dot(const float4 &a, const float4 &b)
    {
        return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
    }
    static __device__ __forceinline__ void fnma(float4 &w, const float4 &u, float c)
    {
        w.x = fmaf(-u.x, c, w.x);
        w.y = fmaf(-u.y, c, w.y);
        w.z = fmaf(-u.z, c, w.z);
        w.w = fmaf(-u.w, c, w.w);
    }
    static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    static __device__ __forceinline__ float get(const float4 &a, int q) { return q == 0 ? a.x : q == 1 ? a.y : q == 2 ? a.z : a.w; }
};
template <>
struct Vec<double> {
    using type = double2;
    static constexpr int V = 2;
    static __device__ __forceinline__ double dot(const double2 &a, const double2 &b) { return fma(a.y, b.y, a.x * b.x); }
    static __device__ __forceinline__ void fnma(double2 &w, const double2 &u, double c)
    {
        w.x = fma(-u.x, c, w.x);
        w.y = fma(-u.y, c, w.y);
    }
    static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ double get(const double2 &a, int q) { return q == 0 ? a.x : a.y; }
};

// Sums over the CTA, in a fixed order, of per-thread values v[slot] held by groups of WPG warps (group
// g: warps g * WPG .. (g + 1) * WPG - 1; other threads hold zeros).  Output o of nout is slot o / G of
// group o % G (interleaved) or slot o % NS of group o / NS.  Warp trees, then the group's warp totals
// in warp order, to out_slots[o * pld + blockIdx.x].  red: >= kBW * NS doubles.
template <int NS>
__device__ __forceinline__ void group_sums(const double (&v)[NS], bool interleaved, int G, int WPG, int nout,
                                           double *red, double *out_slots, int pld)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const double t = warp_sum(v[q]);
        if (lane == 0) red[wid * NS + q] = t;
    }
    __syncthreads();
    const int o = threadIdx.x;
    if (o < nout) {
        const int g = interleaved ? o % G : o / NS, q = interleaved ? o / G : o % NS;
        double t = 0.0;
        for (int w = g * WPG; w < (g + 1) * WPG; ++w) t += red[w * NS + q];
        out_slots[(long long)o * pld + blockIdx.x] = t;
    }
}

// The CTA's tiles (rows row0 .. row0 + 255 of basis columns 0 .. ncol - 1, column c at stage +
// c * kTR) pass through nst shared-memory stages filled with cp.async, nst - 1 tiles ahead of the one
// body(stage, row0) works on.  Rows at or beyond n read as zero.  body may modify its stage.
template <typename T, typename Body>
__device__ __forceinline__ void for_each_tile(T *sm, int nst, const T *U, long long ld, int ncol, int n,
                                              long long ntiles, Body body)
{
    constexpr int kPer = 16 / (int)sizeof(T);  // elements per 16-byte copy
    constexpr int kChunks = kTR / kPer;        // copies per column (64 or 128)
    constexpr int kColsPer = kBT / kChunks;    // columns one pass of the CTA's threads covers
    const int q = threadIdx.x % kChunks, c0 = threadIdx.x / kChunks;
    const long long stage_elems = (long long)ncol * kTR;
    auto issue = [&](long long tile, int stg) {  // commits one group, empty past the last tile
        if (tile < ntiles) {
            T *dst = sm + stg * stage_elems + c0 * kTR + q * kPer;
            const T *src = U + tile * kTR + c0 * ld + q * kPer;
            for (int c = c0; c < ncol; c += kColsPer) {
                cp_async16(dst, src);
                dst += kColsPer * kTR;
                src += kColsPer * ld;
            }
        }
        cp_async_commit();
    };
    const long long step = gridDim.x;
    for (int t = 0; t < nst - 1; ++t) issue(blockIdx.x + t * step, t);
    int it = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += step, ++it) {
        const int stg = it % nst;
        // the stage tile it - 1 used (released by the barrier that ended it) gets tile it + nst - 1
        issue(tile + (long long)(nst - 1) * step, (it + nst - 1) % nst);
        cp_async_wait(nst - 1);
        __syncthreads();
        T *cur = sm + stg * stage_elems;
        const long long row0 = tile * kTR;
        if (row0 + kTR > n) {  // the ragged last tile: its padding rows count as zero
            const int t = threadIdx.x;
            if (t < kTR && row0 + t >= n)
                for (int c = 0; c < ncol; ++c) cur[c * kTR + t] = T(0);
            __syncthreads();
        }
        body(cur, row0);
        __syncthreads();  // the stage is consumed before it is refilled
    }
    cp_async_wait(0);  // the empty groups committed past the last tile
}

// The update of the block's columns on one tile, W -= U coef, written to the tile and (kStore, rows
// below n) to HBM.  Thread t < RG * CG takes row group t % RG (V consecutive rows) and the block's
// columns 2 (t / RG) and 2 (t / RG) + 1; s_coef has SBP = 2 CG columns (zeros beyond SB).  (Splitting
// the sum over c among all the CTA's warps, with the partial sums meeting in shared memory, measured
// slower.)
template <typename T, int SB, bool kStore = true>
__device__ __forceinline__ void tile_update(T *cur, int kc, const T *s_coef, T *W, long long ld, long long row0, int n)
{
    using VT = typename Vec<T>::type;
    constexpr int V = Vec<T>::V, RG = kTR / V, CG = (SB + 1) / 2, SBP = 2 * CG;
    static_assert(RG * CG <= kBT, "update threads");
    const int t = threadIdx.x;
    if (t >= RG * CG) return;
    const int rg = t % RG, ia = 2 * (t / RG), ib = ia + 1;
    VT *sW = reinterpret_cast<VT *>(cur + kc * kTR);
    const VT *sU = reinterpret_cast<const VT *>(cur);
    VT wa = sW[ia * RG + rg];
    VT wb = ib < SB ? sW[ib * RG + rg] : Vec<T>::zero();
#pragma unroll 4
    for (int c = 0; c < kc; ++c) {
        const VT u = sU[c * RG + rg];
        const T ca = s_coef[c * SBP + ia], cb = s_coef[c * SBP + ib];
        Vec<T>::fnma(wa, u, ca);
        Vec<T>::fnma(wb, u, cb);
    }
    sW[ia * RG + rg] = wa;
    if (ib < SB) sW[ib * RG + rg] = wb;
    if (!kStore) return;
    const long long r = row0 + (long long)rg * V;
    if (r + V <= n) {
        *reinterpret_cast<VT *>(W + ia * ld + r) = wa;
        if (ib < SB) *reinterpret_cast<VT *>(W + ib * ld + r) = wb;
    } else {
        for (int v = 0; v < V; ++v)
            if (r + v < n) {
                W[ia * ld + r + v] = Vec<T>::get(wa, v);
                if (ib < SB) W[ib * ld + r + v] = Vec<T>::get(wb, v);
            }
    }
}

// Passes 1 and 2 (KB >= k + 1 columns of Q, bucketed so that each of the 16 warps keeps KB / 16
// columns' sums; SB = the block size sb).  In the dot phase a lane takes V consecutive rows.
// Slots: P[c][i] at o = c * sb + i; pass 1 also ||z_i||^2 at o = (k + 1) * sb + i; pass 2 the Gram
// matrix of the updated block, pair p = tri_index(i, j) at o = (k + 1) * sb + p (a thread takes row
// group t % RG and the pairs p with p % PG = t / RG).
template <typename T, int KB, int SB>
__global__ void __launch_bounds__(kBT) k_bgs_dot(BgsArgs a, Cycle *st, SStep *ss, int nst)
{
    using VT = typename Vec<T>::type;
    constexpr int V = Vec<T>::V, RG = kTR / V, CG = (SB + 1) / 2, SBP = 2 * CG;
    constexpr int CPW = KB / kBW;
    constexpr int NG = SB * (SB + 1) / 2;
    constexpr int PG = kBT / RG;            // pair groups (8 float32, 4 float64)
    constexpr int NS = (NG + PG - 1) / PG;  // pairs per thread
    static_assert(CPW >= 1, "bucket below the warp count");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    __shared__ __align__(16) T s_coef[KB * SBP];
    __shared__ double red[kBW * (NS > 2 ? NS : 2)];
    pdl_wait();
    pdl_trigger();
    if (st->cycle_done || st->j != a.k) return;
    const int kc = a.k + 1, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool upd = a.op == kBgsUpdDot;
    for (int e = tid; e < KB * SBP; e += kBT) {
        const int c = e / SBP, i = e - c * SBP;
        s_coef[e] = (upd && c < kc && i < SB) ? (T)ss->coef[i][c] : T(0);
    }
    T *W = (T *)a.U + (long long)kc * a.ld;
    T acc[CPW][SB];
#pragma unroll
    for (int q = 0; q < CPW; ++q)
#pragma unroll
        for (int i = 0; i < SB; ++i) acc[q][i] = T(0);
    T nacc[2] = {T(0), T(0)};  // pass 1: ||W_i||^2 of this thread's two columns (update mapping)
    KSum<T> g[NS];             // pass 2: Gram pairs
    const int grg = tid % RG, gpg = tid / RG;
    __syncthreads();

    for_each_tile(sm, nst, (const T *)a.U, a.ld, kc + SB, a.n, a.ntiles, [&](T *cur, long long row0) {
        const VT *sW = reinterpret_cast<const VT *>(cur + kc * kTR);
        const VT *sU = reinterpret_cast<const VT *>(cur);
        if (upd) {
            tile_update<T, SB>(cur, kc, s_coef, W, a.ld, row0, a.n);
            __syncthreads();
            VT gw[SB];
#pragma unroll
            for (int i = 0; i < SB; ++i) gw[i] = sW[i * RG + grg];
            int p = 0;
#pragma unroll
            for (int i = 0; i < SB; ++i)
#pragma unroll
                for (int j = i; j < SB; ++j, ++p)
                    if (p % PG == gpg) g[p / PG].add(Vec<T>::dot(gw[i], gw[j]));
        } else if (tid < RG * CG) {
            const int rg = tid % RG, ia = 2 * (tid / RG), ib = ia + 1;
            const VT x = sW[ia * RG + rg];
            nacc[0] += Vec<T>::dot(x, x);
            if (ib < SB) {
                const VT y = sW[ib * RG + rg];
                nacc[1] += Vec<T>::dot(y, y);
            }
        }
        // P[c][i] += U[:, c] . W[:, i] over the tile: warp wid owns columns wid, wid + 16, ...
#pragma unroll
        for (int p = 0; p < RG / 32; ++p) {
            const int rg = lane + 32 * p;
            VT wv[SB];
#pragma unroll
            for (int i = 0; i < SB; ++i) wv[i] = sW[i * RG + rg];
#pragma unroll
            for (int q = 0; q < CPW; ++q) {
                const int c = wid + kBW * q;
                if (c < kc) {
                    const VT u = sU[c * RG + rg];
#pragma unroll
                    for (int i = 0; i < SB; ++i) acc[q][i] += Vec<T>::dot(u, wv[i]);
                }
            }
        }
    });
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
        const int c = wid + kBW * q;
#pragma unroll
        for (int i = 0; i < SB; ++i) {
            const double v = warp_sum((double)acc[q][i]);
            if (lane == 0 && c < kc) a.partials[(long long)(c * SB + i) * a.pld + blockIdx.x] = v;
        }
    }
    if (!upd) {
        // output i = 2 g + slot is held by the warps of column group g (RG / 32 warps each)
        double nv[2] = {(double)nacc[0], (double)nacc[1]};
        group_sums<2>(nv, false, CG, RG / 32, SB, red, a.partials + (long long)(kc * SB) * a.pld, a.pld);
    } else {
        double gv[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) gv[q] = g[q].value();
        group_sums<NS>(gv, true, PG, RG / 32, NG, red, a.partials + (long long)(kc * SB) * a.pld, a.pld);
    }
}

// Pass 3: W -= U coef (the second Gram-Schmidt pass's coefficients), then Q_new = W R^{-1} into
// columns k + 1 .. k + nq (nq = tri_cols, set by the finalisation; R^{-1} in tinv).  No reduction.
// After the update a thread takes row group t % RG and the new columns j with j % JG = t / RG.
template <typename T, int SB>
__global__ void __launch_bounds__(kBT) k_bgs_tri(BgsArgs a, Cycle *st, SStep *ss, int nst)
{
    using VT = typename Vec<T>::type;
    constexpr int V = Vec<T>::V, RG = kTR / V, CG = (SB + 1) / 2, SBP = 2 * CG;
    constexpr int JG = kBT / RG;  // column groups of the triangular step (8 float32, 4 float64)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    __shared__ __align__(16) T s_coef[kSColsMax * SBP];
    __shared__ T tv[kSMax * kSMax];
    __shared__ int s_last;
    pdl_wait();
    pdl_trigger();
    // the finalisation may have ended the cycle, but its columns are still formed (the cycle-end
    // combination reads them); nothing to do when it did not run (tri_cols 0) or ran for another block
    const int nq = ss->tri_cols;
    if (nq == 0 || ss->tri_base != a.k + 1) return;
    const int kc = a.k + 1, tid = threadIdx.x;
    const int rg = tid % RG, jg = tid / RG;
    for (int e = tid; e < kSColsMax * SBP; e += kBT) {
        const int c = e / SBP, i = e - c * SBP;
        s_coef[e] = (c < kc && i < SB) ? (T)ss->coef[i][c] : T(0);
    }
    for (int e = tid; e < kSMax * kSMax; e += kBT) {
        const int j = e / kSMax, i = e - j * kSMax;
        tv[e] = (i <= j && j < nq) ? (T)ss->tinv[e] : T(0);
    }
    T *W = (T *)a.U + (long long)kc * a.ld;
    __syncthreads();
    for_each_tile(sm, nst, (const T *)a.U, a.ld, kc + SB, a.n, a.ntiles, [&](T *cur, long long row0) {
        tile_update<T, SB, false>(cur, kc, s_coef, W, a.ld, row0, a.n);
        __syncthreads();
        const VT *sW = reinterpret_cast<const VT *>(cur + kc * kTR);
        const long long r = row0 + (long long)rg * V;
        for (int j = jg; j < nq; j += JG) {
            VT v = Vec<T>::zero();
            for (int i = 0; i <= j; ++i) Vec<T>::fnma(v, sW[i * RG + rg], -tv[j * kSMax + i]);
            if (r + V <= a.n) {
                *reinterpret_cast<VT *>(W + j * a.ld + r) = v;
            } else {
                for (int q = 0; q < V; ++q)
                    if (r + q < a.n) W[j * a.ld + r + q] = Vec<T>::get(v, q);
            }
        }
    });
    if (last_block_done(&ss->ticket[3], &s_last) && tid == 0) {
        ss->tri_cols = 0;
        ss->ticket[3] = 0;
    }
}

// Flexible form, before the combination x += Z y: y <- M y (Z = P M, P the stored chain vectors).
__global__ void __launch_bounds__(kThreads) k_sstep_flex_y(Cycle *st, SStep *ss, int skip_if_stop)
{
    __shared__ double sy[kSColsMax];
    pdl_wait();
    pdl_trigger();
    const int k = st->k;
    if (k == 0 || k > kSColsMax || (skip_if_stop && st->stop)) return;
    for (int r = threadIdx.x; r < k; r += blockDim.x) sy[r] = st->y[r];
    __syncthreads();
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        double v = 0.0;
        for (int j = r; j < k; ++j) v = fma(ss->M[j][r], sy[j], v);
        st->y[r] = v;
    }
}

// index of (i, j), i <= j < sb, in the packed upper triangle the Gram pass writes
__host__ __device__ constexpr int tri_index(int i, int j, int sb) { return i * sb - i * (i - 1) / 2 + (j - i); }

// The block's finalisation, by the last CTA of pass 3's reduction (all its threads).  red holds
// the Gram matrix of the projected block (packed upper triangle); sh: shared scratch of sh_bytes.
__device__ void cta_finish_block(const BgsArgs &a, Cycle *st, SStep *ss, const double *gram, double *sh,
                                 size_t sh_bytes)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int k = a.k, sb = a.sb;
    __shared__ double L[kSMax][kSMax];  // Cholesky factor, G = L L^T (R = L^T)
    __shared__ double s_gram[kSMax * (kSMax + 1) / 2], s_w0[kSMax], s_rl[kSMax];  // s_rl: 1 / L_jj
    __shared__ int s_f, s_bad, s_kdone;
    __shared__ double sc[4];  // tol * enorm, inner_rtol * beta (or -1), 1 / enorm, theta
    for (int e = tid; e < sb * (sb + 1) / 2; e += nt) s_gram[e] = gram[e];
    if (tid < sb) s_w0[tid] = ss->w0[tid];
    if (tid == 32) {
        const double bn = st->enorm, irt = st->inner_rtol;
        sc[0] = st->tol * bn;
        sc[1] = irt > 0.0 ? irt * st->beta : -1.0;
        sc[2] = 1.0 / bn;
        sc[3] = a.theta;
    }
    __syncthreads();
    if (tid == 0) {
        // left-looking Cholesky with the dependence test; row f of L (entries q < f) is complete
        // when pivot f fails, as the breakdown column needs
        int f = sb, bad = 0;
        for (int j = 0; j < sb && f == sb; ++j) {
            double d = s_gram[tri_index(j, j, sb)];
            for (int q = 0; q < j; ++q) d -= L[j][q] * L[j][q];
            if (!isfinite(d)) {
                bad = 1;
                f = j;
                break;
            }
            if (!(d > a.tau * s_w0[j])) {
                f = j;
                break;
            }
            const double l = sqrt(d), rl = 1.0 / l;
            L[j][j] = l;
            s_rl[j] = rl;
            for (int i = j + 1; i < sb; ++i) {
                double v = s_gram[tri_index(j, i, sb)];
                for (int q = 0; q < j; ++q) v -= L[i][q] * L[j][q];
                L[i][j] = v * rl;
            }
        }
        s_f = f;
        s_bad = bad;
    }
    __syncthreads();
    const int f = s_f;
    const bool brk = f < sb;
    const int sbp = brk ? f + 1 : sb;  // Hessenberg columns this block yields
    const int nq = brk ? f : sb;       // orthonormal columns it adds (Q_new)
    const int ns = k + 1 + sbp;        // rows of S and of the new columns
    // S (ns x (sbp + 1), column-major) and the new columns Hb (ns x sbp) in shared memory
    double *S = sh;
    double *Hb = S + ns * (sbp + 1);
    for (int e = tid; e < ns * (sbp + 1); e += nt) {
        const int col = e / ns, r = e - col * ns;
        double v = 0.0;
        if (col == 0) {
            v = r == k ? 1.0 : 0.0;
        } else {
            const int i = col - 1;  // z_{i+1} = Q C[i] + Q_new R[:, i]
            if (r <= k) {
                v = ss->C[i][r];
            } else {
                const int q = r - k - 1;
                if (q < i) v = L[i][q];
                else if (q == i && i < nq) v = L[i][i];
            }
        }
        S[e] = v;
    }
    __syncthreads();
    // Hb = S T - [H_old S_a; 0], T = theta on the diagonal and 1 below it (raw Newton vectors)
    const double theta = sc[3];
    for (int e = tid; e < ns * sbp; e += nt) {
        const int j = e / ns, r = e - j * ns;
        double v = theta * S[j * ns + r] + S[(j + 1) * ns + r];
        if (r <= k) {  // column q of H_old has rows 0 .. q + 1 (rows below hold older cycles' values)
            const double *Hr = st->H + r;
#pragma unroll 8
            for (int q = r > 0 ? r - 1 : 0; q < k; ++q) v -= Hr[(long long)q * kLdH] * S[j * ns + q];
        }
        Hb[e] = v;
    }
    __syncthreads();
    // Hb := Hb S_b^{-1}, S_b = S rows k .. k + sbp - 1 (upper triangular, diagonal 1, L_00, L_11, ...):
    // row by row
    for (int r = tid; r < ns; r += nt) {
        for (int j = 0; j < sbp; ++j) {
            double v = Hb[j * ns + r];
            for (int q = 0; q < j; ++q) v -= Hb[q * ns + r] * S[j * ns + k + q];
            Hb[j * ns + r] = j == 0 ? v : v * s_rl[j - 1];
        }
    }
    __syncthreads();
    // flexible form: the block's preconditioned columns Z_in = (P_blk - Z_old S_a) S_b^{-1} (the change of
    // basis that gives H), with Z = P M: M[:, k + j] = (e_{k+j} - M[:, 0..k-1] S_a[:, j]
    // - M[:, k..k+j-1] S_b[0..j-1, j]) / S_b[j][j], column by column, rows in parallel (zero below j)
    if (a.flex && !s_bad) {
        for (int j = 0; j < sbp; ++j) {
            const int col = k + j;
            for (int r = tid; r < kSColsMax; r += nt) {
                double v = 0.0;
                if (r <= col) {
                    v = r == col ? 1.0 : 0.0;
                    const double *Sj = S + j * ns;
#pragma unroll 8
                    for (int c = r; c < k; ++c) v -= ss->M[c][r] * Sj[c];  // M[c][r] = 0 for r > c
                    for (int q = 0; q < j; ++q)
                        if (r <= k + q) v -= ss->M[k + q][r] * Sj[k + q];
                    v = j == 0 ? v : v * s_rl[j - 1];
                }
                ss->M[col][r] = v;
            }
            __syncthreads();
        }
    }
    // the columns as built, then the cycle's earlier rotations 0 .. k-1 (one thread per column); the
    // serial part below works on shared-memory copies of the rotations, g and the columns (a dependent
    // access to the device state costs an L2 round trip) and the results are written back in parallel
    __shared__ double s_cs[kSColsMax], s_sn[kSColsMax], s_g[kSColsMax + 1];
    __shared__ int s_jend;
    int bad = s_bad;
    for (int e = tid; e < ns * sbp; e += nt) {
        const int j = e / ns, r = e - j * ns;
        const double h = Hb[e];
        if (r <= k + j + 1) st->H[(long long)(k + j) * kLdH + r] = h;
        if (!isfinite(h)) bad = 1;
    }
    if (bad) s_bad = 1;  // benign race: every writer stores 1
    for (int i = tid; i < k; i += nt) {
        s_cs[i] = st->cs[i];
        s_sn[i] = st->sn[i];
    }
    if (tid == 0) s_g[k] = st->g[k];
    __syncthreads();
    if (tid < sbp) {
        double *h = Hb + tid * ns;
        for (int i = 0; i < k; ++i) {
            const double c = s_cs[i], s = s_sn[i];
            const double x = h[i], y = h[i + 1];
            h[i] = c * x + s * y;
            h[i + 1] = -s * x + c * y;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int kdone = 0;
        if (s_bad) {
            st->error |= kErrNonfinite;
            st->stop = 1;
            st->cycle_done = 1;
            st->k = 0;
            st->j = k + 1;
            kdone = -1;
            s_jend = k;
            publish_progress(st, 1, k + 1);
        } else {
            long long it = st->iters;
            const long long maxit = st->maxit;
            const int m = st->m;
            int jend = k + sbp;
            for (int j = 0; j < sbp; ++j) {
                const int col = k + j;
                double *h = Hb + j * ns;
                for (int i = k; i < col; ++i) {  // this block's earlier rotations
                    const double c = s_cs[i], s = s_sn[i];
                    const double x = h[i], y = h[i + 1];
                    h[i] = c * x + s * y;
                    h[i + 1] = -s * x + c * y;
                }
                const double av = h[col], bv = h[col + 1];
                const double rr = sqrt(fma(av, av, bv * bv));
                double c = 1.0, s = 0.0;
                if (rr != 0.0) {
                    c = av / rr;
                    s = bv / rr;
                }
                s_cs[col] = c;
                s_sn[col] = s;
                h[col] = rr;
                h[col + 1] = 0.0;
                const double gj = s_g[col];
                s_g[col] = c * gj;
                s_g[col + 1] = -s * gj;
                const double res = fabs(s * gj);
                st->est = res * sc[2];
                it += 1;
                const bool last_brk = brk && j == sbp - 1;
                if (last_brk || col + 1 >= m || it >= maxit || res <= sc[0] || res <= sc[1]) {
                    kdone = col + 1;
                    jend = col + 1;
                    break;
                }
            }
            s_jend = jend;
            st->iters = it;
            st->nblocks += 1;
            st->nnewton += sb;
            ss->tri_base = k + 1;
            ss->tri_cols = nq;
            if (brk) {
                st->breakdown = 1;
                st->n_breakdowns += 1;
                // the column after the last one formed holds no basis vector (its subdiagonal entry is
                // zero): scale 0, as the single-vector breakdown leaves it, for the restart projection
                st->sigma[k + 1 + nq] = 0.0;
            }
            st->j = jend;
            if (kdone > 0) {
                st->k = kdone;
                st->cycle_done = 1;
            }
        }
        s_kdone = kdone;
    }
    __syncthreads();
    const int kdone = s_kdone, jend = s_jend;
    // R^{-1} for the triangular pass (R = L^T upper): column j by back substitution, one thread each
    if (kdone >= 0 && tid < nq) {
        const int j = tid;
        double x[kSMax];
        for (int i = j; i >= 0; --i) {
            double v = i == j ? 1.0 : 0.0;
            for (int q = i + 1; q <= j; ++q) v -= L[q][i] * x[q];
            x[i] = v * s_rl[i];
            ss->tinv[j * kSMax + i] = x[i];
        }
        st->sigma[k + 1 + j] = 1.0;
    }
    // the processed columns' rotations, g entries and rotated columns (R) back to the device state
    for (int col = k + tid; col < jend; col += nt) {
        st->cs[col] = s_cs[col];
        st->sn[col] = s_sn[col];
        st->g[col] = s_g[col];
    }
    if (tid == 0 && jend > k) st->g[jend] = s_g[jend];
    for (int e = tid; e < ns * sbp; e += nt) {
        const int j = e / ns, r = e - j * ns;
        if (k + j < jend && r <= k + j + 1) st->R[(long long)(k + j) * kLdH + r] = Hb[e];
    }
    __syncthreads();
    if (kdone > 0) {
        cta_solve_r(st, kdone, sh, sh_bytes);
        if (tid == 0) publish_progress(st, 1, kdone);
    } else if (kdone == 0 && tid == 0) {
        __threadfence();
        publish_progress(st, 0, jend);
    }
}

// Reduction of a pass's per-CTA sums (one warp per sum, fixed order), then the pass's
// finalisation by the last CTA.  Pass 1: C = C1, coef = sigma .* C1, the Newton norms.  Pass 2:
// C += C2, coef = sigma .* C2, and the block's Gram matrix after the second update by Pythagoras,
// G = W'^T W' - C2^T C2 (W' the once-orthogonalised block, C2 = Q^T W' small against it: the
// difference is exact to working precision), then the block's finalisation.
__global__ void __launch_bounds__(kThreads) k_bgs_finish(BgsArgs a, Cycle *st, SStep *ss)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_last, s_bad;
    __shared__ double s_c2[kSMax][kSColsMax];
    __shared__ double s_g[kSMax * (kSMax + 1) / 2];
    pdl_wait();
    pdl_trigger();
    if (st->cycle_done || st->j != a.k) return;
    const int kc = a.k + 1, sb = a.sb, lane = threadIdx.x & 31, ng = sb * (sb + 1) / 2;
    const int gw = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5), nw = gridDim.x * (kThreads / 32);
    const int nout = kc * sb + (a.op == kBgsDot ? sb : ng);
    for (int o = gw; o < nout; o += nw) {
        const double v = reduce_slots_f64(a.partials, a.pld, a.nblk, o);
        if (lane == 0) ss->red[o] = v;
    }
    if (!last_block_done(&ss->ticket[a.op], &s_last)) return;
    const int tid = threadIdx.x;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // C = sigma_c P (q_c = sigma_c U_c), summed over the passes; the next update subtracts U_c (sigma_c C_pass)
    for (int e = tid; e < kc * sb; e += kThreads) {
        const int c = e / sb, i = e - c * sb;
        const double sg = st->sigma[c];
        const double cv = sg * ss->red[e];
        if (!isfinite(cv)) s_bad = 1;
        ss->C[i][c] = a.op == kBgsDot ? cv : ss->C[i][c] + cv;
        ss->coef[i][c] = sg * cv;
        s_c2[i][c] = cv;
    }
    if (a.op == kBgsDot && tid < sb) {
        const double v = ss->red[kc * sb + tid];
        if (!isfinite(v)) s_bad = 1;  // a raw Newton vector overflowed (a zero one is a breakdown)
        ss->w0[tid] = v;
    }
    __syncthreads();
    if (a.op == kBgsUpdDot && tid < ng) {
        int i = 0, q = tid;  // pair tid = (i, j), packed row by row
        while (q >= sb - i) {
            q -= sb - i;
            ++i;
        }
        const int j = i + q;
        double v = ss->red[kc * sb + tid];
        for (int c = 0; c < kc; ++c) v -= s_c2[i][c] * s_c2[j][c];
        if (!isfinite(v)) s_bad = 1;
        s_g[tid] = v;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            // a non-finite sum: the solve ends with the error
            st->error |= kErrNonfinite;
            st->stop = 1;
            st->cycle_done = 1;
            st->k = 0;
            publish_progress(st, 1, st->j);
        }
    } else if (a.op == kBgsUpdDot) {
        double *sh = reinterpret_cast<double *>(smem_raw);
        const size_t sh_bytes = (size_t)(kSColsMax + kSColsMax * kSColsMax) * sizeof(double);
        cta_finish_block(a, st, ss, s_g, sh, sh_bytes);
    }
    if (tid == 0) ss->ticket[a.op] = 0;
}

// Stages of a pass CTA fill this much dynamic shared memory (two CTAs of 16 warps fit one SM where their
// registers do); a single stage may be larger: up to (64 + 8) columns of 256 float64 rows, 144 KB,
// within the attribute kBgsSmemAttr every pass kernel is given.
constexpr size_t kBgsSmemMax = 110 * 1024;
constexpr size_t kBgsSmemAttr = (size_t)(kSColsMax + kSMax) * kTR * sizeof(double);

// shared memory of one stage, and the stage count: as many as the budget holds, 1 .. kMaxStages
template <typename T>
void bgs_stages(int ncol, size_t *smem, int *nst)
{
    const size_t one = (size_t)ncol * kTR * sizeof(T);
    int q = (int)(kBgsSmemMax / one);
    *nst = q < 1 ? 1 : (q > kMaxStages ? kMaxStages : q);
    *smem = one * (size_t)*nst;
}

// Launches a pass kernel on as many CTAs as can be resident at once (cached per kernel and shared-
// memory size), at most one per tile and at most the caller's slot count (a.nblk on entry).
template <typename T, typename... KArgs>
cudaError_t go_pass(void (*kernel)(KArgs...), int key, BgsArgs &a, Cycle *st, SStep *ss, size_t smem, int nst,
                    int num_sms, cudaStream_t s)
{
    static bool attr[4 * kSMax] = {};
    static int per[4 * kSMax][kMaxStages * (kSColsMax + kSMax) + 1] = {};
    if (!attr[key]) {
        const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBgsSmemAttr);
        if (e != cudaSuccess) return e;
        attr[key] = true;
    }
    int &p = per[key][smem / (kTR * sizeof(T))];
    if (p == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, kernel, kBT, smem) != cudaSuccess || p < 1)) {
        cudaGetLastError();
        p = 1;
    }
    long long g = (long long)p * num_sms;
    if (g > a.nblk) g = a.nblk;
    if (g > a.ntiles) g = a.ntiles;
    a.nblk = (int)(g > 0 ? g : 1);
    return launch_pdl(kernel, dim3(a.nblk), dim3(kBT), smem, s, a, st, ss, nst);
}

template <typename T, int SB>
cudaError_t launch_pass_sb(BgsArgs &a, Cycle *st, SStep *ss, size_t smem, int nst, int num_sms, cudaStream_t s)
{
    const int kc = a.k + 1;
    const int key = 4 * (SB - 1);
    if (a.op == kBgsUpdTri) return go_pass<T>(k_bgs_tri<T, SB>, key, a, st, ss, smem, nst, num_sms, s);
    if (kc <= 16) return go_pass<T>(k_bgs_dot<T, 16, SB>, key + 1, a, st, ss, smem, nst, num_sms, s);
    if (kc <= 32) return go_pass<T>(k_bgs_dot<T, 32, SB>, key + 2, a, st, ss, smem, nst, num_sms, s);
    return go_pass<T>(k_bgs_dot<T, 64, SB>, key + 3, a, st, ss, smem, nst, num_sms, s);
}

template <typename T>
cudaError_t launch_bgs_t(BgsArgs a, Cycle *st, SStep *ss, int num_sms, cudaStream_t s)
{
    const int kc = a.k + 1;
    size_t smem;
    int nst;
    bgs_stages<T>(kc + a.sb, &smem, &nst);
    cudaError_t e;
    switch (a.sb) {
    case 1: e = launch_pass_sb<T, 1>(a, st, ss, smem, nst, num_sms, s); break;
    case 2: e = launch_pass_sb<T, 2>(a, st, ss, smem, nst, num_sms, s); break;
    case 3: e = launch_pass_sb<T, 3>(a, st, ss, smem, nst, num_sms, s); break;
    case 4: e = launch_pass_sb<T, 4>(a, st, ss, smem, nst, num_sms, s); break;
    case 5: e = launch_pass_sb<T, 5>(a, st, ss, smem, nst, num_sms, s); break;
    case 6: e = launch_pass_sb<T, 6>(a, st, ss, smem, nst, num_sms, s); break;
    case 7: e = launch_pass_sb<T, 7>(a, st, ss, smem, nst, num_sms, s); break;
    default: e = launch_pass_sb<T, 8>(a, st, ss, smem, nst, num_sms, s); break;
    }
    if (e != cudaSuccess || a.op == kBgsUpdTri) return e;
    static bool attr = false;
    const size_t fsm = (size_t)(kSColsMax + kSColsMax * kSColsMax) * sizeof(double);
    if (!attr) {
        e = cudaFuncSetAttribute(k_bgs_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nout = kc * a.sb + (a.op == kBgsDot ? a.sb : a.sb * (a.sb + 1) / 2);
    const int grid = (nout + kThreads / 32 - 1) / (kThreads / 32);
    return launch_pdl(k_bgs_finish, dim3(grid), dim3(kThreads), fsm, s, a, st, ss);
}

}  // namespace

int bgs_max_blocks(int num_sms) { return 3 * num_sms; }

cudaError_t launch_sstep_flex_y(Cycle *st, SStep *ss, int skip_if_stop, cudaStream_t s)
{
    return launch_pdl(k_sstep_flex_y, dim3(1), dim3(kSColsMax), 0, s, st, ss, skip_if_stop);
}

cudaError_t launch_bgs(int prec, BgsArgs a, Cycle *st, SStep *ss, int num_sms, cudaStream_t s)
{
    if (a.k < 0 || a.k + 1 > kSColsMax || a.sb < 1 || a.sb > kSMax || a.op < kBgsDot || a.op > kBgsUpdTri ||
        a.nblk < 1 || a.nblk > bgs_max_blocks(num_sms) || (a.pld & 1) || a.pld < a.nblk)
        return cudaErrorInvalidValue;
    a.ntiles = ((long long)a.n + kTR - 1) / kTR;
    return prec == kF64 ? launch_bgs_t<double>(a, st, ss, num_sms, s) : launch_bgs_t<float>(a, st, ss, num_sms, s);
}

}  // namespace ppg
