// ppg_batch.cu -- many independent PP-GMRES solves in one persistent launch.
//
// Each system is owned by one thread-block cluster; the cluster's CTAs split the rows.
// Everything of the method runs inside the cluster: the minimum-residual polynomial of
// the system (a (d+1)-step float64 Arnoldi run from a SplitMix64 start vector, harmonic
// Ritz values, Leja order -- Loe, Thornquist, Boman, Sections II and V), then float32
// PP-GMRES(m) cycles with two-pass classical Gram-Schmidt (Section III), each cycle ending
// with a float64 residual and update of x (iterative refinement), until the relative
// residual meets the tolerance.
//
// Synchronisation is the hardware cluster barrier: one after every SpMV whose output is
// gathered next, one inside every reduction.  Reductions go through distributed shared
// memory: each CTA publishes its partial sums, and after the barrier every CTA adds all
// CTAs' partials in rank order, so every CTA holds identical values and runs the small
// dense steps (Givens rotations, the roots of the polynomial) itself -- no broadcast and no
// software spin-wait.  Clusters are scheduled largest system first; the hardware starts a
// new cluster whenever one finishes, which balances the uneven sizes.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "ppg_dense.cuh"
#include "ppg_internal.h"

namespace cg = cooperative_groups;

namespace ppg {

#ifndef PPG_BATCH_DOT_RU
#define PPG_BATCH_DOT_RU 2  // rows per sweep of the float32 block inner products
#endif
#ifndef PPG_BATCH_MIN_BLOCKS
#define PPG_BATCH_MIN_BLOCKS 4  // CTAs per SM the register allocation is sized for
#endif
#ifndef PPG_BATCH_SPMV_U
#define PPG_BATCH_SPMV_U 4  // rows a thread group of the batched SpMV walks together
#endif
#ifndef PPG_BATCH_SPMV_E
#define PPG_BATCH_SPMV_E 2  // entries of each of those rows whose loads are issued together (float32 values)
#endif

constexpr int kBMaxM = 40;      // restart length
constexpr int kBMaxRoots = 32;  // degree + 1
constexpr int kBChunk = 16;     // columns reduced per sweep
constexpr int kBMaxWarps = 16;  // warps of the widest CTA (512 threads)
constexpr int kBLdH = kBMaxRoots + 1;

struct BShared {
    union {
        struct {
            double H[kBLdH * kBMaxRoots];
            double work[kBMaxRoots * kBMaxRoots + kBMaxRoots];
            double wr[kBMaxRoots], wi[kBMaxRoots], score[kBMaxRoots];
            int order[kBMaxRoots], used[kBMaxRoots];
        } c;                                    // construction
        double R[(kBMaxM + 1) * kBMaxM];        // rotated Hessenberg of a GMRES cycle
    } u;
    double sigma[kBMaxM + 2];
    double h1[kBMaxM + 2], h2[kBMaxM + 2], coef[kBMaxM + 2];
    float fcoef[kBMaxM + 2];  // coef in float32 for the float32 basis updates
    double cs[kBMaxM], sn[kBMaxM], g[kBMaxM + 2], y[kBMaxM + 1];
    double part[2][kBMaxM + 2];
    double red[kBMaxM + 2];
    double scratch[kBChunk * kBMaxWarps];
    double roots[2 * kBMaxRoots], table[2 * kBMaxRoots];
    double beta, bnorm, w0sq, est, relres;
    int nroots, status, done, brk, kcols;
    long long iters, cycles, spmvs, breakdowns;
};

__device__ __forceinline__ void csync(cg::cluster_group &cl) { cl.sync(); }

// Cluster sum of this CTA's s.part[buf][0..cnt): afterwards s.red[0..cnt) holds the sum over the
// cluster's CTAs in rank order (identical in every CTA).
__device__ void cluster_reduce(cg::cluster_group &cl, BShared &s, int cnt, int &buf)
{
    csync(cl);
    const int nr = (int)cl.num_blocks();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        double tot = 0.0;
        for (int r = 0; r < nr; ++r) tot += *cl.map_shared_rank(&s.part[buf][t], r);
        s.red[t] = tot;
    }
    __syncthreads();
    buf ^= 1;
}

// s.part[buf][c] = this CTA's rows of V_c . v (c < k); with norm, s.part[buf][k] = this CTA's ||v||^2.
template <typename T>
__device__ void cta_dots(BShared &s, int buf, const T *V, long long ld, int k, const T *v, int r0, int r1, bool norm)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, bd = blockDim.x;
    // float32: a thread takes two of its rows per sweep (the same rows in the same order as one at a
    // time, so the sums are unchanged) to keep twice the loads in flight
    constexpr int RU = sizeof(T) == 4 ? PPG_BATCH_DOT_RU : 1;
    for (int c0 = 0; c0 < k; c0 += kBChunk) {
        const int cn = min(kBChunk, k - c0);
        T acc[kBChunk];
#pragma unroll
        for (int q = 0; q < kBChunk; ++q) acc[q] = T(0);
        for (int r = r0 + tid; r < r1; r += RU * bd) {
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int ru = r + u * bd;
                if (u == 0 || ru < r1) {
                    const T vr = v[ru];
#pragma unroll
                    for (int q = 0; q < kBChunk; ++q)
                        if (q < cn) acc[q] = fma(V[(long long)(c0 + q) * ld + ru], vr, acc[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kBChunk; ++q) {
            if (q < cn) {
                const double t = warp_sum((double)acc[q]);
                if (lane == 0) s.scratch[q * kBMaxWarps + wid] = t;
            }
        }
        __syncthreads();
        if (tid < cn) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s.scratch[tid * kBMaxWarps + q];
            s.part[buf][c0 + tid] = t;
        }
        __syncthreads();
    }
    if (norm) {
        double a = 0.0;
        for (int r = r0 + tid; r < r1; r += blockDim.x) a = fma((double)v[r], (double)v[r], a);
        a = warp_sum(a);
        if (lane == 0) s.scratch[wid] = a;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s.scratch[q];
            s.part[buf][k] = t;
        }
        __syncthreads();
    }
}

// out[r] = w[r] - sum_{c<k} V_c[r] coef[c] on this CTA's rows (w may be null: 0)
template <typename T>
__device__ void cta_update(const T *coef, const T *V, long long ld, int k, const T *w, T *out, int r0, int r1)
{
    // four rows per thread and sweep: their column loads are in flight together (each row's sum runs
    // over the columns in the same order as before)
    constexpr int RU = 4;
    const int bd = blockDim.x;
    for (int base = r0 + threadIdx.x; base < r1; base += RU * bd) {
        T acc[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int r = base + u * bd;
            acc[u] = (w && r < r1) ? w[r] : T(0);
        }
#pragma unroll 4
        for (int c = 0; c < k; ++c) {
            const T cc = -coef[c];
            const T *Vc = V + (long long)c * ld;
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int r = base + u * bd;
                if (r < r1) acc[u] = fma(cc, Vc[r], acc[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int r = base + u * bd;
            if (r < r1) out[r] = acc[u];
        }
    }
}

// One fused SpMV step on this CTA's rows: with Ax = (A (x + s2 x2))[r],
//   o0[r] = a0 Ax + b0 u0[r] + c0 w0[r];   o1[r] = a1 Ax + b1 u1[r] + c1 w1[r]  (null terms dropped)
// G threads per row: lane g of a row's group takes entries g, g + G, ... and the group sums by a
// shuffle tree (rows of a few entries: G = 1; G > 1 keeps all threads busy on systems with fewer
// rows per CTA than threads).  The loop's trip count is the same for every thread of the CTA.
template <int G, typename T, typename TV>
__device__ void cta_spmv_g(const int *rowptr, const int *colidx, const TV *vals, int r0, int r1, const T *x,
                           const T *x2, T s2, T *o0, T a0, const T *u0, T b0, const T *w0, T c0, T *o1, T a1,
                           const T *u1, T b1, const T *w1, T c1)
{
    // each group takes U rows per sweep and walks their entries E at a time: the U x E index/value
    // loads are issued together, then the U x E gathers, so that a sweep waits on two loads in a row
    // per E entries instead of two per entry (the rows are short: latency, not arithmetic, is what a
    // small CTA group waits on).  Each row's entries are still summed in their order.
    constexpr int U = PPG_BATCH_SPMV_U;
    constexpr int E = sizeof(TV) == 4 ? PPG_BATCH_SPMV_E : (PPG_BATCH_SPMV_E > 2 ? PPG_BATCH_SPMV_E / 2 : 1);
    const int per = blockDim.x / G, grp = threadIdx.x / G, g = threadIdx.x % G;
    for (int base = r0; base < r1; base += per * U) {
        int ks[U], ke[U];
        T acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = base + grp + u * per;
            ks[u] = r < r1 ? rowptr[r] + g : 0;
            ke[u] = r < r1 ? rowptr[r + 1] : 0;
            acc[u] = T(0);
        }
        for (int t = 0;; t += G * E) {
            int qi[U][E];
            TV av[U][E];
            bool any = false;
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int k = ks[u] + t + e * G;
                    qi[u][e] = -1;
                    av[u][e] = TV(0);
                    if (k < ke[u]) {
                        qi[u][e] = colidx[k];
                        av[u][e] = vals[k];
                        any = true;
                    }
                }
            if (!any) break;
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int q = qi[u][e];
                    if (q >= 0) {
                        const T xv = x2 ? fma(s2, x2[q], x[q]) : x[q];
                        acc[u] = fma((T)av[u][e], xv, acc[u]);
                    }
                }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int o = G >> 1; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = base + grp + u * per;
            if (r < r1 && g == 0) {
                T v = a0 * acc[u];
                if (u0) v = fma(b0, u0[r], v);
                if (w0) v = fma(c0, w0[r], v);
                o0[r] = v;
                if (o1) {
                    T v1 = a1 * acc[u];
                    if (u1) v1 = fma(b1, u1[r], v1);
                    if (w1) v1 = fma(c1, w1[r], v1);
                    o1[r] = v1;
                }
            }
        }
    }
    // rows are written by other threads than the ones the row-strided loops that follow (dots,
    // updates) give them to
    __syncthreads();
}

template <typename T, typename TV>
__device__ void cta_spmv(int G, const int *rowptr, const int *colidx, const TV *vals, int r0, int r1, const T *x,
                         const T *x2, T s2, T *o0, T a0, const T *u0, T b0, const T *w0, T c0, T *o1, T a1,
                         const T *u1, T b1, const T *w1 = nullptr, T c1 = T(0))
{
    switch (G) {
    case 2:
        cta_spmv_g<2>(rowptr, colidx, vals, r0, r1, x, x2, s2, o0, a0, u0, b0, w0, c0, o1, a1, u1, b1, w1, c1);
        break;
    case 4:
        cta_spmv_g<4>(rowptr, colidx, vals, r0, r1, x, x2, s2, o0, a0, u0, b0, w0, c0, o1, a1, u1, b1, w1, c1);
        break;
    case 8:
        cta_spmv_g<8>(rowptr, colidx, vals, r0, r1, x, x2, s2, o0, a0, u0, b0, w0, c0, o1, a1, u1, b1, w1, c1);
        break;
    default:
        cta_spmv_g<1>(rowptr, colidx, vals, r0, r1, x, x2, s2, o0, a0, u0, b0, w0, c0, o1, a1, u1, b1, w1, c1);
    }
}

// dst = p(src * scale) in product form over the roots in s (float32 vectors).  With defer, a
// final real root is not applied: *dP and *dt receive P and its coefficient so that the caller
// folds it into the SpMV that gathers dst.  Returns the SpMVs done.  buf: P0, P1, T.
__device__ int cluster_poly(cg::cluster_group &cl, const BShared &s, const BatchSys &S, int r0, int r1,
                            const float *src, float scale, float *dst, float *P0, float *P1, float *Tv, bool defer,
                            const float **dP, float *dt)
{
    const int k = s.nroots;
    const float *P = src;
    float sP = scale;  // P_true = sP * P
    bool first = true;
    int pp = 0, spmvs = 0;
    bool tail_write = false;  // the last step wrote dst on this CTA's rows only, without a barrier
    if (defer) *dP = nullptr;
    for (int i = 0; i < k;) {
        const bool real = s.roots[2 * i + 1] == 0.0;
        if (real) {
            const float t = (float)s.table[2 * i];
            if (i == k - 1) {
                if (defer && !first) {
                    *dP = P;
                    *dt = t * sP;
                } else {
                    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x)
                        dst[r] = (first ? 0.f : dst[r]) + t * sP * P[r];
                    tail_write = true;
                }
            } else {
                float *Pn = pp ? P1 : P0;
                cta_spmv<float, float>(S.lanes, S.rowptr, S.colidx, S.vals32, r0, r1, P, nullptr, 0.f, dst, 0.f, P, t * sP,
                                       first ? nullptr : dst, 1.f, Pn, -t * sP, P, sP);
                csync(cl);
                ++spmvs;
                P = Pn;
                sP = 1.f;
                pp ^= 1;
            }
            i += 1;
        } else {
            const float c2a = (float)s.table[2 * i], cq = (float)s.table[2 * i + 1];
            const bool last = (i + 2 >= k);
            cta_spmv<float, float>(S.lanes, S.rowptr, S.colidx, S.vals32, r0, r1, P, nullptr, 0.f, dst, -cq * sP, P, c2a * sP,
                                   first ? nullptr : dst, 1.f, Tv, sP, nullptr, 0.f);
            csync(cl);
            ++spmvs;
            if (!last) {
                float *Pn = pp ? P1 : P0;
                cta_spmv<float, float>(S.lanes, S.rowptr, S.colidx, S.vals32, r0, r1, Tv, nullptr, 0.f, Pn, cq, Tv, -c2a, P,
                                       sP, nullptr, 0.f, nullptr, 0.f);
                csync(cl);
                ++spmvs;
                P = Pn;
                sP = 1.f;
                pp ^= 1;
            }
            i += 2;
        }
        first = false;
    }
    if (tail_write && defer) csync(cl);  // dst is gathered next
    return spmvs;
}

// r = b - A x in float64 on this CTA's rows (rows as the rest of the kernel strides them)
__device__ void cta_residual(const BatchSys &S, double *r_out, int r0, int r1)
{
    cta_spmv<double, double>(S.lanes, S.rowptr, S.colidx, S.vals64, r0, r1, S.x, nullptr, 0.0, r_out, -1.0, S.b, 1.0,
                             nullptr, 0.0, nullptr, 0.0, nullptr, 0.0);
}

// ||r|| over the cluster and the tests of a true residual (Section III): converged, iteration limit,
// non-finite.  Leaves beta, relres, done, status in s.
__device__ void batch_residual_norm(cg::cluster_group &cl, BShared &s, int &buf, const double *r, int r0, int r1,
                                    const BatchParams &p)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double a = 0.0;
    for (int q = r0 + tid; q < r1; q += blockDim.x) a = fma(r[q], r[q], a);
    a = warp_sum(a);
    if (lane == 0) s.scratch[wid] = a;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s.scratch[q];
        s.part[buf][0] = t;
    }
    __syncthreads();
    cluster_reduce(cl, s, 1, buf);
    if (tid == 0) {
        s.beta = sqrt(s.red[0]);
        s.relres = s.bnorm > 0.0 ? s.beta / s.bnorm : 0.0;
        s.spmvs += 1;
        s.done = 0;
        if (!isfinite(s.beta)) s.status = 2;
        else if (s.relres <= p.tol || s.bnorm == 0.0) s.done = 1;
        else if (s.iters >= p.maxit) s.done = 2;
    }
    __syncthreads();
}

// s.part[buf][c] = this CTA's rows of V_c . r (c < k), float32 V and float64 r, summed in float64
__device__ void cta_dots_mixed(BShared &s, int buf, const float *V, long long ld, int k, const double *r, int r0,
                               int r1)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int c0 = 0; c0 < k; c0 += kBChunk) {
        const int cn = min(kBChunk, k - c0);
        double acc[kBChunk];
#pragma unroll
        for (int q = 0; q < kBChunk; ++q) acc[q] = 0.0;
        for (int q0 = r0 + tid; q0 < r1; q0 += blockDim.x) {
            const double vr = r[q0];
#pragma unroll
            for (int q = 0; q < kBChunk; ++q)
                if (q < cn) acc[q] = fma((double)V[(long long)(c0 + q) * ld + q0], vr, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < kBChunk; ++q) {
            if (q < cn) {
                const double t = warp_sum(acc[q]);
                if (lane == 0) s.scratch[q * kBMaxWarps + wid] = t;
            }
        }
        __syncthreads();
        if (tid < cn) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s.scratch[tid * kBMaxWarps + q];
            s.part[buf][c0 + tid] = t;
        }
        __syncthreads();
    }
}

// y = R^{-1} g (k columns of the cycle's rotated Hessenberg matrix), by one thread
__device__ void back_substitute(BShared &s, int k)
{
    for (int i = k - 1; i >= 0; --i) {
        double v = s.g[i];
        for (int q = i + 1; q < k; ++q) v -= s.u.R[i + q * (kBMaxM + 1)] * s.y[q];
        s.y[i] = v / s.u.R[i + i * (kBMaxM + 1)];
    }
}

// x += sum_{c<k} y_c Z_c on this CTA's rows (float32 Z, float64 x and y, float64 sums)
__device__ void cta_xupdate_z(const float *Z, long long ld, int k, const double *y, double *x, int r0, int r1)
{
    constexpr int RU = 4;  // rows per thread and sweep, as in cta_update
    const int bd = blockDim.x;
    for (int base = r0 + threadIdx.x; base < r1; base += RU * bd) {
        double acc[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) acc[u] = 0.0;
#pragma unroll 2
        for (int c = 0; c < k; ++c) {
            const float *Zc = Z + (long long)c * ld;
            const double yc = y[c];
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int r = base + u * bd;
                if (r < r1) acc[u] = fma((double)Zc[r], yc, acc[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int r = base + u * bd;
            if (r < r1) x[r] += acc[u];
        }
    }
}

__device__ __forceinline__ unsigned long long bmix(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// NT threads per CTA: 256, or 512 for large systems (more warps per system to hide the latency of
// its loops; half as many CTAs per SM)
template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? PPG_BATCH_MIN_BLOCKS : 2)
    k_batch(const BatchSys *__restrict__ sys, const int *__restrict__ order, BatchParams p, BatchOut *out)
{
    __shared__ BShared s;
    cg::cluster_group cl = cg::this_cluster();
    const int nr = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int si = order[blockIdx.x / nr];
    const BatchSys S = sys[si];
    const int n = S.n;
    const int chunk = (n + nr - 1) / nr;
    const int r0 = min(n, rank * chunk), r1 = min(n, r0 + chunk);
    const int tid = threadIdx.x;
    int buf = 0;
    const long long t_start = (long long)global_timer_ns();
    if (tid == 0) {
        s.status = 0;
        s.iters = s.cycles = s.spmvs = s.breakdowns = 0;
        s.relres = 1.0;
        s.est = 1.0;
    }
    __syncthreads();

    // ---------------- 1. the polynomial: (d+1)-step float64 Arnoldi from v0
    const long long ld = n;
    double *V64 = S.V64, *w64 = S.dw;
    {
        const unsigned long long base = bmix(p.seed + (unsigned long long)si);
        for (int r = r0 + tid; r < r1; r += blockDim.x) {
            const unsigned long long z = bmix(base + (unsigned long long)(r + 1) * 0x9E3779B97F4A7C15ull);
            V64[r] = -1.0 + 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0));
        }
        cta_dots<double>(s, buf, V64, ld, 0, V64, r0, r1, true);
        cluster_reduce(cl, s, 1, buf);
        if (tid == 0) {
            s.beta = sqrt(s.red[0]);
            s.sigma[0] = 1.0 / s.beta;
            for (int q = 0; q < kBLdH * kBMaxRoots; ++q) s.u.c.H[q] = 0.0;
        }
        __syncthreads();
        const int steps = p.degree + 1;
        int done = 0;
        for (int j = 0; j < steps; ++j) {
            cta_spmv<double, double>(S.lanes, S.rowptr, S.colidx, S.vals64, r0, r1, V64 + j * ld, nullptr, 0.0, w64,
                                     s.sigma[j], nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0);
            cta_dots<double>(s, buf, V64, ld, j + 1, w64, r0, r1, true);
            cluster_reduce(cl, s, j + 2, buf);
            if (tid == 0) {
                for (int c = 0; c <= j; ++c) {
                    s.h1[c] = s.sigma[c] * s.red[c];
                    s.coef[c] = s.h1[c] * s.sigma[c];
                }
                s.w0sq = s.red[j + 1];
            }
            __syncthreads();
            cta_update<double>(s.coef, V64, ld, j + 1, w64, w64, r0, r1);
            cta_dots<double>(s, buf, V64, ld, j + 1, w64, r0, r1, false);
            cluster_reduce(cl, s, j + 1, buf);
            if (tid == 0)
                for (int c = 0; c <= j; ++c) {
                    s.h2[c] = s.sigma[c] * s.red[c];
                    s.coef[c] = s.h2[c] * s.sigma[c];
                }
            __syncthreads();
            cta_update<double>(s.coef, V64, ld, j + 1, w64, V64 + (j + 1) * ld, r0, r1);
            cta_dots<double>(s, buf, V64 + (j + 1) * ld, ld, 0, V64 + (j + 1) * ld, r0, r1, true);
            cluster_reduce(cl, s, 1, buf);
            if (tid == 0) {
                const double nrm = sqrt(s.red[0]);
                for (int c = 0; c <= j; ++c) s.u.c.H[c + j * kBLdH] = s.h1[c] + s.h2[c];
                s.u.c.H[j + 1 + j * kBLdH] = nrm;
                s.brk = !(nrm > 1e-14 * sqrt(s.w0sq));
                s.sigma[j + 1] = s.brk ? 0.0 : 1.0 / nrm;
                if (!isfinite(nrm)) s.status = 2;
            }
            __syncthreads();
            done = j + 1;
            if (s.brk || s.status) break;
        }
        // roots of 1 - z p(z): harmonic Ritz values (warp 0), Leja order, per-step coefficients
        if (s.status == 0) {
            if (tid < 32) {
                int st = harmonic_ritz(done, s.u.c.H, kBLdH, s.u.c.wr, s.u.c.wi, s.u.c.work, tid, 32);
                if (st == 0) leja_order(done, s.u.c.wr, s.u.c.wi, s.u.c.order, s.u.c.used, s.u.c.score, tid, 32);
                __syncwarp();
                if (tid == 0) {
                    if (st) s.status = 3;
                    for (int q = 0; q < done && !st; ++q) {
                        const double re = s.u.c.wr[s.u.c.order[q]], im = s.u.c.wi[s.u.c.order[q]];
                        s.roots[2 * q] = re;
                        s.roots[2 * q + 1] = im;
                        if (!isfinite(re) || !isfinite(im) || (re == 0.0 && im == 0.0)) s.status = 3;
                        if (im == 0.0) {
                            s.table[2 * q] = 1.0 / re;
                            s.table[2 * q + 1] = 0.0;
                        } else if (im > 0.0) {
                            const double qq = re * re + im * im;
                            s.table[2 * q] = 2.0 * re / qq;
                            s.table[2 * q + 1] = 1.0 / qq;
                        } else {
                            s.table[2 * q] = s.table[2 * q + 1] = 0.0;
                        }
                    }
                    s.nroots = done;
                }
            }
            __syncthreads();
        }
        if (tid == 0) s.spmvs += done;
    }

    // ---------------- 2. float32 PP-GMRES cycles with float64 refinement
    float *V = S.V;
    float *fw = S.fw;
    float *w = fw, *P0 = fw + ld, *P1 = fw + 2 * ld, *Tv = fw + 3 * ld, *Y = fw + 4 * ld, *z = fw + 5 * ld;
    {
        double a = 0.0;
        for (int r = r0 + tid; r < r1; r += blockDim.x) a = fma(S.b[r], S.b[r], a);
        a = warp_sum(a);
        if ((tid & 31) == 0) s.scratch[tid >> 5] = a;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s.scratch[q];
            s.part[buf][0] = t;
        }
        __syncthreads();
        cluster_reduce(cl, s, 1, buf);
        if (tid == 0) s.bnorm = sqrt(s.red[0]);
        __syncthreads();
        if (s.bnorm == 0.0)  // b = 0: the solution is x = 0
            for (int r = r0 + tid; r < r1; r += blockDim.x) S.x[r] = 0.0;
    }
    const int m = p.m;
    int kprev = 0;  // columns of the previous cycle (flexible form: the restart projection uses them)
    while (s.status == 0) {
        // true residual r = b - A x in float64
        csync(cl);  // x complete
        cta_residual(S, w64, r0, r1);
        batch_residual_norm(cl, s, buf, w64, r0, r1, p);
        if (s.status || s.done) break;
        if (p.flexible && kprev > 0) {
            // restart projection: y = argmin ||H y - V^T r|| over the previous cycle's space (its
            // rotations and R are still in shared memory), x += Z y, and the residual again
            cta_dots_mixed(s, buf, V, ld, kprev + 1, w64, r0, r1);
            cluster_reduce(cl, s, kprev + 1, buf);
            if (tid == 0) {
                double a = s.sigma[0] * s.red[0];
                for (int i = 0; i < kprev; ++i) {
                    const double bb = s.sigma[i + 1] * s.red[i + 1];
                    s.g[i] = s.cs[i] * a + s.sn[i] * bb;
                    a = -s.sn[i] * a + s.cs[i] * bb;
                }
                back_substitute(s, kprev);
            }
            __syncthreads();
            cta_xupdate_z(S.Z, ld, kprev, s.y, S.x, r0, r1);
            csync(cl);  // x complete
            cta_residual(S, w64, r0, r1);
            batch_residual_norm(cl, s, buf, w64, r0, r1, p);
            if (s.status || s.done) break;
        }
        // start the cycle from r: basis column 0
        for (int r = r0 + tid; r < r1; r += blockDim.x) V[r] = (float)w64[r];
        if (tid == 0) {
            s.cycles += 1;
            s.sigma[0] = 1.0 / s.beta;
            for (int q = 0; q <= m; ++q) s.g[q] = 0.0;
            s.g[0] = s.beta;
        }
        csync(cl);  // column 0 is gathered next
        int kc = 0;
        for (int j = 0; j < m; ++j) {
            // w = A p(A) v_j  (v_j = sigma_j U_j); flexible form: the SpMV also writes z_j = p(A) v_j,
            // the value its own gather forms, to Z_j
            const float *dP = nullptr;
            float dt = 0.f;
            int sp = cluster_poly(cl, s, S, r0, r1, V + j * ld, (float)s.sigma[j], Y, P0, P1, Tv, true, &dP, &dt);
            if (p.flexible)
                cta_spmv<float, float>(S.lanes, S.rowptr, S.colidx, S.vals32, r0, r1, Y, dP, dt, w, 1.f, nullptr, 0.f,
                                       nullptr, 0.f, S.Z + j * ld, 0.f, Y, 1.f, dP, dt);
            else
                cta_spmv<float, float>(S.lanes, S.rowptr, S.colidx, S.vals32, r0, r1, Y, dP, dt, w, 1.f, nullptr, 0.f,
                                       nullptr, 0.f, nullptr, 0.f, nullptr, 0.f);
            // pass 1
            cta_dots<float>(s, buf, V, ld, j + 1, w, r0, r1, true);
            cluster_reduce(cl, s, j + 2, buf);
            if (tid == 0) {
                for (int c = 0; c <= j; ++c) {
                    s.h1[c] = s.sigma[c] * s.red[c];
                    s.coef[c] = s.h1[c] * s.sigma[c];
                    s.fcoef[c] = (float)s.coef[c];
                }
                s.w0sq = s.red[j + 1];
                s.spmvs += sp + 1;
            }
            __syncthreads();
            // pass 2
            cta_update<float>(s.fcoef, V, ld, j + 1, w, w, r0, r1);
            // (with ||w'||^2, so that pass 3 needs no reduction: ||v_{j+1}||^2 = ||w'||^2 - ||h2||^2)
            cta_dots<float>(s, buf, V, ld, j + 1, w, r0, r1, true);
            cluster_reduce(cl, s, j + 2, buf);
            if (tid == 0) {
                double h2sq = 0.0;
                for (int c = 0; c <= j; ++c) {
                    s.h2[c] = s.sigma[c] * s.red[c];
                    h2sq = fma(s.h2[c], s.h2[c], h2sq);
                    s.coef[c] = s.h2[c] * s.sigma[c];
                    s.fcoef[c] = (float)s.coef[c];
                }
                const double wpsq = s.red[j + 1], nsq = wpsq - h2sq;
                // breakdown also when the second pass removed more than 99 % of ||w'||^2 (the difference
                // of squares is no longer accurate there): the cycle ends and the restart carries on
                const bool brk = !(nsq > 1e-28 * s.w0sq) || !(nsq > 1e-2 * wpsq);
                const double nrm = !isfinite(nsq) ? nsq : (brk ? 0.0 : sqrt(nsq));
                double *Rj = s.u.R + j * (kBMaxM + 1);
                bool fin = isfinite(nrm);
                for (int c = 0; c <= j; ++c) {
                    Rj[c] = s.h1[c] + s.h2[c];
                    fin = fin && isfinite(Rj[c]);
                }
                Rj[j + 1] = nrm;
                s.sigma[j + 1] = brk ? 0.0 : 1.0 / nrm;
                for (int c = 0; c < j; ++c) {
                    const double a = Rj[c], b = Rj[c + 1];
                    Rj[c] = s.cs[c] * a + s.sn[c] * b;
                    Rj[c + 1] = -s.sn[c] * a + s.cs[c] * b;
                }
                const double a = Rj[j], b = Rj[j + 1];
                const double rr = hypot(a, b);
                double cc = 1.0, sn = 0.0;
                if (rr != 0.0) {
                    cc = a / rr;
                    sn = b / rr;
                }
                s.cs[j] = cc;
                s.sn[j] = sn;
                Rj[j] = rr;
                Rj[j + 1] = 0.0;
                const double gj = s.g[j];
                s.g[j] = cc * gj;
                s.g[j + 1] = -sn * gj;
                const double res = fabs(s.g[j + 1]);
                s.est = res / s.bnorm;
                s.iters += 1;
                s.kcols = j + 1;
                s.brk = brk;
                if (brk) s.breakdowns += 1;
                if (!fin) s.status = 2;
                s.done = brk || !fin || res <= p.tol * s.bnorm || res <= p.inner_rtol * s.beta || j + 1 >= m ||
                         s.iters >= p.maxit;
            }
            __syncthreads();
            // pass 3: v_{j+1} = w' - V h2 (scaled by sigma_{j+1} where it is used), gathered next
            cta_update<float>(s.fcoef, V, ld, j + 1, w, V + (j + 1) * ld, r0, r1);
            csync(cl);
            kc = j + 1;
            if (s.done) break;
        }
        if (s.status) break;
        // cycle end: y = R^{-1} g; flexible: x += Z y; standard: z = V y, x += p(A) z
        if (tid == 0) {
            back_substitute(s, kc);
            for (int c = 0; c < kc; ++c) {
                s.coef[c] = -s.y[c] * s.sigma[c];
                s.fcoef[c] = (float)s.coef[c];
            }
        }
        __syncthreads();
        if (p.flexible) {
            cta_xupdate_z(S.Z, ld, kc, s.y, S.x, r0, r1);
        } else {
            cta_update<float>(s.fcoef, V, ld, kc, nullptr, z, r0, r1);
            csync(cl);
            const int sp = cluster_poly(cl, s, S, r0, r1, z, 1.f, Y, P0, P1, Tv, false, nullptr, nullptr);
            for (int r = r0 + tid; r < r1; r += blockDim.x) S.x[r] += (double)Y[r];
            if (tid == 0) s.spmvs += sp;
        }
        kprev = kc;
        __syncthreads();
    }
    if (rank == 0 && tid == 0) {
        BatchOut o;
        o.iters = s.iters;
        o.cycles = s.cycles;
        o.spmvs = s.spmvs;
        o.relres = s.relres;
        o.est = s.est;
        o.status = s.status;
        o.degree = s.nroots - 1;
        o.converged = (s.status == 0 && s.done == 1) ? 1 : 0;
        o.breakdowns = (int)s.breakdowns;
        o.t_start = t_start;
        o.t_end = (long long)global_timer_ns();
        out[si] = o;
    }
    // keep this CTA's shared memory alive until every CTA of the cluster is done reading it
    csync(cl);
}

// float32 copy of every system's values (one CTA-strided pass per system)
__global__ void k_batch_cast(const BatchSys *__restrict__ sys, int nsys, const float *const *dst_unused)
{
    (void)dst_unused;
    for (int i = blockIdx.y; i < nsys; i += gridDim.y) {
        const BatchSys S = sys[i];
        float *d = const_cast<float *>(S.vals32);
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S.nnz; k += gridDim.x * blockDim.x)
            d[k] = (float)S.vals64[k];
    }
}

cudaError_t launch_batch_cast(const BatchSys *sys_d, int nsys, cudaStream_t s)
{
    dim3 grid(64, nsys < 65535 ? nsys : 65535);
    k_batch_cast<<<grid, kThreads, 0, s>>>(sys_d, nsys, nullptr);
    return cudaGetLastError();
}

cudaError_t batch_configure()
{
    cudaError_t e = cudaFuncSetAttribute(k_batch<256>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch<512>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

// Number of clusters of `cluster` CTAs of `threads` threads that can be resident at once (0: not launchable).
int batch_max_clusters(int cluster, int threads)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(threads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    const void *fn = threads == 512 ? (const void *)k_batch<512> : (const void *)k_batch<256>;
    if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) return 0;
    return nc;
}

cudaError_t launch_batch(const BatchSys *sys_d, const int *order_d, int nsys, int cluster, const BatchParams &p,
                         BatchOut *out_d, cudaStream_t s, int threads)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nsys * cluster));
    cfg.blockDim = dim3(threads == 512 ? 512 : 256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (threads == 512) return cudaLaunchKernelEx(&cfg, k_batch<512>, sys_d, order_d, p, out_d);
    return cudaLaunchKernelEx(&cfg, k_batch<256>, sys_d, order_d, p, out_d);
}

}  // namespace ppg
