// ppg_spmv.cu -- CSR sparse matrix-vector kernels of the GB300 PP-GMRES library.
//
// The polynomial preconditioner is applied as a chain of SpMVs and vector
// updates (Loe, Thornquist, Boman, Section II, Eq. 2: p(A) = y_{d+1} A^d + ... + y_1).
// Each link of the chain is one launch of k_spmv: a row-block CSR kernel whose
// tile of non-zeros is staged in shared memory by TMA bulk copies, followed by
// a fused epilogue that forms the Horner step (w <- A w + y_j v) or a root-form
// step in the same pass, so every vector crosses HBM once per step.
#include <cuda_runtime.h>

#include "ppg_internal.h"

#include <stdlib.h>

namespace ppg {

bool pdl_enabled()
{
    static const bool on = [] {
        const char *v = getenv("PPG_NO_PDL");
        return !(v && v[0] == '1');
    }();
    return on;
}

// ---------------------------------------------------------------- validation and conversion

__global__ void k_validate(int n, long long nnz, const int *__restrict__ rowptr, const int *__restrict__ colidx,
                           int *flag)
{
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = tid; i <= n; i += stride) {
        int v = rowptr[i];
        if (i == 0 && v != 0) atomicOr(flag, 1);
        if (i == n && (long long)v != nnz) atomicOr(flag, 2);
        if (i < n && rowptr[i + 1] < v) atomicOr(flag, 4);
    }
    for (long long k = tid; k < nnz; k += stride) {
        int c = colidx[k];
        if (c < 0 || c >= n) atomicOr(flag, 8);
    }
}

cudaError_t launch_validate(int n, long long nnz, const int *rowptr, const int *colidx, int *flag, cudaStream_t s)
{
    k_validate<<<1024, kThreads, 0, s>>>(n, nnz, rowptr, colidx, flag);
    return cudaGetLastError();
}

__global__ void k_cast_f32(const double *__restrict__ in, float *__restrict__ out, long long count)
{
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += stride)
        out[i] = (float)in[i];
}

cudaError_t launch_cast_f32(const double *in, float *out, long long count, cudaStream_t s)
{
    k_cast_f32<<<2048, kThreads, 0, s>>>(in, out, count);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- the fused SpMV step

template <typename T, typename IDX>
struct SpmvArgs {
    int n;
    const int *rowptr;
    const IDX *cols;  // int32 column indices, or int16 offsets col - row
    const T *vals;
    int rows_per_tile;
    int lanes_per_row;
    int cap;  // elements of each staging array
    Cycle *st;
    int check_done;
    SpmvEpi e;
};

#ifndef PPG_SPMV_MIN_BLOCKS
#define PPG_SPMV_MIN_BLOCKS 3  // CTAs per SM the register allocation is sized for
#endif
#ifndef PPG_SPMV_CARVEOUT
#define PPG_SPMV_CARVEOUT -1  // preferred shared-memory carveout (percent; -1: the driver's choice)
#endif
#ifndef PPG_SPMV_CTAS_PER_SM
#define PPG_SPMV_CTAS_PER_SM 0  // cap on resident CTAs per SM (0: occupancy)
#endif

#ifndef PPG_SPMV_RPT
#define PPG_SPMV_RPT 1  // rows per consumer thread when rows are short (gathers of all issued together)
#endif

constexpr int kSpmvConsumerWarps = 8;
constexpr int kSpmvRpt = PPG_SPMV_RPT;
constexpr int kSpmvThreads = (kSpmvConsumerWarps + 1) * 32;  // + one producer warp
#ifndef PPG_SPMV_STAGES
#define PPG_SPMV_STAGES 3
#endif
constexpr int kSpmvStages = PPG_SPMV_STAGES;
constexpr int kSpmvRpBytes = (((256 * kSpmvRpt + 1) * 4 + 15) / 16 * 16 + 127) / 128 * 128;  // row pointers
constexpr int kSpmvCapMax = 4096;

__host__ __device__ constexpr size_t round128(size_t b) { return (b + 127) & ~(size_t)127; }

template <typename T, typename IDX>
__host__ __device__ constexpr size_t spmv_stage_bytes(int cap)
{
    return kSpmvRpBytes + round128((size_t)cap * sizeof(T)) + round128((size_t)cap * sizeof(IDX));
}

// column of entry k in row r: int32 indices as stored, int16 entries are offsets from the row
template <typename IDX>
__device__ __forceinline__ int col_of(IDX c, int r)
{
    if constexpr (sizeof(IDX) == 2)
        return r + (int)c;
    else
        return (int)c;
}

// An epilogue with its scalars and vector addresses resolved for this launch.
template <typename T>
struct EpiRes {
    const T *x, *x2;
    T *o0, *o1;
    const T *u0, *w0, *u1, *w1;
    T ca0, cb0, cc0, ca1, cb1, cc1, c2;
};

// Resolves e for the eight consumer warps (threads 0..6 evaluate the scalars into s_coef, then
// the consumers meet at named barrier 1).
template <typename T>
__device__ EpiRes<T> resolve_epi(const SpmvEpi &e, const Cycle *st, double *s_coef, int tid)
{
    switch (tid) {
    case 0: s_coef[0] = resolve(e.a0, st); break;
    case 1: s_coef[1] = resolve(e.b0, st); break;
    case 2: s_coef[2] = resolve(e.c0, st); break;
    case 3: s_coef[3] = resolve(e.a1, st); break;
    case 4: s_coef[4] = resolve(e.b1, st); break;
    case 5: s_coef[5] = resolve(e.c1, st); break;
    case 6: s_coef[6] = resolve(e.s2, st); break;
    default: break;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kSpmvConsumerWarps * 32) : "memory");
    EpiRes<T> E;
    E.x = resolve_ptr<T>(e.x, st);
    E.x2 = resolve_ptr<T>(e.x2, st);
    E.o0 = resolve_ptr<T>(e.out0, st);
    E.u0 = resolve_ptr<T>(e.u0, st);
    E.w0 = resolve_ptr<T>(e.w0, st);
    E.o1 = resolve_ptr<T>(e.out1, st);
    E.u1 = resolve_ptr<T>(e.u1, st);
    E.w1 = resolve_ptr<T>(e.w1, st);
    E.ca0 = (T)s_coef[0];
    E.cb0 = (T)s_coef[1];
    E.cc0 = (T)s_coef[2];
    E.ca1 = (T)s_coef[3];
    E.cb1 = (T)s_coef[4];
    E.cc1 = (T)s_coef[5];
    E.c2 = (T)s_coef[6];
    return E;
}

// x gathers: through the read-only path, or (data written earlier in the same launch by other
// CTAs) with plain loads; a 128-byte line of such a vector is never read before all of it has
// been written, so no stale copy can sit in this SM's L1
template <typename T, bool COH>
__device__ __forceinline__ T gather(const T *p);
template <>
__device__ __forceinline__ float gather<float, false>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ double gather<double, false>(const double *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float gather<float, true>(const float *p)
{
    float v;
    asm volatile("ld.global.ca.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
template <>
__device__ __forceinline__ double gather<double, true>(const double *p)
{
    double v;
    asm volatile("ld.global.ca.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}

// One tile of a fused SpMV step, for the calling consumer thread: rows lr + q (256 / G) of the
// tile whose row pointers, values and column indices the stage at base holds (or, for a tile
// larger than a stage, whose values and columns are read from global memory).  COH: x and x2
// were written earlier in the same launch and are gathered with coherent loads.
template <typename T, typename IDX, bool COH>
__device__ __forceinline__ void spmv_tile(const unsigned char *base, size_t val_off, size_t col_off, int cap,
                                          long long tile, int R, int G, int n, const IDX *gcols, const T *gvals,
                                          const EpiRes<T> &E, int tid)
{
    constexpr int VA = 16 / (int)sizeof(T);
    constexpr int CA = 16 / (int)sizeof(IDX);
    const int lr = tid / G;  // first row of this lane group; rows lr + q * (256 / G), q < kSpmvRpt
    const int lg = tid & (G - 1);
    constexpr int RP = kSpmvRpt;
    const int rstep = kThreads / G;
    const int *s_rp = reinterpret_cast<const int *>(base);
    const T *s_val = reinterpret_cast<const T *>(base + val_off);
    const IDX *s_col = reinterpret_cast<const IDX *>(base + col_off);
    const int r0 = (int)(tile * R);
    const int rows = min(R, n - r0);
    const int e0 = s_rp[0], e1 = s_rp[rows];
    const int vs = e0 & ~(VA - 1), ve = (e1 + VA - 1) & ~(VA - 1);
    const int cs = e0 & ~(CA - 1), ce = (e1 + CA - 1) & ~(CA - 1);
    const bool staged = (ve - vs) <= cap && (ce - cs) <= cap && e1 > e0;
    T acc[RP], pu0[RP], pw0[RP], pu1[RP], pw1[RP];
    int kb[RP], ke[RP], rr[RP];
    bool ok[RP];
#pragma unroll
    for (int q = 0; q < RP; ++q) {
        const int l = lr + q * rstep;
        ok[q] = l < rows;
        rr[q] = r0 + l;
        kb[q] = ok[q] ? s_rp[l] + lg : 0;
        ke[q] = ok[q] ? s_rp[l + 1] : 0;
        acc[q] = pu0[q] = pw0[q] = pu1[q] = pw1[q] = T(0);
        // epilogue operands first: their loads overlap the gathers below
        if (lg == 0 && ok[q]) {
            if (E.u0) pu0[q] = E.u0[rr[q]];
            if (E.w0) pw0[q] = E.w0[rr[q]];
            if (E.o1) {
                if (E.u1) pu1[q] = E.u1[rr[q]];
                if (E.w1) pw1[q] = E.w1[rr[q]];
            }
        }
    }
    if (staged) {
        // all of a lane's gathers (up to 8 per row per batch) are issued before the first FMA
        bool more = true;
        while (more) {
            int qc[RP][8];
            T xv[RP][8];
#pragma unroll
            for (int q = 0; q < RP; ++q)
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int kk = kb[q] + t * G;
                    qc[q][t] = kk < ke[q] ? col_of<IDX>(s_col[kk - cs], rr[q]) : -1;
                }
            if (E.x2 == nullptr) {
#pragma unroll
                for (int q = 0; q < RP; ++q)
#pragma unroll
                    for (int t = 0; t < 8; ++t) xv[q][t] = qc[q][t] >= 0 ? gather<T, COH>(E.x + qc[q][t]) : T(0);
            } else {
#pragma unroll
                for (int q = 0; q < RP; ++q)
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        xv[q][t] = qc[q][t] >= 0
                                       ? fma(E.c2, gather<T, COH>(E.x2 + qc[q][t]), gather<T, COH>(E.x + qc[q][t]))
                                       : T(0);
            }
            more = false;
#pragma unroll
            for (int q = 0; q < RP; ++q) {
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (qc[q][t] >= 0) acc[q] = fma(s_val[kb[q] + t * G - vs], xv[q][t], acc[q]);
                kb[q] += 8 * G;
                more = more || kb[q] < ke[q];
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < RP; ++q)
            for (int k = kb[q]; k < ke[q]; k += G) {
                const int qq = col_of<IDX>(__ldg(gcols + k), rr[q]);
                const T xv = E.x2 ? fma(E.c2, gather<T, COH>(E.x2 + qq), gather<T, COH>(E.x + qq))
                                  : gather<T, COH>(E.x + qq);
                acc[q] = fma(__ldg(gvals + k), xv, acc[q]);
            }
    }
#pragma unroll
    for (int q = 0; q < RP; ++q) {
        for (int o = G >> 1; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        if (lg == 0 && ok[q]) {
            T v = E.ca0 * acc[q];
            if (E.u0) v = fma(E.cb0, pu0[q], v);
            if (E.w0) v = fma(E.cc0, pw0[q], v);
            E.o0[rr[q]] = v;
            if (E.o1) {
                T v1 = E.ca1 * acc[q];
                if (E.u1) v1 = fma(E.cb1, pu1[q], v1);
                if (E.w1) v1 = fma(E.cc1, pw1[q], v1);
                E.o1[rr[q]] = v1;
            }
        }
    }
}

// Persistent, warp-specialised row-block CSR SpMV.  Tiles of R consecutive rows are
// dealt round-robin to the CTAs.  The producer warp keeps up to three tiles in flight:
// for each it reads the tile's non-zero range from the row pointers and issues TMA bulk
// copies of the row-pointer segment, the values and the column indices (ranges widened
// to 16-byte boundaries) into a shared-memory stage.  Eight consumer warps take the
// stages in order: G = 256/R lanes per row form the row's dot product from shared
// memory, gathering x (x + s2 x2 when a second input is given), then the row's first
// lane applies the fused epilogue and the warp releases the stage.  Tiles whose
// non-zeros exceed the stage read values and columns from global memory instead.
template <typename T, typename IDX>
__global__ void __launch_bounds__(kSpmvThreads, PPG_SPMV_MIN_BLOCKS) k_spmv(SpmvArgs<T, IDX> a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kSpmvStages];
    __shared__ __align__(8) uint64_t empty[kSpmvStages];
    __shared__ double s_coef[7];

    Cycle *st = a.st;
    const int R = a.rows_per_tile;
    const int G = a.lanes_per_row;
    const long long ntiles = ((long long)a.n + R - 1) / R;
    const size_t stage_bytes = spmv_stage_bytes<T, IDX>(a.cap);
    const size_t val_off = kSpmvRpBytes;
    const size_t col_off = kSpmvRpBytes + round128((size_t)a.cap * sizeof(T));
    constexpr int VA = 16 / (int)sizeof(T);
    constexpr int CA = 16 / (int)sizeof(IDX);
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    // tiles of this CTA whose matrix data is fetched before the predecessor kernel finishes
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int prefetched = (int)min((long long)kSpmvStages, my_tiles);

    if (tid == 0) {
        for (int s = 0; s < kSpmvStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kSpmvConsumerWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (wid == kSpmvConsumerWarps) {
        // ---------------- producer
        if (lane == 0) {
            // the next tile's non-zero range is loaded one tile ahead, so that its latency
            // overlaps the wait for a free stage
            auto bounds = [&](long long t, int &e0, int &e1) {
                const int r0 = (int)(t * R);
                e0 = __ldg(a.rowptr + r0);
                e1 = __ldg(a.rowptr + min(r0 + R, a.n));
            };
            int ne0 = 0, ne1 = 0;
            if (blockIdx.x < ntiles) bounds(blockIdx.x, ne0, ne1);
            int i = 0;
            for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
                if (i == prefetched) {
                    // the first stages hold matrix data only (constant): from here on the
                    // predecessor must be complete, and this launch may have nothing to do
                    pdl_wait();
                    pdl_trigger();
                    if ((a.check_done == kSkipIfDone && st->cycle_done) ||
                        (a.check_done == kSkipIfNoCols && st->k == 0))
                        break;
                }
                const int e0 = ne0, e1 = ne1;
                if (tile + gridDim.x < ntiles) bounds(tile + gridDim.x, ne0, ne1);
                const int s = i % kSpmvStages, round = i / kSpmvStages;
                if (round > 0 && !mbar_wait_bounded(&empty[s], (round - 1) & 1, kWaitLimitNs)) {
                    timeout_stop(st);
                    break;
                }
                const int r0 = (int)(tile * R);
                const int rows = min(R, a.n - r0);
                const int vs = e0 & ~(VA - 1), ve = (e1 + VA - 1) & ~(VA - 1);
                const int cs = e0 & ~(CA - 1), ce = (e1 + CA - 1) & ~(CA - 1);
                const bool staged = (ve - vs) <= a.cap && (ce - cs) <= a.cap && e1 > e0;
                unsigned char *base = smem + s * stage_bytes;
                const uint32_t rpb = ((uint32_t)(rows + 1) * 4u + 15u) & ~15u;
                const uint32_t vb = staged ? (uint32_t)(ve - vs) * (uint32_t)sizeof(T) : 0u;
                const uint32_t cb = staged ? (uint32_t)(ce - cs) * (uint32_t)sizeof(IDX) : 0u;
                mbar_arrive_expect_tx(&full[s], rpb + vb + cb);
                bulk_g2s(base, a.rowptr + r0, rpb, &full[s]);
                if (staged) {
                    bulk_g2s(base + val_off, a.vals + vs, vb, &full[s]);
                    bulk_g2s(base + col_off, a.cols + cs, cb, &full[s]);
                }
            }
        }
        return;
    }

    // consumers: nothing a predecessor wrote is read before this point
    pdl_wait();
    pdl_trigger();
    if ((a.check_done == kSkipIfDone && st->cycle_done) || (a.check_done == kSkipIfNoCols && st->k == 0)) {
        // nothing to do: let the prefetched matrix tiles land before the CTA exits
        for (int q = 0; q < prefetched; ++q) mbar_wait_bounded(&full[q], 0, kWaitLimitNs);
        return;
    }
    if (tid < 7) {
        switch (tid) {
        case 0: s_coef[0] = resolve(a.e.a0, st); break;
        case 1: s_coef[1] = resolve(a.e.b0, st); break;
        case 2: s_coef[2] = resolve(a.e.c0, st); break;
        case 3: s_coef[3] = resolve(a.e.a1, st); break;
        case 4: s_coef[4] = resolve(a.e.b1, st); break;
        case 5: s_coef[5] = resolve(a.e.c1, st); break;
        default: s_coef[6] = resolve(a.e.s2, st); break;
        }
    }
    // consumer-only barrier (named barrier 1, the eight consumer warps)
    asm volatile("bar.sync 1, %0;" ::"n"(kSpmvConsumerWarps * 32) : "memory");

    const T *__restrict__ x = resolve_ptr<T>(a.e.x, st);
    const T *__restrict__ x2 = resolve_ptr<T>(a.e.x2, st);
    T *o0 = resolve_ptr<T>(a.e.out0, st);
    const T *u0 = resolve_ptr<T>(a.e.u0, st);
    const T *w0 = resolve_ptr<T>(a.e.w0, st);
    T *o1 = resolve_ptr<T>(a.e.out1, st);
    const T *u1 = resolve_ptr<T>(a.e.u1, st);
    const T *w1 = resolve_ptr<T>(a.e.w1, st);
    const T ca0 = (T)s_coef[0], cb0 = (T)s_coef[1], cc0 = (T)s_coef[2];
    const T ca1 = (T)s_coef[3], cb1 = (T)s_coef[4], cc1 = (T)s_coef[5], c2 = (T)s_coef[6];
    const int lr = tid / G;  // first row of this lane group; rows lr + q * (256 / G), q < kSpmvRpt
    const int lg = tid & (G - 1);
    constexpr int RP = kSpmvRpt;
    const int rstep = kThreads / G;
    int i = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
        const int s = i % kSpmvStages;
        if (!mbar_wait_bounded(&full[s], (i / kSpmvStages) & 1, kWaitLimitNs)) {
            if (lane == 0) timeout_stop(st);
            mbar_wait_bounded(&full[s], (i / kSpmvStages) & 1, kWaitLimitNs);
            return;
        }
        const unsigned char *base = smem + s * stage_bytes;
        const int *s_rp = reinterpret_cast<const int *>(base);
        const T *s_val = reinterpret_cast<const T *>(base + val_off);
        const IDX *s_col = reinterpret_cast<const IDX *>(base + col_off);
        const int r0 = (int)(tile * R);
        const int rows = min(R, a.n - r0);
        const int e0 = s_rp[0], e1 = s_rp[rows];
        const int vs = e0 & ~(VA - 1), ve = (e1 + VA - 1) & ~(VA - 1);
        const int cs = e0 & ~(CA - 1), ce = (e1 + CA - 1) & ~(CA - 1);
        const bool staged = (ve - vs) <= a.cap && (ce - cs) <= a.cap && e1 > e0;
        T acc[RP], pu0[RP], pw0[RP], pu1[RP], pw1[RP];
        int kb[RP], ke[RP], rr[RP];
        bool ok[RP];
#pragma unroll
        for (int q = 0; q < RP; ++q) {
            const int l = lr + q * rstep;
            ok[q] = l < rows;
            rr[q] = r0 + l;
            kb[q] = ok[q] ? s_rp[l] + lg : 0;
            ke[q] = ok[q] ? s_rp[l + 1] : 0;
            acc[q] = pu0[q] = pw0[q] = pu1[q] = pw1[q] = T(0);
            // epilogue operands first: their loads overlap the gathers below
            if (lg == 0 && ok[q]) {
                if (u0) pu0[q] = u0[rr[q]];
                if (w0) pw0[q] = w0[rr[q]];
                if (o1) {
                    if (u1) pu1[q] = u1[rr[q]];
                    if (w1) pw1[q] = w1[rr[q]];
                }
            }
        }
        if (staged) {
            // all of a lane's gathers (up to 8 per row per batch) are issued before the first FMA
            bool more = true;
            while (more) {
                int qc[RP][8];
                T xv[RP][8];
#pragma unroll
                for (int q = 0; q < RP; ++q)
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int kk = kb[q] + t * G;
                        qc[q][t] = kk < ke[q] ? col_of<IDX>(s_col[kk - cs], rr[q]) : -1;
                    }
                if (x2 == nullptr) {
#pragma unroll
                    for (int q = 0; q < RP; ++q)
#pragma unroll
                        for (int t = 0; t < 8; ++t) xv[q][t] = qc[q][t] >= 0 ? __ldg(x + qc[q][t]) : T(0);
                } else {
#pragma unroll
                    for (int q = 0; q < RP; ++q)
#pragma unroll
                        for (int t = 0; t < 8; ++t)
                            xv[q][t] = qc[q][t] >= 0 ? fma(c2, __ldg(x2 + qc[q][t]), __ldg(x + qc[q][t])) : T(0);
                }
                more = false;
#pragma unroll
                for (int q = 0; q < RP; ++q) {
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        if (qc[q][t] >= 0) acc[q] = fma(s_val[kb[q] + t * G - vs], xv[q][t], acc[q]);
                    kb[q] += 8 * G;
                    more = more || kb[q] < ke[q];
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < RP; ++q)
                for (int k = kb[q]; k < ke[q]; k += G) {
                    const int qq = col_of<IDX>(__ldg(a.cols + k), rr[q]);
                    const T xv = x2 ? fma(c2, __ldg(x2 + qq), __ldg(x + qq)) : __ldg(x + qq);
                    acc[q] = fma(__ldg(a.vals + k), xv, acc[q]);
                }
        }
#pragma unroll
        for (int q = 0; q < RP; ++q) {
            for (int o = G >> 1; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            if (lg == 0 && ok[q]) {
                T v = ca0 * acc[q];
                if (u0) v = fma(cb0, pu0[q], v);
                if (w0) v = fma(cc0, pw0[q], v);
                o0[rr[q]] = v;
                if (o1) {
                    T v1 = ca1 * acc[q];
                    if (u1) v1 = fma(cb1, pu1[q], v1);
                    if (w1) v1 = fma(cc1, pw1[q], v1);
                    o1[rr[q]] = v1;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ---------------------------------------------------------------- staged x windows (float32)

// The float32 SpMV step with every operand of a tile in shared memory.  Besides the tile's row
// pointers, values and column indices, the producer copies the tile's x windows (up to kXWin
// contiguous column ranges covering every column its rows reference, precomputed per tile) and the
// tile's rows of the epilogue's row-wise operands (up to kWSlots distinct vectors), so the consumers
// gather x from shared memory instead of L1/L2 and read no global memory at all.  The matrix part of
// the first stages is requested before the wait on the predecessor (constant data), the vector parts
// after it.  Tiles without windows gather from global memory; the last, partial tile reads its row
// operands from global memory.  Arithmetic and its order are those of k_spmv.
#ifndef PPG_SPMV_STAGE_ROWS
#define PPG_SPMV_STAGE_ROWS 0  // 1: the staged kernel also stages the update operands' rows (measured slower)
#endif
constexpr int kWSlots = 3;

template <typename IDX>
struct SpmvWArgs {
    SpmvArgs<float, IDX> a;  // a.cols: the real column indices (tiles without windows)
    const short *lidx;       // window-buffer index of every entry (staged in place of the columns)
    const int *twin;
    int nslot;
    VecRef slot[kWSlots];  // distinct row-operand vectors
    int slot_of[4];        // u0, w0, u1, w1: their slot, or -1 (absent)
};

__host__ __device__ constexpr size_t spmvw_stage_bytes(int cap, int idx_bytes)
{
    return kSpmvRpBytes + round128((size_t)cap * 4) + round128((size_t)cap * 2) + round128((size_t)kXCap * 4) +
           (size_t)kWSlots * 256 * 4 + 128 + 0 * idx_bytes;
}

template <typename IDX>
__global__ void __launch_bounds__(kSpmvThreads, PPG_SPMV_MIN_BLOCKS) k_spmv_w(SpmvWArgs<IDX> p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kSpmvStages];
    __shared__ __align__(8) uint64_t empty[kSpmvStages];
    __shared__ double s_coef[7];
    using T = float;

    const SpmvArgs<float, IDX> &a = p.a;
    Cycle *st = a.st;
    const int R = a.rows_per_tile;
    const int G = a.lanes_per_row;
    const long long ntiles = ((long long)a.n + R - 1) / R;
    const size_t stage_bytes = spmvw_stage_bytes(a.cap, (int)sizeof(IDX));
    const size_t val_off = kSpmvRpBytes;
    const size_t col_off = val_off + round128((size_t)a.cap * sizeof(T));
    const size_t xw_off = col_off + round128((size_t)a.cap * 2);
    const size_t sl_off = xw_off + round128((size_t)kXCap * 4);
    const size_t hd_off = sl_off + (size_t)kWSlots * 256 * 4;
    constexpr int VA = 16 / (int)sizeof(T);
    constexpr int CA = 8;  // the staged indices are int16
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int prefetched = (int)min((long long)kSpmvStages, my_tiles);

    if (tid == 0) {
        for (int q = 0; q < kSpmvStages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kSpmvConsumerWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (wid == kSpmvConsumerWarps) {
        // ---------------- producer
        if (lane == 0) {
            auto bounds = [&](long long t, int &e0, int &e1) {
                const int r0 = (int)(t * R);
                e0 = __ldg(a.rowptr + r0);
                e1 = __ldg(a.rowptr + min(r0 + R, a.n));
            };
            // the matrix part of tile t into stage s (bytes expected, no arrival): row pointers, values
            // and the entries' window-buffer indices
            auto issue_matrix = [&](long long t, int s, int e0, int e1) {
                const int r0 = (int)(t * R);
                const int rows = min(R, a.n - r0);
                const int vs = e0 & ~(VA - 1), ve = (e1 + VA - 1) & ~(VA - 1);
                const int cs = e0 & ~(CA - 1), ce = (e1 + CA - 1) & ~(CA - 1);
                const bool staged = (ve - vs) <= a.cap && (ce - cs) <= a.cap && e1 > e0;
                unsigned char *base = smem + s * stage_bytes;
                const uint32_t rpb = ((uint32_t)(rows + 1) * 4u + 15u) & ~15u;
                const uint32_t vb = staged ? (uint32_t)(ve - vs) * (uint32_t)sizeof(T) : 0u;
                const uint32_t cb = staged ? (uint32_t)(ce - cs) * 2u : 0u;
                mbar_expect_tx(&full[s], rpb + vb + cb);
                bulk_g2s(base, a.rowptr + r0, rpb, &full[s]);
                if (staged) {
                    bulk_g2s(base + val_off, a.vals + vs, vb, &full[s]);
                    bulk_g2s(base + col_off, p.lidx + cs, cb, &full[s]);
                }
            };
            // the vector part of tile t (x windows, row operands, header), then the arrival
            const T *x = nullptr;
            const T *sv[kWSlots] = {nullptr, nullptr, nullptr};
            // window descriptors of the prefetched stages and, one tile ahead, of the next tile
            int4 dlo[kSpmvStages], dln[kSpmvStages];
            auto desc = [&](long long t, int4 &lo4, int4 &ln4) {
                lo4 = __ldg(reinterpret_cast<const int4 *>(p.twin + t * 2 * kXWin));
                ln4 = __ldg(reinterpret_cast<const int4 *>(p.twin + t * 2 * kXWin + kXWin));
            };
            auto issue_vectors = [&](long long t, int s, const int4 lo4, const int4 ln4) {
                unsigned char *base = smem + s * stage_bytes;
                int *hd = reinterpret_cast<int *>(base + hd_off);
                const int r0 = (int)(t * R);
                const int lo[kXWin] = {lo4.x, lo4.y, lo4.z, lo4.w};
                const int ln[kXWin] = {ln4.x, ln4.y, ln4.z, ln4.w};
                uint32_t bytes = 0;
                int off = 0, nw = 0;
                for (int w = 0; w < kXWin; ++w) {
                    hd[w] = ln[w] > 0 ? lo[w] : 0x7fffffff;
                    hd[kXWin + w] = off;
                    if (ln[w] > 0) {
                        bytes += (uint32_t)ln[w] * 4u;
                        off += ln[w];
                        ++nw;
                    }
                }
                const bool full_tile = r0 + R <= a.n && p.nslot > 0;
                hd[2 * kXWin] = nw;
                hd[2 * kXWin + 1] = full_tile ? 1 : 0;
                if (full_tile) bytes += (uint32_t)p.nslot * (uint32_t)R * 4u;
                mbar_arrive_expect_tx(&full[s], bytes);
                for (int w = 0, o = 0; w < kXWin; ++w)
                    if (ln[w] > 0) {
                        bulk_g2s(base + xw_off + (size_t)o * 4, x + lo[w], (uint32_t)ln[w] * 4u, &full[s]);
                        o += ln[w];
                    }
                if (full_tile)
                    for (int q = 0; q < p.nslot; ++q)
                        bulk_g2s(base + sl_off + (size_t)q * 256 * 4, sv[q] + r0, (uint32_t)R * 4u, &full[s]);
            };
            int ne0 = 0, ne1 = 0;
            int4 nlo = make_int4(0, 0, 0, 0), nln = make_int4(0, 0, 0, 0);
            if (my_tiles > 0) {
                bounds(blockIdx.x, ne0, ne1);
                desc(blockIdx.x, nlo, nln);
            }
            int i = 0;
            bool waited = false;
            for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
                if (i == prefetched) {
                    waited = true;
                    pdl_wait();
                    pdl_trigger();
                    if ((a.check_done == kSkipIfDone && st->cycle_done) ||
                        (a.check_done == kSkipIfNoCols && st->k == 0)) {
                        // the prefetched stages still expect no arrival: complete them so that the
                        // consumers' drain can see their copies land
                        for (int q = 0; q < prefetched; ++q) mbar_arrive(&full[q]);
                        break;
                    }
                    x = resolve_ptr<T>(a.e.x, st);
                    for (int q = 0; q < p.nslot; ++q) sv[q] = resolve_ptr<T>(p.slot[q], st);
                    for (int q = 0; q < prefetched; ++q)
                        issue_vectors(blockIdx.x + (long long)q * gridDim.x, q, dlo[q], dln[q]);
                }
                const int e0 = ne0, e1 = ne1;
                const int4 clo = nlo, cln = nln;
                if (tile + gridDim.x < ntiles) {
                    bounds(tile + gridDim.x, ne0, ne1);
                    desc(tile + gridDim.x, nlo, nln);
                }
                const int s = i % kSpmvStages, round = i / kSpmvStages;
                if (round > 0 && !mbar_wait_bounded(&empty[s], (round - 1) & 1, kWaitLimitNs)) {
                    timeout_stop(st);
                    break;
                }
                issue_matrix(tile, s, e0, e1);
                if (i >= prefetched) issue_vectors(tile, s, clo, cln);
                else {
                    dlo[i] = clo;
                    dln[i] = cln;
                }
            }
            if (!waited) {
                // no more tiles than stages: the wait and the vector parts were not reached in the loop
                pdl_wait();
                pdl_trigger();
                if ((a.check_done == kSkipIfDone && st->cycle_done) ||
                    (a.check_done == kSkipIfNoCols && st->k == 0)) {
                    for (int q = 0; q < i; ++q) mbar_arrive(&full[q]);
                } else {
                    x = resolve_ptr<T>(a.e.x, st);
                    for (int q = 0; q < p.nslot; ++q) sv[q] = resolve_ptr<T>(p.slot[q], st);
                    for (int q = 0; q < i; ++q) issue_vectors(blockIdx.x + (long long)q * gridDim.x, q, dlo[q], dln[q]);
                }
            }
        }
        return;
    }

    // consumers: nothing a predecessor wrote is read before this point
    pdl_wait();
    pdl_trigger();
    if ((a.check_done == kSkipIfDone && st->cycle_done) || (a.check_done == kSkipIfNoCols && st->k == 0)) {
        for (int q = 0; q < prefetched; ++q) mbar_wait_bounded(&full[q], 0, kWaitLimitNs);
        return;
    }
    if (tid < 7) {
        switch (tid) {
        case 0: s_coef[0] = resolve(a.e.a0, st); break;
        case 1: s_coef[1] = resolve(a.e.b0, st); break;
        case 2: s_coef[2] = resolve(a.e.c0, st); break;
        case 3: s_coef[3] = resolve(a.e.a1, st); break;
        case 4: s_coef[4] = resolve(a.e.b1, st); break;
        case 5: s_coef[5] = resolve(a.e.c1, st); break;
        default: s_coef[6] = resolve(a.e.s2, st); break;
        }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kSpmvConsumerWarps * 32) : "memory");

    const T *__restrict__ x = resolve_ptr<T>(a.e.x, st);
    T *o0 = resolve_ptr<T>(a.e.out0, st);
    const T *u0 = resolve_ptr<T>(a.e.u0, st);
    const T *w0 = resolve_ptr<T>(a.e.w0, st);
    T *o1 = resolve_ptr<T>(a.e.out1, st);
    const T *u1 = resolve_ptr<T>(a.e.u1, st);
    const T *w1 = resolve_ptr<T>(a.e.w1, st);
    const T ca0 = (T)s_coef[0], cb0 = (T)s_coef[1], cc0 = (T)s_coef[2];
    const T ca1 = (T)s_coef[3], cb1 = (T)s_coef[4], cc1 = (T)s_coef[5];
    const int lr = tid / G;
    const int lg = tid & (G - 1);
    int i = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
        const int s = i % kSpmvStages;
        if (!mbar_wait_bounded(&full[s], (i / kSpmvStages) & 1, kWaitLimitNs)) {
            if (lane == 0) timeout_stop(st);
            mbar_wait_bounded(&full[s], (i / kSpmvStages) & 1, kWaitLimitNs);
            return;
        }
        const unsigned char *base = smem + s * stage_bytes;
        const int *s_rp = reinterpret_cast<const int *>(base);
        const T *s_val = reinterpret_cast<const T *>(base + val_off);
        const short *s_li = reinterpret_cast<const short *>(base + col_off);
        const T *s_x = reinterpret_cast<const T *>(base + xw_off);
        const T *s_sl = reinterpret_cast<const T *>(base + sl_off);
        const int *hd = reinterpret_cast<const int *>(base + hd_off);
        const int nw = hd[2 * kXWin];
        const bool rows_staged = hd[2 * kXWin + 1] != 0;
        const int r0 = (int)(tile * R);
        const int rows = min(R, a.n - r0);
        const int e0 = s_rp[0], e1 = s_rp[rows];
        const int vs = e0 & ~(VA - 1), ve = (e1 + VA - 1) & ~(VA - 1);
        const int cs = e0 & ~(CA - 1), ce = (e1 + CA - 1) & ~(CA - 1);
        const bool staged = (ve - vs) <= a.cap && (ce - cs) <= a.cap && e1 > e0;
        const int l = lr;
        const bool ok = l < rows;
        const int rr = r0 + l;
        int kb = ok ? s_rp[l] + lg : 0;
        const int ke = ok ? s_rp[l + 1] : 0;
        T acc = T(0), pu0 = T(0), pw0 = T(0), pu1 = T(0), pw1 = T(0);
        if (lg == 0 && ok) {
            if (rows_staged) {
                if (u0) pu0 = s_sl[p.slot_of[0] * 256 + l];
                if (w0) pw0 = s_sl[p.slot_of[1] * 256 + l];
                if (o1) {
                    if (u1) pu1 = s_sl[p.slot_of[2] * 256 + l];
                    if (w1) pw1 = s_sl[p.slot_of[3] * 256 + l];
                }
            } else {
                if (u0) pu0 = u0[rr];
                if (w0) pw0 = w0[rr];
                if (o1) {
                    if (u1) pu1 = u1[rr];
                    if (w1) pw1 = w1[rr];
                }
            }
        }
        if (staged && nw > 0) {
            // every column lies in the staged windows: one shared-memory load per entry
            bool more = true;
            while (more) {
                bool in[8];
                T xv[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int kk = kb + t * G;
                    in[t] = kk < ke;
                    xv[t] = in[t] ? s_x[s_li[kk - cs]] : T(0);
                }
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (in[t]) acc = fma(s_val[kb + t * G - vs], xv[t], acc);
                kb += 8 * G;
                more = kb < ke;
            }
        } else if (staged) {
            // no windows for this tile: the values are staged, the columns and x come from global memory
            bool more = true;
            while (more) {
                int qc[8];
                T xv[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int kk = kb + t * G;
                    qc[t] = kk < ke ? col_of<IDX>(__ldg(a.cols + kk), rr) : -1;
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) xv[t] = qc[t] >= 0 ? __ldg(x + qc[t]) : T(0);
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (qc[t] >= 0) acc = fma(s_val[kb + t * G - vs], xv[t], acc);
                kb += 8 * G;
                more = kb < ke;
            }
        } else {
            for (int k = kb; k < ke; k += G) {
                const int qq = col_of<IDX>(__ldg(a.cols + k), rr);
                acc = fma(__ldg(a.vals + k), __ldg(x + qq), acc);
            }
        }
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lg == 0 && ok) {
            T v = ca0 * acc;
            if (u0) v = fma(cb0, pu0, v);
            if (w0) v = fma(cc0, pw0, v);
            o0[rr] = v;
            if (o1) {
                T v1 = ca1 * acc;
                if (u1) v1 = fma(cb1, pu1, v1);
                if (w1) v1 = fma(cc1, pw1, v1);
                o1[rr] = v1;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ---------------------------------------------------------------- staged x windows, tile-ELL (float32)

// As k_spmv_w for one thread per row, with each tile of kThreads rows stored as a dense R x w block
// (entry k of row l at k R + l): the stage holds the block's values and window indices and the tile's
// x windows plus a zero at index xcap (the matrix's longest window total, at most kXCap) for the
// padding, so a row is w shared-memory multiply-adds with no row pointers or bounds tests.  G: the
// row-block kernel's lanes per row; the thread keeps G sums (entries k = g mod G) and combines them
// in that kernel's shuffle order, so the results are k_spmv's bits (padding adds 0 * 0).  X2: the
// epilogue's second input x2 (A (x + s2 x2)) is staged too, over the same windows, and combined per
// gathered entry as k_spmv does.
__host__ __device__ constexpr size_t spmve_stage_bytes(int wmax, bool x2, int xcap, int sv = 4)
{
    return round128((size_t)kThreads * wmax * sv) + round128((size_t)kThreads * wmax * 2) +
           (x2 ? 2 : 1) * round128((size_t)(xcap + 4) * sv) + 128;
}

struct SpmvEArgs {
    int n;
    const void *vals;   // tile-ELL values (float or double, the kernel's T)
    const short *idx;   // tile-ELL window indices
    const int *toff;
    const int *twin;
    int wmax;
    int xcap;  // index of the zero after the windows (padding entries point there)
    int nst;   // pipeline stages in use (2 or 3: three when they fit the shared memory)
    Cycle *st;
    int check_done;
    SpmvEpi e;
};

template <typename T, bool X2, int G>
__global__ void __launch_bounds__(kSpmvThreads, PPG_SPMV_MIN_BLOCKS) k_spmv_e(SpmvEArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kSpmvStages];
    __shared__ __align__(8) uint64_t empty[kSpmvStages];
    __shared__ int4 s_desc[kSpmvStages][4];
    __shared__ double s_coef[7];
    constexpr int R = kThreads;
    constexpr int SV = (int)sizeof(T);
    const T *vals = static_cast<const T *>(a.vals);
    const int S = a.nst;

    Cycle *st = a.st;
    const long long ntiles = ((long long)a.n + R - 1) / R;
    const size_t stage_bytes = spmve_stage_bytes(a.wmax, X2, a.xcap, SV);
    const size_t ix_off = round128((size_t)R * a.wmax * SV);
    const size_t xw_off = ix_off + round128((size_t)R * a.wmax * 2);
    const size_t xw_bytes = round128((size_t)(a.xcap + 4) * SV);
    const size_t hd_off = xw_off + (X2 ? 2 : 1) * xw_bytes;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int prefetched = (int)min((long long)S, my_tiles);
    // the CTA's i-th tile; a reversed launch visits the same tiles last to first, so it starts on the
    // tiles the previous (forward) link read last, which are still in L2
    const bool rev = a.e.rev != 0;
    auto tile_at = [&](long long i) { return blockIdx.x + (rev ? my_tiles - 1 - i : i) * (long long)gridDim.x; };

    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kSpmvConsumerWarps);
        }
        fence_mbar_init();
    }
    if (tid < S * 4) {  // the zero the padding indexes, in every stage (no copy writes there)
        T *z = reinterpret_cast<T *>(smem + (tid / 4) * stage_bytes + xw_off);
        z[a.xcap + (tid & 3)] = T(0);
        if (X2) z[xw_bytes / SV + a.xcap + (tid & 3)] = T(0);
    }
    __syncthreads();

    if (wid == kSpmvConsumerWarps) {
        // ---------------- producer
        if (lane == 0) {
            // a tile's window descriptors: starts in d[0..1], lengths in d[2..3] (kEWin each); those of
            // the tiles requested before the wait are kept in shared memory until their windows are
            // requested after it
            auto desc = [&](long long t, int4 *d) {
                const int4 *src = reinterpret_cast<const int4 *>(a.twin + t * 2 * kEWin);
#pragma unroll
                for (int u = 0; u < 4; ++u) d[u] = __ldg(src + u);
            };
            auto span = [&](long long t, int &o0, int &o1) {
                o0 = __ldg(a.toff + t);
                o1 = __ldg(a.toff + t + 1);
            };
            auto issue_matrix = [&](int s, int o0, int o1) {
                unsigned char *base = smem + s * stage_bytes;
                const uint32_t nb = (uint32_t)(o1 - o0);
                mbar_expect_tx(&full[s], nb * (uint32_t)(SV + 2));
                if (nb) {
                    bulk_g2s(base, vals + o0, nb * (uint32_t)SV, &full[s]);
                    bulk_g2s(base + ix_off, a.idx + o0, nb * 2u, &full[s]);
                }
                reinterpret_cast<int *>(base + hd_off)[0] = (int)(nb / R);
            };
            const T *x = nullptr, *x2 = nullptr;
            auto issue_vectors = [&](int s, const int4 *d) {
                unsigned char *base = smem + s * stage_bytes;
                const int lo[kEWin] = {d[0].x, d[0].y, d[0].z, d[0].w, d[1].x, d[1].y, d[1].z, d[1].w};
                const int ln[kEWin] = {d[2].x, d[2].y, d[2].z, d[2].w, d[3].x, d[3].y, d[3].z, d[3].w};
                uint32_t bytes = 0;
#pragma unroll
                for (int w = 0; w < kEWin; ++w) bytes += (uint32_t)ln[w] * (uint32_t)SV;
                mbar_arrive_expect_tx(&full[s], X2 ? 2 * bytes : bytes);
                int o = 0;
#pragma unroll
                for (int w = 0; w < kEWin; ++w)
                    if (ln[w] > 0) {
                        bulk_g2s(base + xw_off + (size_t)o * SV, x + lo[w], (uint32_t)ln[w] * (uint32_t)SV, &full[s]);
                        if (X2)
                            bulk_g2s(base + xw_off + xw_bytes + (size_t)o * SV, x2 + lo[w],
                                     (uint32_t)ln[w] * (uint32_t)SV, &full[s]);
                        o += ln[w];
                    }
            };
            int no0 = 0, no1 = 0;
            int4 nd[4];
            if (my_tiles > 0) {
                span(tile_at(0), no0, no1);
                desc(tile_at(0), nd);
            }
            int i = 0, ps = 0, pround = 0;  // stage and round of tile i (no division by S)
            bool waited = false;
            for (; i < my_tiles; ++i) {
                if (i == prefetched) {
                    waited = true;
                    pdl_wait();
                    pdl_trigger();
                    if ((a.check_done == kSkipIfDone && st->cycle_done) ||
                        (a.check_done == kSkipIfNoCols && st->k == 0)) {
                        for (int q = 0; q < prefetched; ++q) mbar_arrive(&full[q]);
                        break;
                    }
                    x = resolve_ptr<T>(a.e.x, st);
                    if (X2) x2 = resolve_ptr<T>(a.e.x2, st);
                    for (int q = 0; q < prefetched; ++q) issue_vectors(q, s_desc[q]);
                }
                // this tile's bounds and descriptors (loaded one step ago); the next tile's are
                // loaded while this stage waits to be free
                const int o0 = no0, o1 = no1;
                const int s = ps, round = pround;
                if (++ps == S) {
                    ps = 0;
                    ++pround;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) s_desc[s][u] = nd[u];
                if (i + 1 < my_tiles) {
                    span(tile_at(i + 1), no0, no1);
                    desc(tile_at(i + 1), nd);
                }
                if (round > 0 && !mbar_wait_bounded(&empty[s], (round - 1) & 1, kWaitLimitNs)) {
                    timeout_stop(st);
                    break;
                }
                issue_matrix(s, o0, o1);
                if (i >= prefetched) issue_vectors(s, s_desc[s]);
            }
            if (!waited) {
                pdl_wait();
                pdl_trigger();
                if ((a.check_done == kSkipIfDone && st->cycle_done) ||
                    (a.check_done == kSkipIfNoCols && st->k == 0)) {
                    for (int q = 0; q < i; ++q) mbar_arrive(&full[q]);
                } else {
                    x = resolve_ptr<T>(a.e.x, st);
                    if (X2) x2 = resolve_ptr<T>(a.e.x2, st);
                    for (int q = 0; q < i; ++q) issue_vectors(q, s_desc[q]);
                }
            }
        }
        return;
    }

    // consumers: nothing a predecessor wrote is read before this point
    pdl_wait();
    pdl_trigger();
    if ((a.check_done == kSkipIfDone && st->cycle_done) || (a.check_done == kSkipIfNoCols && st->k == 0)) {
        for (int q = 0; q < prefetched; ++q) mbar_wait_bounded(&full[q], 0, kWaitLimitNs);
        return;
    }
    if (tid < 7) {
        switch (tid) {
        case 0: s_coef[0] = resolve(a.e.a0, st); break;
        case 1: s_coef[1] = resolve(a.e.b0, st); break;
        case 2: s_coef[2] = resolve(a.e.c0, st); break;
        case 3: s_coef[3] = resolve(a.e.a1, st); break;
        case 4: s_coef[4] = resolve(a.e.b1, st); break;
        case 5: s_coef[5] = resolve(a.e.c1, st); break;
        default: s_coef[6] = resolve(a.e.s2, st); break;
        }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kSpmvConsumerWarps * 32) : "memory");

    T *o0 = resolve_ptr<T>(a.e.out0, st);
    const T *u0 = resolve_ptr<T>(a.e.u0, st);
    const T *w0 = resolve_ptr<T>(a.e.w0, st);
    T *o1 = resolve_ptr<T>(a.e.out1, st);
    const T *u1 = resolve_ptr<T>(a.e.u1, st);
    const T *w1 = resolve_ptr<T>(a.e.w1, st);
    const T ca0 = (T)s_coef[0], cb0 = (T)s_coef[1], cc0 = (T)s_coef[2];
    const T ca1 = (T)s_coef[3], cb1 = (T)s_coef[4], cc1 = (T)s_coef[5];
    const T c2 = (T)s_coef[6];
    int s = 0;
    uint32_t ph = 0;  // stage and phase of the current tile (no division by S)
    for (long long i = 0; i < my_tiles; ++i) {
        const long long tile = tile_at(i);
        const int rr = (int)(tile * R) + tid;
        const bool ok = rr < a.n;
        // row operands first: their loads overlap the wait and the products
        T pu0 = T(0), pw0 = T(0), pu1 = T(0), pw1 = T(0);
        if (ok) {
            if (u0) pu0 = u0[rr];
            if (w0) pw0 = w0[rr];
            if (o1) {
                if (u1) pu1 = u1[rr];
                if (w1) pw1 = w1[rr];
            }
        }
        if (!mbar_wait_bounded(&full[s], ph, kWaitLimitNs)) {
            if (lane == 0) timeout_stop(st);
            mbar_wait_bounded(&full[s], ph, kWaitLimitNs);
            return;
        }
        const unsigned char *base = smem + s * stage_bytes;
        const T *s_val = reinterpret_cast<const T *>(base);
        const short *s_ix = reinterpret_cast<const short *>(base + ix_off);
        const T *s_x = reinterpret_cast<const T *>(base + xw_off);
        const int w = reinterpret_cast<const int *>(base + hd_off)[0];
        T acc = T(0);
        if constexpr (G == 1) {
            if (X2) {
                const T *s_x2 = s_x + xw_bytes / SV;
#pragma unroll 8
                for (int k = 0; k < w; ++k) {
                    const int q = s_ix[k * R + tid];
                    acc = fma(s_val[k * R + tid], fma(c2, s_x2[q], s_x[q]), acc);
                }
            } else {
#pragma unroll 8
                for (int k = 0; k < w; ++k) acc = fma(s_val[k * R + tid], s_x[s_ix[k * R + tid]], acc);
            }
        } else {
            // w is a multiple of G (the host pads each tile to it)
            T part[G];
#pragma unroll
            for (int g = 0; g < G; ++g) part[g] = T(0);
            const T *s_x2 = s_x + xw_bytes / SV;
#pragma unroll 2
            for (int k = 0; k < w; k += G) {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int e = (k + g) * R + tid;
                    const int q = s_ix[e];
                    const T xv = X2 ? fma(c2, s_x2[q], s_x[q]) : s_x[q];
                    part[g] = fma(s_val[e], xv, part[g]);
                }
            }
#pragma unroll
            for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
                for (int l = 0; l < o; ++l) part[l] = part[l] + part[l + o];
            acc = part[0];
        }
        if (ok) {
            T v = ca0 * acc;
            if (u0) v = fma(cb0, pu0, v);
            if (w0) v = fma(cc0, pw0, v);
            o0[rr] = v;
            if (o1) {
                T v1 = ca1 * acc;
                if (u1) v1 = fma(cb1, pu1, v1);
                if (w1) v1 = fma(cc1, pw1, v1);
                o1[rr] = v1;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == S) {
            s = 0;
            ph ^= 1u;
        }
    }
}

// ---------------------------------------------------------------- two chain steps in one launch

// A tile's staged matrix data serves two consecutive links of the p(A) chain (Section II,
// Eq. 2): y1 = step 1 (A x), y2 = step 2 (A y1), where y2's input is an output of step 1.
// Tiles are dealt round-robin, so round i of the persistent grid covers tiles i G .. i G + G-1.
// Each CTA runs step 1 on its round-i tile, then step 2 on its round-(i-2) tile from the same
// (still resident) stage.  Step 2 of a tile gathers step-1 rows up to the matrix bandwidth away;
// with the bandwidth at most G tiles these lie in rounds i-3 .. i-1, whose completion the CTAs
// count in round_done (a bounded wait; the last CTA clears the counters).  The CTAs wait on one
// another, so the kernel is launched cooperatively (the whole grid resident at once).  The rows step 2
// writes are no longer gathered by any step 1 at that point (rounds up to i-1 are complete and
// round i gathers only rounds i-1 .. i+1), so step 2 may write into step 1's input vector.
constexpr int kSpmv2Lag = 2;
constexpr int kSpmv2Stages = kSpmvStages + kSpmv2Lag;

template <typename T, typename IDX>
struct Spmv2Args {
    SpmvArgs<T, IDX> a;  // a.e: the first step
    SpmvEpi e2;          // the second step (x, x2: outputs of the first)
    int *round_done;     // per round: CTAs that have finished its first step (zero at launch)
    unsigned int *ticket;
    int *diag;           // 8 ints: where a bounded wait gave up (first CTA to time out)
    unsigned long long round_wait_ns;  // limit of one round-counter wait
    int extra_need;      // tests of the failure path: CTAs a round needs beyond the launch's (0 normally)
};

// records a wait that gave up: kind 1 full barrier, 2 round counter; the first CTA wins
__device__ __forceinline__ void spmv2_diag(int *diag, int kind, long long i, long long r, int have, int need)
{
    if (atomicCAS(diag, 0, kind) == 0) {
        diag[1] = blockIdx.x;
        diag[2] = (int)i;
        diag[3] = (int)r;
        diag[4] = have;
        diag[5] = need;
        diag[6] = gridDim.x;
    }
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename T, typename IDX>
__global__ void __launch_bounds__(kSpmvThreads, PPG_SPMV_MIN_BLOCKS) k_spmv2(Spmv2Args<T, IDX> p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kSpmv2Stages];
    __shared__ __align__(8) uint64_t empty[kSpmv2Stages];
    __shared__ double s_coef1[7], s_coef2[7];
    __shared__ int s_fail;

    const SpmvArgs<T, IDX> &a = p.a;
    Cycle *st = a.st;
    const int R = a.rows_per_tile;
    const int G = a.lanes_per_row;
    const long long ntiles = ((long long)a.n + R - 1) / R;
    const size_t stage_bytes = spmv_stage_bytes<T, IDX>(a.cap);
    const size_t val_off = kSpmvRpBytes;
    const size_t col_off = kSpmvRpBytes + round128((size_t)a.cap * sizeof(T));
    constexpr int VA = 16 / (int)sizeof(T);
    constexpr int CA = 16 / (int)sizeof(IDX);
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const long long NG = gridDim.x;
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / NG + 1 : 0;
    const int prefetched = (int)min((long long)kSpmvStages, my_tiles);

    if (tid == 0) {
        for (int q = 0; q < kSpmv2Stages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kSpmvConsumerWarps);
        }
        fence_mbar_init();
        s_fail = 0;
    }
    __syncthreads();

    if (wid == kSpmvConsumerWarps) {
        // ---------------- producer: as in k_spmv, with stages released after the second step
        if (lane == 0) {
            auto bounds = [&](long long t, int &e0, int &e1) {
                const int r0 = (int)(t * R);
                e0 = __ldg(a.rowptr + r0);
                e1 = __ldg(a.rowptr + min(r0 + R, a.n));
            };
            int ne0 = 0, ne1 = 0;
            if (my_tiles > 0) bounds(blockIdx.x, ne0, ne1);
            int i = 0;
            for (long long tile = blockIdx.x; tile < ntiles; tile += NG, ++i) {
                if (i == prefetched) {
                    pdl_wait();
                    pdl_trigger();
                    if ((a.check_done == kSkipIfDone && st->cycle_done) ||
                        (a.check_done == kSkipIfNoCols && st->k == 0))
                        break;
                }
                const int e0 = ne0, e1 = ne1;
                if (tile + NG < ntiles) bounds(tile + NG, ne0, ne1);
                const int s = i % kSpmv2Stages, use = i / kSpmv2Stages;
                if (use > 0 && !mbar_wait_bounded(&empty[s], (use - 1) & 1, kWaitLimitNs)) {
                    timeout_stop(st);
                    break;
                }
                const int r0 = (int)(tile * R);
                const int rows = min(R, a.n - r0);
                const int vs = e0 & ~(VA - 1), ve = (e1 + VA - 1) & ~(VA - 1);
                const int cs = e0 & ~(CA - 1), ce = (e1 + CA - 1) & ~(CA - 1);
                const bool staged = (ve - vs) <= a.cap && (ce - cs) <= a.cap && e1 > e0;
                unsigned char *base = smem + s * stage_bytes;
                const uint32_t rpb = ((uint32_t)(rows + 1) * 4u + 15u) & ~15u;
                const uint32_t vb = staged ? (uint32_t)(ve - vs) * (uint32_t)sizeof(T) : 0u;
                const uint32_t cb = staged ? (uint32_t)(ce - cs) * (uint32_t)sizeof(IDX) : 0u;
                mbar_arrive_expect_tx(&full[s], rpb + vb + cb);
                bulk_g2s(base, a.rowptr + r0, rpb, &full[s]);
                if (staged) {
                    bulk_g2s(base + val_off, a.vals + vs, vb, &full[s]);
                    bulk_g2s(base + col_off, a.cols + cs, cb, &full[s]);
                }
            }
        }
        return;
    }

    pdl_wait();
    pdl_trigger();
    if ((a.check_done == kSkipIfDone && st->cycle_done) || (a.check_done == kSkipIfNoCols && st->k == 0)) {
        for (int q = 0; q < prefetched; ++q) mbar_wait_bounded(&full[q], 0, kWaitLimitNs);
        return;
    }
    const EpiRes<T> E1 = resolve_epi<T>(a.e, st, s_coef1, tid);
    const EpiRes<T> E2 = resolve_epi<T>(p.e2, st, s_coef2, tid);
    const long long nrounds = (ntiles + NG - 1) / NG;
    int loaded = 0;  // stages this CTA's consumers have waited for (all copies issued so far landed)
    for (long long i = 0; i < my_tiles + kSpmv2Lag; ++i) {
        if (i < my_tiles) {
            const int s = (int)(i % kSpmv2Stages);
            if (!mbar_wait_bounded(&full[s], (int)(i / kSpmv2Stages) & 1, kWaitLimitNs)) {
                if (lane == 0) {
                    timeout_stop(st);
                    spmv2_diag(p.diag, 1, i, i, s, 0);
                }
                s_fail = 1;
            }
            asm volatile("bar.sync 1, %0;" ::"n"(kSpmvConsumerWarps * 32) : "memory");
            if (s_fail) break;
            loaded = (int)i + 1;
            spmv_tile<T, IDX, false>(smem + s * stage_bytes, val_off, col_off, a.cap, blockIdx.x + i * NG, R, G,
                                     a.n, a.cols, a.vals, E1, tid);
            // this CTA's part of round i is written: publish it
            asm volatile("bar.sync 1, %0;" ::"n"(kSpmvConsumerWarps * 32) : "memory");
            if (tid == 0) {
                __threadfence();
                atomicAdd(p.round_done + i, 1);
            }
        }
        const long long j = i - kSpmv2Lag;
        if (j >= 0 && j < my_tiles) {
            if (tid == 0) {
                // first-step rows within the bandwidth of round j: rounds j-1 .. j+1 complete
                const unsigned long long t0 = global_timer_ns();
                for (long long r = (j > 0 ? j - 1 : 0); r <= j + 1 && r < nrounds && !s_fail; ++r) {
                    const int need = (int)min(NG, ntiles - r * NG) + p.extra_need;
                    for (unsigned int spins = 1; ld_acquire(p.round_done + r) < need; ++spins)
                        if ((spins & 63u) == 0 && global_timer_ns() - t0 > p.round_wait_ns) {
                            timeout_stop(st);
                            spmv2_diag(p.diag, 2, i, r, ld_acquire(p.round_done + r), need);
                            s_fail = 1;
                            break;
                        }
                }
            }
            asm volatile("bar.sync 1, %0;" ::"n"(kSpmvConsumerWarps * 32) : "memory");
            if (s_fail) break;
            const int s = (int)(j % kSpmv2Stages);
            spmv_tile<T, IDX, true>(smem + s * stage_bytes, val_off, col_off, a.cap, blockIdx.x + j * NG, R, G, a.n,
                                    a.cols, a.vals, E2, tid);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    if (s_fail) {
        // copies the producer issued but no consumer waited for land before the CTA exits
        for (long long q = loaded; q < my_tiles && q < loaded + kSpmv2Stages; ++q)
            if (tid == 0) mbar_wait_bounded(&full[q % kSpmv2Stages], (int)(q / kSpmv2Stages) & 1, kWaitLimitNs);
    }
    // the last CTA clears the round counters for the next launch
    asm volatile("bar.sync 1, %0;" ::"n"(kSpmvConsumerWarps * 32) : "memory");
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(p.ticket, 1u) == gridDim.x - 1) {
            for (long long r = 0; r < nrounds; ++r) p.round_done[r] = 0;
            __threadfence();
            *p.ticket = 0u;
        }
    }
}

// ---------------------------------------------------------------- the fused SpMV step, sliced ELL

// Streaming loads of matrix data: read once per launch, so they bypass L1 (which keeps the x gathers).
template <typename T>
__device__ __forceinline__ T ld_matrix(const T *p);
template <>
__device__ __forceinline__ double ld_matrix<double>(const double *p)
{
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
template <>
__device__ __forceinline__ float ld_matrix<float>(const float *p)
{
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
template <>
__device__ __forceinline__ short ld_matrix<short>(const short *p)
{
    unsigned short v;
    asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return (short)v;
}
template <>
__device__ __forceinline__ int ld_matrix<int>(const int *p)
{
    int v;
    asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// column of a sliced-ELL entry, or -1 for padding
template <typename IDX>
__device__ __forceinline__ int sell_col(IDX c, int r)
{
    if constexpr (sizeof(IDX) == 2)
        return c == kSellPadOff ? -1 : r + (int)c;
    else
        return (int)c;
}

template <typename T, typename IDX>
struct SellArgs {
    int n;
    int nslices;
    const int *sptr;
    const IDX *cols;
    const T *vals;
    Cycle *st;
    int check_done;
    SpmvEpi e;
};

#ifndef PPG_SELL_MIN_BLOCKS
#define PPG_SELL_MIN_BLOCKS 8  // 128-thread CTAs per SM the register allocation is sized for (float)
#endif
#ifndef PPG_SELL_MIN_BLOCKS_64
#define PPG_SELL_MIN_BLOCKS_64 4  // (double)
#endif

constexpr int kSellWarps = 4;  // slices per 128-thread CTA
constexpr int kSellChunk = 8;  // entries of a row loaded together

// Loads chunk k0 of a slice's entries for one lane: kSellChunk entries 32 apart (padding and
// entries past the slice read as value 0, column -1).
template <typename T, typename IDX>
__device__ __forceinline__ void sell_load(const T *vals, const IDX *cols, int k0, int ke, int lane, int row, T *v,
                                          int *c)
{
#pragma unroll
    for (int u = 0; u < kSellChunk; ++u) {
        const int k = k0 + 32 * u;
        const bool in = k < ke;
        v[u] = in ? ld_matrix<T>(vals + k + lane) : T(0);
        c[u] = in ? sell_col<IDX>(ld_matrix<IDX>(cols + k + lane), row) : -1;
    }
}

template <typename T>
__device__ __forceinline__ T sell_dot(const T *__restrict__ x, const T *__restrict__ x2, T c2, const T *v,
                                      const int *c, T acc)
{
    T xv[kSellChunk];
    if (x2 == nullptr) {
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : T(0);
    } else {
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) xv[u] = c[u] >= 0 ? fma(c2, __ldg(x2 + c[u]), __ldg(x + c[u])) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kSellChunk; ++u)
        if (c[u] >= 0) acc = fma(v[u], xv[u], acc);
    return acc;
}

// Persistent: each CTA owns a contiguous range of 32-row slices (neighbouring rows share x in
// L1) and its warps take every kSellWarps-th slice of it, one lane per row.  A slice's entries
// are stored entry index by entry index, so each load of values and indices is one coalesced
// request.  The first entries of the next slice are requested before this slice's x gathers,
// and the first slice's before the wait on the predecessor kernel (the matrix is constant),
// which overlaps them with the previous link of the chain.  Epilogue as in k_spmv.
template <typename T, typename IDX>
__global__ void __launch_bounds__(kSellWarps * 32, sizeof(T) == 4 ? PPG_SELL_MIN_BLOCKS : PPG_SELL_MIN_BLOCKS_64)
    k_spmv_sell(SellArgs<T, IDX> a)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int per = (a.nslices + gridDim.x - 1) / gridDim.x;
    const int s_end = min(a.nslices, (int)blockIdx.x * per + per);
    int sl = (int)blockIdx.x * per + wid;
    if (sl >= s_end) return;
    T v[kSellChunk];
    int c[kSellChunk];
    int kb = a.sptr[sl], ke = a.sptr[sl + 1];
    int kbn = 0, ken = 0;
    if (sl + kSellWarps < s_end) {
        kbn = a.sptr[sl + kSellWarps];
        ken = a.sptr[sl + kSellWarps + 1];
    }
    sell_load<T, IDX>(a.vals, a.cols, kb, ke, lane, sl * 32 + lane, v, c);

    pdl_wait();
    pdl_trigger();
    const Cycle *st = a.st;
    if ((a.check_done == kSkipIfDone && st->cycle_done) || (a.check_done == kSkipIfNoCols && st->k == 0)) return;
    double cf = 0.0;
    switch (lane) {
    case 0: cf = resolve(a.e.a0, st); break;
    case 1: cf = resolve(a.e.b0, st); break;
    case 2: cf = resolve(a.e.c0, st); break;
    case 3: cf = resolve(a.e.a1, st); break;
    case 4: cf = resolve(a.e.b1, st); break;
    case 5: cf = resolve(a.e.c1, st); break;
    case 6: cf = resolve(a.e.s2, st); break;
    default: break;
    }
    const T ca0 = (T)__shfl_sync(0xffffffffu, cf, 0), cb0 = (T)__shfl_sync(0xffffffffu, cf, 1);
    const T cc0 = (T)__shfl_sync(0xffffffffu, cf, 2), ca1 = (T)__shfl_sync(0xffffffffu, cf, 3);
    const T cb1 = (T)__shfl_sync(0xffffffffu, cf, 4), cc1 = (T)__shfl_sync(0xffffffffu, cf, 5);
    const T c2 = (T)__shfl_sync(0xffffffffu, cf, 6);
    const T *__restrict__ x = resolve_ptr<T>(a.e.x, st);
    const T *__restrict__ x2 = resolve_ptr<T>(a.e.x2, st);
    T *o0 = resolve_ptr<T>(a.e.out0, st);
    const T *u0 = resolve_ptr<T>(a.e.u0, st);
    const T *w0 = resolve_ptr<T>(a.e.w0, st);
    T *o1 = resolve_ptr<T>(a.e.out1, st);
    const T *u1 = resolve_ptr<T>(a.e.u1, st);
    const T *w1 = resolve_ptr<T>(a.e.w1, st);

    for (; sl < s_end; sl += kSellWarps) {
        const int row = sl * 32 + lane;
        const bool live = row < a.n;
        // epilogue operands first: their loads overlap the gathers
        T pu0 = T(0), pw0 = T(0), pu1 = T(0), pw1 = T(0);
        if (live) {
            if (u0) pu0 = u0[row];
            if (w0) pw0 = w0[row];
            if (o1) {
                if (u1) pu1 = u1[row];
                if (w1) pw1 = w1[row];
            }
        }
        // the next slice's first entries and the slice offsets of the one after it
        const int sn = sl + kSellWarps;
        T vn[kSellChunk];
        int cn[kSellChunk];
        sell_load<T, IDX>(a.vals, a.cols, kbn, ken, lane, sn * 32 + lane, vn, cn);
        int kbnn = 0, kenn = 0;
        if (sn + kSellWarps < s_end) {
            kbnn = a.sptr[sn + kSellWarps];
            kenn = a.sptr[sn + kSellWarps + 1];
        }
        T acc = sell_dot<T>(x, x2, c2, v, c, T(0));
        for (int k = kb + 32 * kSellChunk; k < ke; k += 32 * kSellChunk) {  // rows longer than one chunk
            sell_load<T, IDX>(a.vals, a.cols, k, ke, lane, row, v, c);
            acc = sell_dot<T>(x, x2, c2, v, c, acc);
        }
        if (live) {
            T r0 = ca0 * acc;
            if (u0) r0 = fma(cb0, pu0, r0);
            if (w0) r0 = fma(cc0, pw0, r0);
            o0[row] = r0;
            if (o1) {
                T r1 = ca1 * acc;
                if (u1) r1 = fma(cb1, pu1, r1);
                if (w1) r1 = fma(cc1, pw1, r1);
                o1[row] = r1;
            }
        }
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) {
            v[u] = vn[u];
            c[u] = cn[u];
        }
        kb = kbn;
        ke = ken;
        kbn = kbnn;
        ken = kenn;
    }
}

// one thread per row (rows n .. 32 nslices - 1 are empty): copies the row's entries into its
// slice and marks the slice's remaining entries of the row as padding
__global__ void k_sell_fill(int n, int nslices, const int *__restrict__ rowptr, const int *__restrict__ colidx,
                            const double *__restrict__ vals, const int *__restrict__ sptr, short *soff, int *scol,
                            double *svals)
{
    const int stride = gridDim.x * blockDim.x;
    const int rows = nslices * 32;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
        const int sl = r >> 5;
        const int base = sptr[sl] + (r & 31);
        const int width = (sptr[sl + 1] - sptr[sl]) >> 5;
        const int k0 = r < n ? rowptr[r] : 0, len = r < n ? rowptr[r + 1] - k0 : 0;
        for (int q = 0; q < width; ++q) {
            const int pos = base + 32 * q;
            const bool real = q < len;
            svals[pos] = real ? vals[k0 + q] : 0.0;
            if (soff) soff[pos] = real ? (short)(colidx[k0 + q] - r) : kSellPadOff;
            if (scol) scol[pos] = real ? colidx[k0 + q] : -1;
        }
    }
}

cudaError_t launch_sell_fill(int n, int nslices, const int *rowptr, const int *colidx, const double *vals,
                             const int *sptr, short *soff, int *scol, double *svals, cudaStream_t s)
{
    int grid = (nslices * 32 + kThreads - 1) / kThreads;
    if (grid > 8192) grid = 8192;
    if (grid < 1) grid = 1;
    k_sell_fill<<<grid, kThreads, 0, s>>>(n, nslices, rowptr, colidx, vals, sptr, soff, scol, svals);
    return cudaGetLastError();
}

namespace {
template <typename T, typename IDX>
int spmv_per_sm(int cap)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv<T, IDX>, kSpmvThreads,
                                                  kSpmvStages * spmv_stage_bytes<T, IDX>(cap));
    if (PPG_SPMV_CTAS_PER_SM > 0 && nb > PPG_SPMV_CTAS_PER_SM) nb = PPG_SPMV_CTAS_PER_SM;
    return nb > 0 ? nb : 1;
}

template <typename T, typename IDX>
cudaError_t spmv_go(const DevMatrix &A, const T *vals, const IDX *cols, int cap, int blocks, const SpmvEpi &e,
                    Cycle *st, int check_done, cudaStream_t s)
{
    const int R = A.rows_per_tile;
    const long long ntiles = ((long long)A.n + R - 1) / R;
    SpmvArgs<T, IDX> a{A.n, A.rowptr, cols, vals, R, A.lanes_per_row, cap, st, check_done, e};
    long long g = blocks;
    if (g > ntiles) g = ntiles;
    return launch_pdl(k_spmv<T, IDX>, dim3((unsigned)g), dim3(kSpmvThreads),
                      kSpmvStages * spmv_stage_bytes<T, IDX>(cap), s, a);
}

// the opt-in shared memory per CTA of this device
int smem_optin()
{
    static int v = 0;
    if (v == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (v <= 0) v = 48 * 1024;
    }
    return v;
}

// CTAs per SM of the two-step kernel, 0 when its stages do not fit a CTA's shared memory
template <typename T, typename IDX>
int spmv2_per_sm(int cap)
{
    if (kSpmv2Stages * spmv_stage_bytes<T, IDX>(cap) + 1024 > (size_t)smem_optin()) return 0;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv2<T, IDX>, kSpmvThreads,
                                                  kSpmv2Stages * spmv_stage_bytes<T, IDX>(cap));
    return nb > 0 ? nb : 0;
}

template <typename T, typename IDX>
cudaError_t spmv2_go(const DevMatrix &A, const T *vals, const IDX *cols, int cap, int blocks, const SpmvEpi &e1,
                     const SpmvEpi &e2, Cycle *st, int check_done, int *round_done, unsigned int *ticket, int *diag,
                     const WaitCfg &wc, cudaStream_t s)
{
    const int R = A.rows_per_tile;
    const long long ntiles = ((long long)A.n + R - 1) / R;
    Spmv2Args<T, IDX> p{{A.n, A.rowptr, cols, vals, R, A.lanes_per_row, cap, st, check_done, e1},
                        e2, round_done, ticket, diag, wc.ns, wc.extra_need};
    long long g = blocks;
    if (g > ntiles) g = ntiles;
    return launch_coop(k_spmv2<T, IDX>, dim3((unsigned)g), dim3(kSpmvThreads),
                       kSpmv2Stages * spmv_stage_bytes<T, IDX>(cap), s, p);
}

bool vec_same(const VecRef &u, const VecRef &v)
{
    return u.base == v.base && u.ld == v.ld && u.col == v.col && u.follow == v.follow;
}

// a vector the TMA engine may copy from: 16-byte aligned start, and for a column reference a
// column stride of whole 16-byte units
bool vec_aligned(const VecRef &v)
{
    return ((uintptr_t)v.base & 15u) == 0 && (v.follow == 0 || ((v.ld * 4) & 15) == 0) &&
           (((long long)v.col * v.ld * 4) & 15) == 0;
}

// The tile-ELL launch for value type T (float: ell[0], double: ell[1]).
template <typename T>
cudaError_t spmve_go(const DevMatrix &A, const SpmvEpi &e, Cycle *st, int check_done, cudaStream_t s, bool *launched)
{
    *launched = false;
    const EllLaunch &L = A.ell[sizeof(T) == 8 ? 1 : 0];
    const bool x2 = e.x2.base != nullptr;
    long long g = x2 ? L.blocks_x2 : L.blocks;
    const int nst = x2 ? L.nst_x2 : L.nst;
    if (g <= 0) return cudaSuccess;
    const void *vals = sizeof(T) == 8 ? (const void *)A.evals64 : (const void *)A.evals;
    SpmvEArgs q{A.n, vals, A.eidx, A.toff, A.etwin, A.ewmax, A.excap, nst, st, check_done, e};
    const long long etiles = ((long long)A.n + kThreads - 1) / kThreads;
    if (g > etiles) g = etiles;
    *launched = true;
    const size_t smem = (size_t)nst * spmve_stage_bytes(A.ewmax, x2, A.excap, (int)sizeof(T));
    const dim3 grid((unsigned)g), block(kSpmvThreads);
    const size_t wb = sizeof(T) == 4 ? A.l2_bytes : 0;  // the float32 blocks may stay in L2
    switch (A.lanes_per_row) {
    case 2:
        return x2 ? launch_pdl_l2(k_spmv_e<T, true, 2>, grid, block, smem, s, A.l2_base, wb, A.l2_hit, q)
                  : launch_pdl_l2(k_spmv_e<T, false, 2>, grid, block, smem, s, A.l2_base, wb, A.l2_hit, q);
    case 4:
        return x2 ? launch_pdl_l2(k_spmv_e<T, true, 4>, grid, block, smem, s, A.l2_base, wb, A.l2_hit, q)
                  : launch_pdl_l2(k_spmv_e<T, false, 4>, grid, block, smem, s, A.l2_base, wb, A.l2_hit, q);
    default:
        return x2 ? launch_pdl_l2(k_spmv_e<T, true, 1>, grid, block, smem, s, A.l2_base, wb, A.l2_hit, q)
                  : launch_pdl_l2(k_spmv_e<T, false, 1>, grid, block, smem, s, A.l2_base, wb, A.l2_hit, q);
    }
}

template <typename IDX>
cudaError_t spmvw_go(const DevMatrix &A, const IDX *cols, const SpmvEpi &e, Cycle *st, int check_done, cudaStream_t s,
                     bool *launched)
{
    *launched = false;
    if (!vec_aligned(e.x) || e.x2.base) return cudaSuccess;
    SpmvWArgs<IDX> p{};
    const VecRef *ops[4] = {&e.u0, &e.w0, &e.u1, &e.w1};
    p.nslot = 0;
    for (int q = 0; q < 4; ++q) {
        p.slot_of[q] = -1;
        if (!PPG_SPMV_STAGE_ROWS || !ops[q]->base || (q >= 2 && !e.out1.base)) continue;
        if (!vec_aligned(*ops[q])) return cudaSuccess;
        int found = -1;
        for (int t = 0; t < p.nslot; ++t)
            if (vec_same(p.slot[t], *ops[q])) found = t;
        if (found < 0) {
            if (p.nslot == kWSlots) return cudaSuccess;
            p.slot[p.nslot] = *ops[q];
            found = p.nslot++;
        }
        p.slot_of[q] = found;
    }
    const int R = A.rows_per_tile;
    const long long ntiles = ((long long)A.n + R - 1) / R;
    p.a = SpmvArgs<float, IDX>{A.n, A.rowptr, cols, A.vals32, R, A.lanes_per_row, A.cap32, st, check_done, e};
    p.lidx = A.lidx;
    p.twin = A.twin;
    long long g = A.spmvw_blocks32;
    if (g > ntiles) g = ntiles;
    if (g <= 0) return cudaSuccess;
    *launched = true;
    return launch_pdl(k_spmv_w<IDX>, dim3((unsigned)g), dim3(kSpmvThreads),
                      kSpmvStages * spmvw_stage_bytes(A.cap32, (int)sizeof(IDX)), s, p);
}

template <typename T, typename IDX>
cudaError_t sell_go(const DevMatrix &A, const T *vals, const IDX *cols, const SpmvEpi &e, Cycle *st, int check_done,
                    cudaStream_t s)
{
    SellArgs<T, IDX> a{A.n, A.nslices, A.sptr, cols, vals, st, check_done, e};
    static int per_sm = 0;
    if (per_sm == 0) {
        int nb = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_sell<T, IDX>, kSellWarps * 32, 0);
        if (err != cudaSuccess) return err;
        per_sm = nb > 0 ? nb : 1;
    }
    long long grid = (long long)per_sm * A.num_sms;
    const long long need = (A.nslices + kSellWarps - 1) / kSellWarps;
    if (grid > need) grid = need;
    return launch_pdl(k_spmv_sell<T, IDX>, dim3((unsigned)grid), dim3(kSellWarps * 32), 0, s, a);
}

// Dynamic shared memory limit (the widest tile and the largest windows) and the largest
// shared-memory carveout for the tile-ELL kernels: they alternate with the Gram-Schmidt passes, and
// consecutive launches should never wait for an SM to change its L1 / shared-memory split.
template <typename T, int G>
cudaError_t spmve_set_smem()
{
    const int sv = (int)sizeof(T);
    const size_t cap = (size_t)smem_optin() - 1024;
    size_t b1 = kSpmvStages * spmve_stage_bytes(kEllWidthMax, false, kXCap, sv);
    size_t b2 = kSpmvStages * spmve_stage_bytes(kEllWidthMax, true, kXCap, sv);
    if (b1 > cap) b1 = cap;
    if (b2 > cap) b2 = cap;
    cudaError_t e = cudaFuncSetAttribute(k_spmv_e<T, false, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spmv_e<T, true, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b2);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spmv_e<T, false, G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spmv_e<T, true, G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

template <typename T, typename IDX>
cudaError_t spmv_set_smem()
{
    cudaError_t e = cudaFuncSetAttribute(k_spmv<T, IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kSpmvStages * spmv_stage_bytes<T, IDX>(kSpmvCapMax)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(
            k_spmv2<T, IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)min(kSpmv2Stages * spmv_stage_bytes<T, IDX>(kSpmvCapMax), (size_t)smem_optin() - 1024));
    if (e == cudaSuccess && PPG_SPMV_CARVEOUT >= 0)
        e = cudaFuncSetAttribute(k_spmv<T, IDX>, cudaFuncAttributePreferredSharedMemoryCarveout, PPG_SPMV_CARVEOUT);
    if (e == cudaSuccess && sizeof(T) == 4)
        e = cudaFuncSetAttribute(k_spmv_w<IDX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kSpmvStages * spmvw_stage_bytes(kSpmvCapMax, (int)sizeof(IDX))));
    if (e == cudaSuccess) e = spmve_set_smem<T, 1>();
    if (e == cudaSuccess) e = spmve_set_smem<T, 2>();
    if (e == cudaSuccess) e = spmve_set_smem<T, 4>();
    return e;
}

template <typename IDX>
int spmvw_per_sm(int cap)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_w<IDX>, kSpmvThreads,
                                                  kSpmvStages * spmvw_stage_bytes(cap, (int)sizeof(IDX)));
    return nb > 0 ? nb : 0;
}
}  // namespace

cudaError_t launch_spmv(const DevMatrix &A, int prec, const SpmvEpi &e, Cycle *st, int check_done, cudaStream_t s)
{
    // staged storage: the tile-ELL blocks where they exist, else the windowed CSR kernel (float32)
    if (A.format == kFmtCsrStaged && A.evals && vec_aligned(e.x) && (!e.x2.base || vec_aligned(e.x2))) {
        bool launched = false;
        const cudaError_t err = prec == kF64 ? spmve_go<double>(A, e, st, check_done, s, &launched)
                                             : spmve_go<float>(A, e, st, check_done, s, &launched);
        if (launched || err != cudaSuccess) return err;
    }
    if (A.format == kFmtCsrStaged && prec == kF32 && A.twin) {
        bool launched = false;
        const cudaError_t err = A.coloff ? spmvw_go<short>(A, A.coloff, e, st, check_done, s, &launched)
                                         : spmvw_go<int>(A, A.colidx, e, st, check_done, s, &launched);
        if (launched || err != cudaSuccess) return err;
    }
    if (A.format == kFmtSell && A.nslices > 0) {
        if (prec == kF64) {
            if (A.soff) return sell_go<double, short>(A, A.svals64, A.soff, e, st, check_done, s);
            return sell_go<double, int>(A, A.svals64, A.scol, e, st, check_done, s);
        }
        if (A.soff) return sell_go<float, short>(A, A.svals32, A.soff, e, st, check_done, s);
        return sell_go<float, int>(A, A.svals32, A.scol, e, st, check_done, s);
    }
    if (prec == kF64) {
        if (A.coloff) return spmv_go<double, short>(A, A.vals64, A.coloff, A.cap64, A.spmv_blocks64, e, st, check_done, s);
        return spmv_go<double, int>(A, A.vals64, A.colidx, A.cap64, A.spmv_blocks64, e, st, check_done, s);
    }
    if (A.coloff) return spmv_go<float, short>(A, A.vals32, A.coloff, A.cap32, A.spmv_blocks32, e, st, check_done, s);
    return spmv_go<float, int>(A, A.vals32, A.colidx, A.cap32, A.spmv_blocks32, e, st, check_done, s);
}

cudaError_t launch_spmv2(const DevMatrix &A, int prec, const SpmvEpi &e1, const SpmvEpi &e2, Cycle *st, int check_done,
                         int *round_done, unsigned int *ticket, int *diag, const WaitCfg &wc, cudaStream_t s)
{
    if (prec == kF64) {
        if (A.coloff)
            return spmv2_go<double, short>(A, A.vals64, A.coloff, A.cap64, A.spmv2_blocks64, e1, e2, st, check_done,
                                           round_done, ticket, diag, wc, s);
        return spmv2_go<double, int>(A, A.vals64, A.colidx, A.cap64, A.spmv2_blocks64, e1, e2, st, check_done,
                                     round_done, ticket, diag, wc, s);
    }
    if (A.coloff)
        return spmv2_go<float, short>(A, A.vals32, A.coloff, A.cap32, A.spmv2_blocks32, e1, e2, st, check_done,
                                      round_done, ticket, diag, wc, s);
    return spmv2_go<float, int>(A, A.vals32, A.colidx, A.cap32, A.spmv2_blocks32, e1, e2, st, check_done, round_done,
                                ticket, diag, wc, s);
}

template <typename T, int G>
int spmve_per_sm_g(int wmax, bool x2, int xcap, int nst)
{
    int nb = 0;
    const size_t smem = (size_t)nst * spmve_stage_bytes(wmax, x2, xcap, (int)sizeof(T));
    if (smem > (size_t)smem_optin() - 1024) return 0;
    if (x2)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_e<T, true, G>, kSpmvThreads, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_e<T, false, G>, kSpmvThreads, smem);
    return nb > 0 ? nb : 0;
}

template <typename T>
int spmve_per_sm_t(int G, int wmax, bool x2, int xcap, int nst)
{
    if (G == 2) return spmve_per_sm_g<T, 2>(wmax, x2, xcap, nst);
    if (G == 4) return spmve_per_sm_g<T, 4>(wmax, x2, xcap, nst);
    return spmve_per_sm_g<T, 1>(wmax, x2, xcap, nst);
}

// Tile-ELL grid and pipeline depth for value type T: kSpmvStages stages when they fit, else fewer.
template <typename T>
void spmve_plan(DevMatrix *A, EllLaunch *L)
{
    for (int x2 = 0; x2 < 2; ++x2) {
        // the deepest pipeline that leaves at least one CTA per SM
        int nst = kSpmvStages, per = 0;
        for (; nst >= 2; --nst) {
            per = spmve_per_sm_t<T>(A->lanes_per_row, A->ewmax, x2 != 0, A->excap, nst);
            if (per > 0) break;
        }
        if (nst < 2) nst = 2;
        (x2 ? L->blocks_x2 : L->blocks) = per * A->num_sms;
        (x2 ? L->nst_x2 : L->nst) = nst;
    }
}

// Sets the dynamic shared memory limit (for the largest staging capacity, once) and returns
// the persistent grid sizes for this matrix's capacities and index format.
cudaError_t spmv_configure(DevMatrix *A)
{
    static bool done = false;
    if (!done) {
        cudaError_t err = spmv_set_smem<double, int>();
        if (err == cudaSuccess) err = spmv_set_smem<double, short>();
        if (err == cudaSuccess) err = spmv_set_smem<float, int>();
        if (err == cudaSuccess) err = spmv_set_smem<float, short>();
        if (err != cudaSuccess) return err;
        done = true;
    }
    A->ell[0] = EllLaunch{};
    A->ell[1] = EllLaunch{};
    if (A->evals) spmve_plan<float>(A, &A->ell[0]);
    if (A->evals64) spmve_plan<double>(A, &A->ell[1]);
    if (A->coloff) {
        A->spmv_blocks64 = spmv_per_sm<double, short>(A->cap64) * A->num_sms;
        A->spmv_blocks32 = spmv_per_sm<float, short>(A->cap32) * A->num_sms;
        A->spmv2_blocks64 = spmv2_per_sm<double, short>(A->cap64) * A->num_sms;
        A->spmv2_blocks32 = spmv2_per_sm<float, short>(A->cap32) * A->num_sms;
        A->spmvw_blocks32 = spmvw_per_sm<short>(A->cap32) * A->num_sms;
    } else {
        A->spmv_blocks64 = spmv_per_sm<double, int>(A->cap64) * A->num_sms;
        A->spmv_blocks32 = spmv_per_sm<float, int>(A->cap32) * A->num_sms;
        A->spmv2_blocks64 = spmv2_per_sm<double, int>(A->cap64) * A->num_sms;
        A->spmv2_blocks32 = spmv2_per_sm<float, int>(A->cap32) * A->num_sms;
        A->spmvw_blocks32 = spmvw_per_sm<int>(A->cap32) * A->num_sms;
    }
    return cudaSuccess;
}

// int16 column offsets (col - row) when every entry is within 32767 of its row; flag[0] = 1
// otherwise.  flag[1] receives the bandwidth max |col - row|.
__global__ void k_make_coloff(int n, const int *__restrict__ rowptr, const int *__restrict__ colidx, short *out,
                              int *flag)
{
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        int bw = 0;
        for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            const int d = colidx[k] - r;
            if (d < -32767 || d > 32767) atomicOr(flag, 1);
            out[k] = (short)d;
            bw = max(bw, abs(d));
        }
        if (bw > 0) atomicMax(flag + 1, bw);
    }
}

cudaError_t launch_make_coloff(int n, const int *rowptr, const int *colidx, short *out, int *flag, cudaStream_t s)
{
    int grid = (n + kThreads - 1) / kThreads;
    if (grid > 8192) grid = 8192;
    k_make_coloff<<<grid, kThreads, 0, s>>>(n, rowptr, colidx, out, flag);
    return cudaGetLastError();
}

int spmv_cap_max() { return kSpmvCapMax; }

int spmv_rows_per_thread() { return kSpmvRpt; }

// ---------------------------------------------------------------- matrix-free epilogue (last root of the product form)

template <typename T>
__global__ void k_axpy(int n, SpmvEpi e, Cycle *st, int check)
{
    pdl_wait();
    pdl_trigger();
    if (check == kSkipIfDone && st->cycle_done) return;
    if (check == kSkipIfNoCols && st->k == 0) return;
    T *o0 = resolve_ptr<T>(e.out0, st);
    const T *u0 = resolve_ptr<T>(e.u0, st);
    const T *w0 = resolve_ptr<T>(e.w0, st);
    const T b0 = (T)resolve(e.b0, st), c0 = (T)resolve(e.c0, st);
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        T v = T(0);
        if (u0) v = b0 * u0[r];
        if (w0) v = fma(c0, w0[r], v);
        o0[r] = v;
    }
}

cudaError_t launch_axpy(int n, int prec, const SpmvEpi &e, Cycle *st, int check, cudaStream_t s)
{
    int grid = (n + kThreads - 1) / kThreads;
    if (grid > 8192) grid = 8192;
    if (prec == kF64) return launch_pdl(k_axpy<double>, dim3(grid), dim3(kThreads), 0, s, n, e, st, check);
    return launch_pdl(k_axpy<float>, dim3(grid), dim3(kThreads), 0, s, n, e, st, check);
}

// ---------------------------------------------------------------- true residual and cycle start

// Starts a restart cycle from r = b - A x (float64), stored in basis column 0 as
// U_0 = r with sigma_0 = 1/||r||: tests convergence (relative residual, Section III),
// the iteration limit and finiteness, and resets the Givens right-hand side g = beta e_1.
// proj = 1 (the residual before a restart projection): the same tests, but a solve that goes on
// keeps the finished cycle's k, rotations and R for the projection; the residual after it starts
// the cycle.
__device__ void finish_residual(Cycle *st, double sumsq, int proj)
{
    const double beta = sqrt(sumsq);
    st->beta = beta;
    st->relres = beta / st->bnorm;
    st->nres += 1;
    if (!isfinite(beta)) {
        st->error |= kErrNonfinite;
        st->stop = 1;
    } else if (st->relres <= st->tol) {
        st->converged = 1;
        st->stop = 1;
    } else if (st->iters >= st->maxit) {
        st->stop = 1;
    }
    if (proj && !st->stop) return;
    st->k = 0;
    st->j = 0;
    st->breakdown = 0;
    if (st->stop) {
        st->cycle_done = 1;
        return;
    }
    st->cycle_done = 0;
    st->cycles += 1;
    st->sigma[0] = 1.0 / beta;
    for (int i = 0; i <= st->m; ++i) st->g[i] = 0.0;
    st->g[0] = beta;
}

template <typename Tout>
__global__ void __launch_bounds__(kThreads) k_residual(int n, const int *__restrict__ rowptr,
                                                       const int *__restrict__ colidx,
                                                       const double *__restrict__ vals, const double *__restrict__ b,
                                                       const double *__restrict__ x, Tout *__restrict__ out, Cycle *st,
                                                       double *partials, int proj)
{
    __shared__ double scratch[33];
    __shared__ int s_last;
    pdl_wait();
    pdl_trigger();
    if (st->stop) return;
    double nrm = 0.0;
    const int stride = gridDim.x * blockDim.x;
    // one warp handles 32 consecutive rows; each lane walks its own row
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        double acc = 0.0;
        const int k1 = rowptr[r + 1];
        for (int k = rowptr[r]; k < k1; ++k) acc = fma(vals[k], x[colidx[k]], acc);
        const double v = b[r] - acc;
        out[r] = (Tout)v;
        nrm = fma(v, v, nrm);
    }
    nrm = block_sum(nrm, scratch);
    if (threadIdx.x == 0) partials[blockIdx.x] = nrm;
    if (last_block_done(&st->ticket[0], &s_last)) {
        if (threadIdx.x < 32) {
            const double tot = reduce_partials(partials, gridDim.x, 0);
            if (threadIdx.x == 0) {
                finish_residual(st, tot, proj);
                st->ticket[0] = 0;
            }
        }
    }
}

cudaError_t launch_residual(const DevMatrix &A, int out_prec, const double *b, const double *x, void *out, Cycle *st,
                            double *partials, cudaStream_t s, int proj)
{
    const int grid = A.resid_blocks;
    if (out_prec == kF64)
        return launch_pdl(k_residual<double>, dim3(grid), dim3(kThreads), 0, s, A.n, A.rowptr, A.colidx, A.vals64, b,
                          x, (double *)out, st, partials, proj);
    return launch_pdl(k_residual<float>, dim3(grid), dim3(kThreads), 0, s, A.n, A.rowptr, A.colidx, A.vals64, b, x,
                      (float *)out, st, partials, proj);
}

// ||v||.  mode 0: st->bnorm = st->enorm = ||v|| (right-hand side).  mode 1: start an Arnoldi run from
// v: out = v (converted), beta = ||v||, sigma_0 = 1/beta, j = 0.  mode 2: st->enorm = ||v|| (the
// left-preconditioned right-hand side M^{-1} b).  mode 3: unless the solve has stopped, start a GMRES
// cycle from v (the left-preconditioned residual): out = v, beta, sigma_0, g = beta e_1, j = k = 0.
template <typename Tout>
__global__ void __launch_bounds__(kThreads) k_norm_start(int n, const double *__restrict__ v, Tout *__restrict__ out,
                                                         int mode, Cycle *st, double *partials)
{
    __shared__ double scratch[33];
    __shared__ int s_last;
    pdl_wait();
    pdl_trigger();
    if (mode == 3 && st->stop) return;
    double acc = 0.0;
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const double t = v[r];
        acc = fma(t, t, acc);
        if (out) out[r] = (Tout)t;
    }
    acc = block_sum(acc, scratch);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    if (last_block_done(&st->ticket[1], &s_last)) {
        if (threadIdx.x < 32) {
            const double tot = reduce_partials(partials, gridDim.x, 0);
            if (threadIdx.x == 0) {
                const double nv = sqrt(tot);
                if (mode == 0) {
                    st->bnorm = nv;
                    st->enorm = nv;
                } else if (mode == 2) {
                    st->enorm = nv;
                } else if (mode == 3) {
                    st->beta = nv;
                    st->sigma[0] = (nv > 0.0) ? 1.0 / nv : 0.0;
                    st->j = 0;
                    st->k = 0;
                    st->breakdown = 0;
                    st->cycles += 1;
                    st->cycle_done = (nv > 0.0 && isfinite(nv)) ? 0 : 1;
                    if (!isfinite(nv)) {
                        st->error |= kErrNonfinite;
                        st->stop = 1;
                    }
                    for (int i = 0; i <= st->m; ++i) st->g[i] = 0.0;
                    st->g[0] = nv;
                } else {
                    st->beta = nv;
                    st->bnorm = nv;
                    st->enorm = nv;
                    st->sigma[0] = (nv > 0.0) ? 1.0 / nv : 0.0;
                    st->j = 0;
                    st->k = 0;
                    st->cycle_done = (nv > 0.0 && isfinite(nv)) ? 0 : 1;
                    if (!isfinite(nv)) st->error |= kErrNonfinite;
                    st->breakdown = 0;
                    for (int i = 0; i <= st->m; ++i) st->g[i] = 0.0;
                    st->g[0] = nv;
                }
                st->ticket[1] = 0;
            }
        }
    }
}

cudaError_t launch_norm_start(int n, int out_prec, const double *v, void *out, int mode, Cycle *st, double *partials,
                              int nblk, cudaStream_t s)
{
    if (out_prec == kF64)
        return launch_pdl(k_norm_start<double>, dim3(nblk), dim3(kThreads), 0, s, n, v, (double *)out, mode, st,
                          partials);
    return launch_pdl(k_norm_start<float>, dim3(nblk), dim3(kThreads), 0, s, n, v, (float *)out, mode, st, partials);
}

// x += e (e in the inner precision), skipped when the cycle produced no columns.
template <typename Te>
__global__ void k_xupdate(int n, const Te *__restrict__ e, double *__restrict__ x, Cycle *st)
{
    pdl_wait();
    pdl_trigger();
    if (st->k == 0) return;
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) x[r] += (double)e[r];
}

cudaError_t launch_xupdate(int n, int prec, const void *e, double *x, Cycle *st, cudaStream_t s)
{
    int grid = (n + kThreads - 1) / kThreads;
    if (grid > 8192) grid = 8192;
    if (prec == kF64) return launch_pdl(k_xupdate<double>, dim3(grid), dim3(kThreads), 0, s, n, (const double *)e, x, st);
    return launch_pdl(k_xupdate<float>, dim3(grid), dim3(kThreads), 0, s, n, (const float *)e, x, st);
}

template <typename T>
__global__ void k_copy_in(int n, const T *__restrict__ src, T *__restrict__ dst)
{
    pdl_wait();
    pdl_trigger();
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) dst[r] = src[r];
}

cudaError_t launch_copy_in(int n, int prec, const void *src, void *dst, cudaStream_t s)
{
    int grid = (n + kThreads - 1) / kThreads;
    if (grid > 8192) grid = 8192;
    if (prec == kF64)
        return launch_pdl(k_copy_in<double>, dim3(grid), dim3(kThreads), 0, s, n, (const double *)src, (double *)dst);
    return launch_pdl(k_copy_in<float>, dim3(grid), dim3(kThreads), 0, s, n, (const float *)src, (float *)dst);
}

// ---------------------------------------------------------------- SplitMix64 (Steele, Lea, Flood 2014)

__device__ __forceinline__ unsigned long long splitmix_mix(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_fill_uniform(double *out, long long n, unsigned long long seed)
{
    const unsigned long long base = splitmix_mix(seed);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long z = splitmix_mix(base + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull);
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        out[i] = -1.0 + 2.0 * u;
    }
}

cudaError_t launch_fill_uniform(double *out, long long n, unsigned long long seed, cudaStream_t s)
{
    k_fill_uniform<<<2048, kThreads, 0, s>>>(out, n, seed);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- adjoint helpers

// out_k = alpha * u_{row(k)} * v_{col(k)} over the CSR pattern (dL/dvals = -lambda_i x_j).
__global__ void k_csr_outer(int n, const int *__restrict__ rowptr, const int *__restrict__ colidx,
                            const double *__restrict__ u, const double *__restrict__ v, double alpha,
                            double *__restrict__ out)
{
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const double ur = alpha * u[r];
        for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) out[k] = ur * v[colidx[k]];
    }
}

cudaError_t launch_csr_outer(const DevMatrix &A, const double *u, const double *v, double alpha, double *out,
                             cudaStream_t s)
{
    int grid = (A.n + kThreads - 1) / kThreads;
    if (grid > 8192) grid = 8192;
    k_csr_outer<<<grid, kThreads, 0, s>>>(A.n, A.rowptr, A.colidx, u, v, alpha, out);
    return cudaGetLastError();
}

// Transpose by counting sort: column counts (atomics), an exclusive scan (single CTA,
// chunked), a scatter that walks each source row in order, and a per-row sort that makes
// the order within each row of A^T ascending and independent of atomic timing.
__global__ void k_count_cols(long long nnz, const int *__restrict__ colidx, int *counts)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += stride)
        atomicAdd(&counts[colidx[k] + 1], 1);
}

// in-place inclusive scan of counts[0..n] by one CTA (counts[0] = 0 gives exclusive offsets)
__global__ void k_scan_single(int n1, int *data)
{
    __shared__ int s_carry;
    __shared__ int s_warp[32];
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < n1; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int v = (i < n1) ? data[i] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) s_warp[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int w = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int add = s_carry + (wid > 0 ? s_warp[wid - 1] : 0);
        if (i < n1) data[i] = v + add;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = add + v;
        __syncthreads();
    }
}

__global__ void k_scatter_t(int n, const int *__restrict__ rowptr, const int *__restrict__ colidx,
                            const double *__restrict__ vals, const int *__restrict__ rpT, int *fill, int *ciT,
                            double *vaT)
{
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            const int c = colidx[k];
            const int dst = rpT[c] + atomicAdd(&fill[c], 1);
            ciT[dst] = r;
            vaT[dst] = vals[k];
        }
    }
}

__global__ void k_sort_rows(int n, const int *__restrict__ rpT, int *ciT, double *vaT)
{
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const int s = rpT[r], e = rpT[r + 1];
        for (int i = s + 1; i < e; ++i) {  // insertion sort: rows are short
            const int c = ciT[i];
            const double v = vaT[i];
            int j = i - 1;
            while (j >= s && ciT[j] > c) {
                ciT[j + 1] = ciT[j];
                vaT[j + 1] = vaT[j];
                --j;
            }
            ciT[j + 1] = c;
            vaT[j + 1] = v;
        }
    }
}

cudaError_t launch_transpose(const DevMatrix &A, int *rpT, int *ciT, double *vaT, int *work, cudaStream_t s)
{
    cudaError_t err = cudaMemsetAsync(rpT, 0, sizeof(int) * (A.n + 1), s);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(work, 0, sizeof(int) * A.n, s);
    if (err != cudaSuccess) return err;
    k_count_cols<<<1024, kThreads, 0, s>>>(A.nnz, A.colidx, rpT);
    k_scan_single<<<1, 1024, 0, s>>>(A.n + 1, rpT);
    int grid = (A.n + kThreads - 1) / kThreads;
    if (grid > 8192) grid = 8192;
    k_scatter_t<<<grid, kThreads, 0, s>>>(A.n, A.rowptr, A.colidx, A.vals64, rpT, work, ciT, vaT);
    k_sort_rows<<<grid, kThreads, 0, s>>>(A.n, rpT, ciT, vaT);
    return cudaGetLastError();
}

}  // namespace ppg
