// ppg_ilu.cu -- ILU(0) on the left of the polynomial preconditioner (Loe, Thornquist, Boman,
// Section VI: M^{-1} A p(M^{-1} A) y = M^{-1} b, x = p(M^{-1} A) y, with M = L U the incomplete LU
// factorisation without fill).
//
// Factorisation: row by row with the textbook no-fill rule -- for each entry k < i of row i in
// increasing column order, l_ik = a_ik / u_kk, then every later entry of row i that row k also
// has is reduced by l_ik u_kj.  Row i needs the rows k it references to be final, so rows are
// grouped in levels (level(i) = 1 + max level of those rows, computed on the host from the
// pattern) and each level is one launch, one thread per row.  Products and differences are rounded
// separately, as in a plain IEEE evaluation of the same loops.
//
// Triangular solves: one cooperative launch (every CTA resident) where each group of lanes takes a row
// from the level-sorted list in order, waits -- with a time limit -- for the rows its row depends on,
// forms the row and publishes it.  The solution vector is its own ready mark: a fill launch sets every
// entry to a signalling-NaN pattern that no arithmetic produces, a row's result replaces it with one
// store, and a waiting lane polls the entry itself, so the value arrives with the load that sees it
// ready (one L2 round trip per dependency instead of a flag and then the value).  A row's
// dependencies are earlier in the list and every warp walks the list in order, so the earliest
// unfinished row can always proceed; no level barriers.
#include <cuda_runtime.h>

#include <algorithm>

#include "ppg_internal.h"

namespace ppg {

__global__ void __launch_bounds__(kThreads) k_ilu0_level(const int *__restrict__ rows, int count,
                                                          const int *__restrict__ rp, const int *__restrict__ ci,
                                                          const int *__restrict__ diag, double *lu)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    const int i = rows[q];
    const int e1 = rp[i + 1];
    for (int t = rp[i]; t < e1; ++t) {
        const int k = ci[t];
        if (k >= i) break;
        const double lik = lu[t] / lu[diag[k]];
        lu[t] = lik;
        // row k's entries after its diagonal against row i's entries after t (both ascending)
        int p = t + 1;
        for (int s = diag[k] + 1; s < rp[k + 1] && p < e1; ++s) {
            const int j = ci[s];
            while (p < e1 && ci[p] < j) ++p;
            if (p < e1 && ci[p] == j) lu[p] = __dsub_rn(lu[p], __dmul_rn(lik, lu[s]));
        }
    }
}

cudaError_t launch_ilu0_level(const int *rows, int count, const int *rp, const int *ci, const int *diag, double *lu,
                              cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_ilu0_level<<<(count + kThreads - 1) / kThreads, kThreads, 0, s>>>(rows, count, rp, ci, diag, lu);
    return cudaGetLastError();
}

__global__ void k_ilu_cast(const double *__restrict__ in, float *__restrict__ out, long long count)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        out[q] = (float)in[q];
}

// Bit patterns of a pending entry (a signalling NaN: arithmetic only returns quiet NaNs) and of the
// quiet NaN stored in its place should a result ever have the pending pattern.
template <typename T>
struct IluBits;
template <>
struct IluBits<float> {
    using U = unsigned int;
    static constexpr U kPending = 0x7FA11CE5u;
    static constexpr U kQuietNaN = 0x7FFFFFFFu;
    static __device__ __forceinline__ U bits(float v) { return __float_as_uint(v); }
    static __device__ __forceinline__ float value(U b) { return __uint_as_float(b); }
};
template <>
struct IluBits<double> {
    using U = unsigned long long;
    static constexpr U kPending = 0x7FF4A11CE5A11CE5ull;
    static constexpr U kQuietNaN = 0x7FFFFFFFFFFFFFFFull;
    static __device__ __forceinline__ U bits(double v) { return (U)__double_as_longlong(v); }
    static __device__ __forceinline__ double value(U b) { return __longlong_as_double((long long)b); }
};

__device__ __forceinline__ unsigned int ilu_ld(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ilu_ld(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void ilu_st(unsigned int *p, unsigned int v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void ilu_st(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename T>
__global__ void k_ilu_pending(typename IluBits<T>::U *y, long long n)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        y[q] = IluBits<T>::kPending;
}

// G lanes per row (the row walked in passes of G entries): a warp takes 32 / G consecutive rows of
// the list per step.  Each group of G lanes waits, reduces and publishes on its
// own (shuffles over the group's lanes only), so a row whose dependency sits in another group of the
// same warp never waits for that group to finish its step.
template <typename T, bool LOWER, int G>
__global__ void __launch_bounds__(kThreads) k_ilu_solve(IluSolveArgs a)
{
    Cycle *st = a.st;
    if ((a.check == kSkipIfDone && st->cycle_done) || (a.check == kSkipIfNoCols && st->k == 0) ||
        (a.check == kSkipIfStop && st->stop))
        return;
    constexpr int R = 32 / G;
    using B = IluBits<T>;
    using U = typename B::U;
    const T *lu = static_cast<const T *>(a.lu);
    const T *rd = static_cast<const T *>(a.rdiag);
    const T *xin = resolve_ptr<T>(a.x, st);
    U *yb = static_cast<U *>(a.y);
    T *o0 = resolve_ptr<T>(a.e.out0, st);
    const T *u0 = resolve_ptr<T>(a.e.u0, st);
    const T *w0 = resolve_ptr<T>(a.e.w0, st);
    T *o1 = resolve_ptr<T>(a.e.out1, st);
    const T *u1 = resolve_ptr<T>(a.e.u1, st);
    const T *w1 = resolve_ptr<T>(a.e.w1, st);
    const T ca0 = (T)resolve(a.e.a0, st), cb0 = (T)resolve(a.e.b0, st), cc0 = (T)resolve(a.e.c0, st);
    const T ca1 = (T)resolve(a.e.a1, st), cb1 = (T)resolve(a.e.b1, st), cc1 = (T)resolve(a.e.c1, st);
    const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (sub * G));
    const long long W = (long long)gridDim.x * (blockDim.x >> 5);
    const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // the next row's list entry, bounds and pivot reciprocal are loaded a step ahead (they do not depend
    // on other rows)
    int ni = 0, ne0 = 0, ne1 = 0;
    T nrd = T(0);
    if (wg * R + sub < a.n) {
        ni = a.order[wg * R + sub];
        ne0 = a.rp[ni];
        ne1 = a.rp[ni + 1];
        if (!LOWER) nrd = rd[ni];
    }
    for (long long q0 = wg * R; q0 < a.n; q0 += W * R) {
        const long long q = q0 + sub;
        bool ok = true;
        const int i = ni, e0 = ne0, e1 = ne1;
        const T rdi = nrd;
        if (q + W * R < a.n) {
            ni = a.order[q + W * R];
            ne0 = a.rp[ni];
            ne1 = a.rp[ni + 1];
            if (!LOWER) nrd = rd[ni];
        }
        if (q < a.n) {
            T sum = T(0);
            for (int e = e0 + gl; e < e1; e += G) {
                const int k = a.ci[e];
                if (LOWER ? (k < i) : (k > i)) {
                    U v = ilu_ld(yb + k);
                    if (v == B::kPending || a.unreachable) {
                        const unsigned long long t0 = global_timer_ns();
                        for (unsigned int spins = 1; (v = ilu_ld(yb + k)) == B::kPending || a.unreachable; ++spins) {
                            if ((spins & 63u) == 0 && global_timer_ns() - t0 > a.wait_ns) {
                                ok = false;
                                break;
                            }
                        }
                    }
                    if (ok) sum = fma(lu[e], B::value(v), sum);
                }
            }
            ok = __all_sync(gmask, ok);
            // lanes at or above the longest row hold zero: reduce over the first a.red lanes only
            for (int o = min(a.red, G) >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(gmask, sum, o);
            if (ok && gl == 0) {
                const T yi = LOWER ? xin[i] - sum : (xin[i] - sum) * rdi;
                if (o0) {
                    T v = ca0 * yi;
                    if (u0) v = fma(cb0, u0[i], v);
                    if (w0) v = fma(cc0, w0[i], v);
                    o0[i] = v;
                }
                if (o1) {
                    T v = ca1 * yi;
                    if (u1) v = fma(cb1, u1[i], v);
                    if (w1) v = fma(cc1, w1[i], v);
                    o1[i] = v;
                }
                const U ub = B::bits(yi);
                ilu_st(yb + i, ub == B::kPending ? B::kQuietNaN : ub);  // the value is the row's ready mark
            }
        }
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) {
                timeout_stop(st);
                atomicCAS(a.abort, 0, i + 1);
            }
            return;
        }
        if ((q0 & 63) == 0 && *(volatile int *)a.abort) return;
    }
}

template <typename T, bool LOWER, int G>
cudaError_t ilu_solve_go(const IluSolveArgs &a, int num_sms, cudaStream_t s)
{
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ilu_solve<T, LOWER, G>, kThreads, 0);
    long long g = (long long)(per > 0 ? per : 1) * num_sms;  // every CTA resident (cooperative launch)
    const long long rows_per_cta = (kThreads / 32) * (32 / G);
    const long long need = ((long long)a.n + rows_per_cta - 1) / rows_per_cta;
    if (g > need) g = need;
    if (g < 1) g = 1;
    return launch_coop(k_ilu_solve<T, LOWER, G>, dim3((unsigned)g), dim3(kThreads), 0, s, a);
}

// One warp per row: measured on the 128^3 stencil (one M^{-1} A x, float32), 2.2 ms against 5.1 ms with
// groups of eight lanes taking four rows per warp; a pause between polls changed nothing, and fewer
// CTAs per SM were slower.
cudaError_t launch_ilu_solve(int prec, bool lower, const IluSolveArgs &a, int num_sms, cudaStream_t s)
{
    const unsigned fill_grid = (unsigned)std::min<long long>(((long long)a.n + kThreads - 1) / kThreads, 8LL * num_sms);
    if (prec == kF64)
        k_ilu_pending<double><<<fill_grid, kThreads, 0, s>>>(static_cast<IluBits<double>::U *>(a.y), a.n);
    else
        k_ilu_pending<float><<<fill_grid, kThreads, 0, s>>>(static_cast<IluBits<float>::U *>(a.y), a.n);
    const cudaError_t fe = cudaGetLastError();
    if (fe != cudaSuccess) return fe;
    if (prec == kF64)
        return lower ? ilu_solve_go<double, true, 32>(a, num_sms, s) : ilu_solve_go<double, false, 32>(a, num_sms, s);
    return lower ? ilu_solve_go<float, true, 32>(a, num_sms, s) : ilu_solve_go<float, false, 32>(a, num_sms, s);
}

cudaError_t launch_ilu_cast(const double *in, float *out, long long count, cudaStream_t s)
{
    k_ilu_cast<<<1024, kThreads, 0, s>>>(in, out, count);
    return cudaGetLastError();
}

}  // namespace ppg
