// ppg_common.cuh -- shared device definitions of the GB300 PP-GMRES library.
//
// Device-resident solver state, the scalar/vector operand descriptors that let a
// captured kernel sequence follow the iteration index kept on the device, and
// inline-PTX helpers for mbarriers and TMA bulk copies (sm_100+ / sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ppg {

constexpr int kThreads = 256;      // threads per CTA of every streaming kernel
constexpr int kKmax = 128;         // largest Krylov basis (restart + 1)
constexpr int kSmallMax = 64;      // largest dense eigen/Cholesky problem (degree + 1 + 1)
constexpr int kLdPad = 1024;       // internal vectors are padded to a multiple of this many entries

// error bits kept in Cycle::error
enum : int {
    kErrNone = 0,
    kErrTimeout = 1,
    kErrNonfinite = 2,
};

// Device-resident state of one Arnoldi / GMRES(m) run.  Every kernel of an
// iteration reads the iteration index j from here, so one captured sequence
// of launches serves every iteration of every cycle.
struct Cycle {
    int j;           // next basis column to build (iteration index within the cycle)
    int k;           // columns of the finished cycle to combine (0 = nothing to update)
    int cycle_done;  // 1: the remaining iteration kernels of this cycle return at once
    int converged;   // true residual met the tolerance
    int breakdown;   // this cycle ended by a (lucky) breakdown
    int error;       // kErr* bits
    int m;           // restart length
    int mode;        // 0: GMRES (Givens, tests); 1: plain Arnoldi (no tests, stop at m)
    int stop;        // 1: solve finished (converged, maxit or error)
    int n_breakdowns;
    int *prog;       // host-mapped progress word: (cycle_done << 16) | j after each iteration, or null
    long long iters;    // iterations over all cycles
    long long maxit;
    long long cycles;
    long long nres;     // float64 true residuals computed (b - A x)
    long long nproj;    // restart projections done (flexible float32 solves)
    long long nblocks;  // s-step blocks finished (each: three global reductions)
    long long nnewton;  // s-step Newton vectors built (each: one application of A p(A))
    double bnorm;       // ||b||
    double enorm;       // the norm the in-cycle estimate is relative to: ||b||, or ||M^{-1} b|| with ILU(0)
                        // on the left (the residual left-preconditioned GMRES minimises)
    double tol;         // relative tolerance
    double inner_rtol;  // cycle ends when |g_{j+1}| <= inner_rtol * beta (0: off)
    double beta;        // ||r|| at the start of the cycle
    double relres;      // last true relative residual
    double est;         // last estimate |g_{j+1}| / ||b||
    double w0sq;        // ||w||^2 before orthogonalisation (breakdown test)
    double sigma[kKmax + 1];  // stored basis column c equals v_c / sigma_c  (v_c = sigma_c * U_c)
    double h1[kKmax + 1];     // first Gram-Schmidt pass coefficients of the current column
    double h2[kKmax + 1];     // second pass
    double coef[kKmax + 1];   // coefficients the next update kernel multiplies U columns by
    double H[(kKmax + 1) * kKmax];  // Hessenberg matrix as built (column-major, ld kKmax + 1)
    double R[(kKmax + 1) * kKmax];  // rotated copy (upper triangular part used)
    double cs[kKmax], sn[kKmax];
    double g[kKmax + 1];
    double y[kKmax];
    unsigned int ticket[8];  // last-CTA-done counters, one per kernel kind
};

constexpr int kLdH = kKmax + 1;

// A scalar operand resolved on the device: imm * p[idx] * q[qidx], where a null pointer
// contributes 1 and an index may follow the iteration index j kept in Cycle.
struct Scalar {
    double imm;
    const double *p;
    int p_off;     // index into p
    int p_follow;  // 1: index is Cycle::j + p_off
    const double *q;
    int q_off;
    int q_follow;
};

// A vector operand: base + column * ld elements, the column optionally following Cycle::j.
struct VecRef {
    const void *base;
    long long ld;
    int col;     // fixed column, or offset from j when follow = 1
    int follow;
};

__host__ __device__ inline Scalar scalar_imm(double v) { return Scalar{v, nullptr, 0, 0, nullptr, 0, 0}; }

#ifdef __CUDACC__
__device__ __forceinline__ double resolve(const Scalar &s, const Cycle *st)
{
    double v = s.imm;
    if (s.p) v *= s.p[s.p_follow ? st->j + s.p_off : s.p_off];
    if (s.q) v *= s.q[s.q_follow ? st->j + s.q_off : s.q_off];
    return v;
}

template <typename T>
__device__ __forceinline__ T *resolve_ptr(const VecRef &v, const Cycle *st)
{
    if (!v.base) return nullptr;
    long long c = v.follow ? (long long)st->j + v.col : (long long)v.col;
    return (T *)v.base + c * v.ld;
}

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// adds to the bytes the current phase waits for, without arriving
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// TMA bulk copy global -> shared (the CTA's own shared memory), completion counted on bar.
// Requires 16-byte aligned src and dst and a byte count that is a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// TMA tiled copy of one box of a 2-D tensor map (global -> this CTA's shared memory) at element
// coordinates (x innermost, y), completion counted on bar.  tmap: the generic address of a
// __grid_constant__ CUtensorMap kernel parameter.  x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// The same for a 3-D tensor map at (x, y, z), x innermost.
__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the barrier phase with a time limit (about one second).  Returns false on
// timeout; the caller records kErrTimeout and leaves after a second bounded wait.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    for (unsigned int spins = 1;; ++spins) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spins & 63u) == 0 && global_timer_ns() - t0 > limit_ns) return false;
    }
}

constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

// A bounded wait ran out: record it and end the solve, so that the kernels still queued for the
// cycle return at once (the host then reports PPG_ERR_TIMEOUT).
__device__ __forceinline__ void timeout_stop(Cycle *st)
{
    atomicOr(&st->error, kErrTimeout);
    st->stop = 1;
    st->cycle_done = 1;
    st->k = 0;
}

// Named barrier `id` over `nthreads` threads that also ORs a predicate across them.
__device__ __forceinline__ bool bar_any(int id, int nthreads, bool v)
{
    unsigned int r;
    asm volatile(
        "{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.or.pred q, %2, %3, p; selp.u32 %0, 1, 0, q; }"
        : "=r"(r)
        : "r"((unsigned int)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Programmatic dependent launch.  Kernels of the solve path are launched so that they may
// start while the previous kernel of the stream drains.  Each waits for its predecessor's
// completion and memory (pdl_wait) before it reads anything the predecessor may have written,
// and only then lets its own dependents start (pdl_trigger).  So when a kernel starts, every
// kernel launched before its predecessor has completed: data those wrote (and constant data)
// may be read before the wait.  Both are no-ops for ordinary launches.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// A float32 value carried as an unevaluated sum hi + lo.  Adding two of them with Knuth's
// two-sum keeps the rounding error of the high parts, so a warp tree of such additions is
// accurate to about float64 level using float32 arithmetic only (float64 instructions are
// scarce on this GPU: a warp-wide float64 add occupies the FP64 pipe ~64 times longer).
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const float s = a.hi + b.hi;
    const float bv = s - a.hi;
    const float err = (a.hi - (s - bv)) + (b.hi - bv);
    const float lo = a.lo + b.lo + err;
    const float hi = s + lo;
    return F2{hi, lo - (hi - s)};
}

// warp tree of compensated float32 sums (lane 0's result is the one used)
__device__ __forceinline__ F2 warp_tree_f2(F2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const F2 w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = f2_add(v, w);
    }
    return v;
}

// the same, converted to float64 once
__device__ __forceinline__ double warp_sum_f2(F2 v)
{
    v = warp_tree_f2(v);
    return (double)v.hi + (double)v.lo;
}

// Sum over the CTA in a fixed order (warp trees, then warp 0 over the warp sums).
// Every thread must call it; the result is valid in every thread.
__device__ __forceinline__ double block_sum(double v, double *scratch /* >= 33 doubles */)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double t = (lane < (int)(blockDim.x >> 5)) ? scratch[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) scratch[32] = t;
    }
    __syncthreads();
    return scratch[32];
}

// The "last CTA done" ticket: every CTA calls this after writing its partial results;
// exactly one CTA (the last to arrive) gets true.  Includes the fences that make the
// other CTAs' partials visible to it.
__device__ __forceinline__ bool last_block_done(unsigned int *ticket, int *s_flag)
{
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int prev = atomicAdd(ticket, 1u);
        *s_flag = (prev == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (*s_flag) {
        __threadfence();
        return true;
    }
    return false;
}

// Sum of a compensated float32 value over the CTA, kept as a pair: warp trees, then thread 0 adds
// the warp totals in warp order.  Every thread must call it; the result is valid in every thread.
__device__ __forceinline__ F2 block_sum_f2_pair(F2 v, F2 *scratch /* >= 33 */)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_tree_f2(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        F2 t = scratch[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) t = f2_add(t, scratch[q]);
        scratch[32] = t;
    }
    __syncthreads();
    return scratch[32];
}

// Deterministic sums of per-CTA partial slots slot[c * ld + b], b < nblk, for one column c by one
// warp, with many loads in flight: lane l takes the slot pairs (2q, 2q + 1) for q = l + 32 u in
// increasing u, kSlotLoads 16-byte loads at a time (one round for up to 512 CTAs), then a fixed
// shuffle tree.  ld is even and the
// slots are 16-byte aligned.  Float64 slots, or compensated float32 pairs (F2) in 8-byte slots.
constexpr int kSlotLoads = 8;

__device__ __forceinline__ double reduce_slots_f64(const double *slot, int ld, int nblk, int c)
{
    const int lane = threadIdx.x & 31;
    const double2 *p = reinterpret_cast<const double2 *>(slot + (long long)c * ld);
    const int npair = (nblk + 1) >> 1;
    double s = 0.0;
    for (int q0 = lane; q0 < npair; q0 += 32 * kSlotLoads) {
        double2 v[kSlotLoads];
#pragma unroll
        for (int u = 0; u < kSlotLoads; ++u) {
            const int q = q0 + 32 * u;
            v[u] = q < npair ? __ldcg(p + q) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < kSlotLoads; ++u) {
            const int q = q0 + 32 * u;
            if (q < npair) {
                s += v[u].x;
                if (2 * q + 1 < nblk) s += v[u].y;
            }
        }
    }
    return warp_sum(s);
}

__device__ __forceinline__ double reduce_slots_f2(const double *slot, int ld, int nblk, int c)
{
    const int lane = threadIdx.x & 31;
    const float4 *p = reinterpret_cast<const float4 *>(slot + (long long)c * ld);
    const int npair = (nblk + 1) >> 1;
    F2 s{0.f, 0.f};
    for (int q0 = lane; q0 < npair; q0 += 32 * kSlotLoads) {
        float4 v[kSlotLoads];
#pragma unroll
        for (int u = 0; u < kSlotLoads; ++u) {
            const int q = q0 + 32 * u;
            v[u] = q < npair ? __ldcg(p + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kSlotLoads; ++u) {
            const int q = q0 + 32 * u;
            if (q < npair) {
                s = f2_add(s, F2{v[u].x, v[u].y});
                if (2 * q + 1 < nblk) s = f2_add(s, F2{v[u].z, v[u].w});
            }
        }
    }
    return warp_sum_f2(s);
}

// Deterministic reduction of partials[c * nblk + b] over b for one column c by one warp:
// lane l adds b = l, l + 32, ... in order, then a fixed shuffle tree.
__device__ __forceinline__ double reduce_partials(const double *partials, int nblk, int c)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    const double *p = partials + (long long)c * nblk;
    for (int b = lane; b < nblk; b += 32) s += __ldcg(p + b);
    return warp_sum(s);
}
#endif  // __CUDACC__

}  // namespace ppg
