// ppg_cycle.cuh -- device routines shared by the kernels that finish a GMRES step on the device
// (the Gram-Schmidt passes and the s-step block finalisation): the host-mapped progress word and
// the cycle-end back substitution y = R^{-1} g.
#pragma once

#include "ppg_common.cuh"

namespace ppg {

// Publishes the iteration count and the end-of-cycle flag to the host-mapped progress word, so
// that the host stops enqueueing a cycle's iterations once it has ended.  The host uses the word
// only to pace its launches (anything it acts on is read after the stream has synchronised), so
// the store needs no fence.
static __device__ __forceinline__ void publish_progress(const Cycle *st, int cycle_done, int j)
{
    if (st->prog) *(volatile int *)st->prog = (cycle_done << 16) | j;
}

// y = R^{-1} g[0..k-1] with the cycle's triangle R (st->R) and right-hand side st->g, by the whole
// CTA: R staged in shared memory when it fits, then column-oriented back substitution by warp 0
// (y_i = g_i / R_ii, then g_q -= R_qi y_i for q < i in parallel).  Writes y and the combination
// coefficients coef = -y .* sigma.  sh: shared scratch of sh_bytes, free for this call.
static __device__ __noinline__ void cta_solve_r(Cycle *st, int k, double *sh, size_t sh_bytes)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    double *g = sh;            // k values
    double *Rs = sh + k;       // k x k, column-major, ld k
    const bool staged = (size_t)(k + k * k) * sizeof(double) <= sh_bytes;
    for (int i = tid; i < k; i += nt) g[i] = st->g[i];
    if (staged)
        for (int e = tid; e < k * k; e += nt) {
            const int q = e / k, i = e - q * k;
            Rs[e] = i <= q ? st->R[(long long)q * kLdH + i] : 0.0;
        }
    __syncthreads();
    if (tid < 32) {
        for (int i = k - 1; i >= 0; --i) {
            const double *Ri = staged ? Rs + (long long)i * k : st->R + (long long)i * kLdH;
            const double yi = g[i] / Ri[i];
            __syncwarp();
            for (int q = tid; q < i; q += 32) g[q] -= Ri[q] * yi;
            if (tid == 0) g[i] = yi;
            __syncwarp();
        }
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt) {
        const double y = g[c];
        st->y[c] = y;
        st->coef[c] = -y * st->sigma[c];
    }
    __syncthreads();
}


}  // namespace ppg
