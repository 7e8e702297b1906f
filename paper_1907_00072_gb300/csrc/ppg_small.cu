// ppg_small.cu -- single-thread device kernels for the polynomial's roots.
//
// The minimum-residual polynomial p of degree d (Loe, Thornquist, Boman, Section II)
// satisfies 1 - z p(z) = prod_i (1 - z / theta_i), where theta_1..theta_{d+1} are the
// harmonic Ritz values of the (d+1)-step Arnoldi run from v0.  Applying p(A) through
// these roots, in Leja order, avoids the power basis whose Gram matrix stops being
// positive definite near degree 10 (Section IV).  This file computes the roots on the
// device from the run's Hessenberg matrix and the per-step coefficients of the
// product-form application:
//   real theta:        y += w / theta,                 w -= (A w) / theta
//   pair a +- ib:      t = A w; y += (2a w - t) / q;   w -= (2a t - A t) / q,  q = a^2 + b^2
#include <cuda_runtime.h>

#include "ppg_dense.cuh"
#include "ppg_internal.h"

namespace ppg {

// roots_out: 2k doubles (re, im) in application order.  table_out: 2k doubles, per root
// position: real -> (1/theta, 0); first of a pair -> (2a/q, 1/q); second of a pair -> (0, 0).
// status_out[0]: 0 ok, 1 QR did not converge, 2 singular H_k, 3 zero or non-finite root.
__global__ void __launch_bounds__(32) k_roots(const Cycle *st, int k, double *roots_out, double *table_out,
                                              int *status_out)
{
    __shared__ double work[kSmallMax * kSmallMax + kSmallMax];
    __shared__ double wr[kSmallMax], wi[kSmallMax], score[kSmallMax];
    __shared__ int order[kSmallMax], used[kSmallMax];
    const int lane = threadIdx.x;
    int status = harmonic_ritz(k, st->H, kLdH, wr, wi, work, lane, 32);
    if (status == 0) leja_order(k, wr, wi, order, used, score, lane, 32);
    __syncwarp();
    if (lane != 0) return;
    if (status == 0) {
        for (int p = 0; p < k; ++p) {
            const double re = wr[order[p]], im = wi[order[p]];
            roots_out[2 * p] = re;
            roots_out[2 * p + 1] = im;
            if (!isfinite(re) || !isfinite(im) || (re == 0.0 && im == 0.0)) status = 3;
        }
        for (int p = 0; p < k; ++p) {
            const double re = roots_out[2 * p], im = roots_out[2 * p + 1];
            if (im == 0.0) {
                table_out[2 * p] = 1.0 / re;
                table_out[2 * p + 1] = 0.0;
            } else if (im > 0.0) {
                const double q = re * re + im * im;
                table_out[2 * p] = 2.0 * re / q;
                table_out[2 * p + 1] = 1.0 / q;
            } else {
                table_out[2 * p] = 0.0;
                table_out[2 * p + 1] = 0.0;
            }
        }
    }
    status_out[0] = status;
}

// Per-step coefficients for roots given by the caller (already in application order).
__global__ void k_root_table(int k, const double *roots, double *table_out, int *status_out)
{
    if (threadIdx.x != 0) return;
    int status = 0;
    for (int p = 0; p < k; ++p) {
        const double re = roots[2 * p], im = roots[2 * p + 1];
        if (!isfinite(re) || !isfinite(im) || (re == 0.0 && im == 0.0)) status = 3;
        if (im == 0.0) {
            table_out[2 * p] = 1.0 / re;
            table_out[2 * p + 1] = 0.0;
        } else if (im > 0.0) {
            const double q = re * re + im * im;
            table_out[2 * p] = 2.0 * re / q;
            table_out[2 * p + 1] = 1.0 / q;
        } else {
            table_out[2 * p] = 0.0;
            table_out[2 * p + 1] = 0.0;
        }
    }
    status_out[0] = status;
}

cudaError_t launch_root_table(int k, const double *roots, double *table_out, int *status_out, cudaStream_t s)
{
    k_root_table<<<1, 32, 0, s>>>(k, roots, table_out, status_out);
    return cudaGetLastError();
}

cudaError_t launch_roots(const Cycle *st, int k, double *roots_out, double *table_out, int *status_out,
                         cudaStream_t s)
{
    k_roots<<<1, 32, 0, s>>>(st, k, roots_out, table_out, status_out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(32) k_hess_eigs(int k, const double *H, int ld, double *wr, double *wi,
                                                  int *status_out)
{
    __shared__ double m[kSmallMax * kSmallMax];
    __shared__ double r[kSmallMax], im[kSmallMax];
    const int lane = threadIdx.x;
    for (int t = lane; t < k * k; t += 32) {
        const int i = t % k, j = t / k;
        m[i + j * k] = (i <= j + 1) ? H[i + (long)j * ld] : 0.0;
    }
    __syncwarp();
    const int st = hess_eigs(k, m, k, r, im, lane, 32);
    __syncwarp();
    for (int i = lane; i < k; i += 32) {
        wr[i] = r[i];
        wi[i] = im[i];
    }
    if (lane == 0) status_out[0] = st;
}

cudaError_t launch_hess_eigs(int k, const double *H, int ld, double *wr, double *wi, int *status_out, cudaStream_t s)
{
    k_hess_eigs<<<1, 32, 0, s>>>(k, H, ld, wr, wi, status_out);
    return cudaGetLastError();
}

}  // namespace ppg
