// ppg_dense.cuh -- small dense float64 routines for the polynomial's roots.
//
// They turn the (d+2) x (d+1) Hessenberg matrix of a short Arnoldi run into the
// roots of the GMRES residual polynomial 1 - z p(z) (the harmonic Ritz values), the
// representation in which p(A) stays accurate at high degree.  Sizes are at most
// 64 x 64.  On the device one warp runs them: scalar control (deflation tests,
// shifts, reflector vectors) is computed identically by every lane from shared
// memory, and the O(n) loops of each step (applying a reflector to the rows or
// columns it touches, eliminating rows, scoring Leja candidates) are split across
// the lanes with a warp barrier after each.  With lane = 0, nl = 1 the same code runs
// serially, which is how the host build of the library's own checks uses it.
#pragma once

#include <math.h>

namespace ppg {

#ifndef PPG_HD
#define PPG_HD __host__ __device__
#endif

#if defined(__CUDA_ARCH__)
#define PPG_WSYNC() __syncwarp()
#else
#define PPG_WSYNC() \
    do {            \
    } while (0)
#endif

// Eigenvalues of the n x n upper Hessenberg matrix a (column-major, leading dimension
// lda; overwritten) by the Francis implicit double-shift QR iteration (Francis 1961;
// Golub and Van Loan, Matrix Computations, Sec. 7.5): deflation at negligible
// subdiagonal entries, 1x1 and 2x2 blocks read off directly, an exceptional shift after
// every 10 iterations without deflation.  Only the active block is transformed since no
// Schur vectors are wanted.  Returns 0, or 1 if the iteration limit (40 n sweeps) is hit.
// All nl lanes call it with the same arguments; a, wr and wi are shared.
PPG_HD inline int hess_eigs(int n, double *a, int lda, double *wr, double *wi, int lane = 0, int nl = 1)
{
#define PPG_A(i, j) a[(i) + (long)(j) * lda]
    const double eps = 2.220446049250313e-16;
    double anorm = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= (j + 1 < n - 1 ? j + 1 : n - 1); ++i) anorm = fmax(anorm, fabs(PPG_A(i, j)));
    int hi = n - 1;
    int its = 0, total = 0;
    while (hi >= 0) {
        // l: the largest index <= hi whose subdiagonal entry is negligible (0 if none)
        int l = hi;
        bool scan = true;
#if defined(__CUDA_ARCH__)
        if (nl == 32) {  // one candidate per lane, the largest found by a ballot
            bool neg = false;
            const int c = hi - lane;
            if (c > 0) {
                double s = fabs(PPG_A(c - 1, c - 1)) + fabs(PPG_A(c, c));
                if (s == 0.0) s = anorm;
                neg = fabs(PPG_A(c, c - 1)) <= eps * s;
            }
            const unsigned int m = __ballot_sync(0xffffffffu, neg);
            if (m) {
                l = hi - (__ffs(m) - 1);
                scan = false;
            } else if (hi <= 32) {
                l = 0;
                scan = false;
            }
        }
#endif
        if (scan) {  // serial scan (host build, or no hit among more than 32 candidates)
            l = hi;
            while (l > 0) {
                double s = fabs(PPG_A(l - 1, l - 1)) + fabs(PPG_A(l, l));
                if (s == 0.0) s = anorm;
                if (fabs(PPG_A(l, l - 1)) <= eps * s) break;
                --l;
            }
        }
        PPG_WSYNC();
        if (l > 0 && lane == 0) PPG_A(l, l - 1) = 0.0;
        if (l == hi) {
            if (lane == 0) {
                wr[hi] = PPG_A(hi, hi);
                wi[hi] = 0.0;
            }
            PPG_WSYNC();
            --hi;
            its = 0;
            continue;
        }
        if (l == hi - 1) {
            const double p = PPG_A(hi - 1, hi - 1), q = PPG_A(hi - 1, hi);
            const double r = PPG_A(hi, hi - 1), s = PPG_A(hi, hi);
            const double mid = 0.5 * (p + s);
            const double disc = 0.25 * (p - s) * (p - s) + q * r;
            PPG_WSYNC();
            if (lane == 0) {
                if (disc >= 0.0) {
                    const double sq = sqrt(disc);
                    const double l1 = mid + copysign(sq, mid);
                    const double det = p * s - q * r;
                    const double l2 = (l1 != 0.0) ? det / l1 : mid - copysign(sq, mid);
                    wr[hi - 1] = l1;
                    wi[hi - 1] = 0.0;
                    wr[hi] = l2;
                    wi[hi] = 0.0;
                } else {
                    const double sq = sqrt(-disc);
                    wr[hi - 1] = mid;
                    wi[hi - 1] = sq;
                    wr[hi] = mid;
                    wi[hi] = -sq;
                }
            }
            PPG_WSYNC();
            hi -= 2;
            its = 0;
            continue;
        }
        PPG_WSYNC();
        if (total >= 40 * n) return 1;
        ++its;
        ++total;
        double ssum, sprod;
        if (its % 10 == 0) {
            const double w = fabs(PPG_A(hi, hi - 1)) + fabs(PPG_A(hi - 1, hi - 2));
            ssum = 1.5 * w;
            sprod = w * w;
        } else {
            const double p = PPG_A(hi - 1, hi - 1), q = PPG_A(hi - 1, hi);
            const double r = PPG_A(hi, hi - 1), s = PPG_A(hi, hi);
            ssum = p + s;
            sprod = p * s - q * r;
        }
        // first column of (H - s1 I)(H - s2 I) restricted to rows l..l+2
        const double h00 = PPG_A(l, l), h10 = PPG_A(l + 1, l), h01 = PPG_A(l, l + 1), h11 = PPG_A(l + 1, l + 1);
        double x = h00 * h00 + h01 * h10 - ssum * h00 + sprod;
        double y = h10 * (h00 + h11 - ssum);
        double z = h10 * PPG_A(l + 2, l + 1);  // l + 2 <= hi here
        for (int k = l; k <= hi - 1; ++k) {
            const int nr = (k + 2 <= hi) ? 3 : 2;
            if (nr == 2) z = 0.0;
            const double scale = fabs(x) + fabs(y) + fabs(z);
            PPG_WSYNC();
            if (scale != 0.0) {
                // reflector I - beta v v^T mapping (x, y, z) to (alpha, 0, 0); the entries are scaled by
                // 1 / scale only when their squares could leave the float64 range (float64 division
                // and square root are slow on this GPU).  With alpha = -sign(x) ||(x, y, z)|| and
                // v0 = x - alpha, v^T v = -2 alpha v0.
                const bool wide = scale > 1e150 || scale < 1e-150;
                const double rs = wide ? 1.0 / scale : 1.0;
                const double xs = wide ? x * rs : x, ys = wide ? y * rs : y, zs = wide ? z * rs : z;
                double alpha = sqrt(fma(xs, xs, fma(ys, ys, zs * zs)));
                if (xs > 0.0) alpha = -alpha;
                const double v0 = xs - alpha, v1 = ys, v2 = zs;
                const double beta = -1.0 / (alpha * v0);
                const int jlo = (k - 1 > l) ? k - 1 : l;
                for (int j = jlo + lane; j <= hi; j += nl) {
                    double t = v0 * PPG_A(k, j) + v1 * PPG_A(k + 1, j);
                    if (nr == 3) t += v2 * PPG_A(k + 2, j);
                    t *= beta;
                    PPG_A(k, j) -= t * v0;
                    PPG_A(k + 1, j) -= t * v1;
                    if (nr == 3) PPG_A(k + 2, j) -= t * v2;
                }
                PPG_WSYNC();
                const int ihi = (k + 3 < hi) ? k + 3 : hi;
                for (int i = l + lane; i <= ihi; i += nl) {
                    double t = v0 * PPG_A(i, k) + v1 * PPG_A(i, k + 1);
                    if (nr == 3) t += v2 * PPG_A(i, k + 2);
                    t *= beta;
                    PPG_A(i, k) -= t * v0;
                    PPG_A(i, k + 1) -= t * v1;
                    if (nr == 3) PPG_A(i, k + 2) -= t * v2;
                }
                PPG_WSYNC();
                if (k > l && lane == 0) {
                    PPG_A(k + 1, k - 1) = 0.0;
                    if (nr == 3) PPG_A(k + 2, k - 1) = 0.0;
                }
                PPG_WSYNC();
            }
            if (k + 1 <= hi - 1) {
                x = PPG_A(k + 1, k);
                y = PPG_A(k + 2, k);
                z = (k + 3 <= hi) ? PPG_A(k + 3, k) : 0.0;
            }
        }
    }
    return 0;
#undef PPG_A
}

// Solves M f = rhs for a dense n x n matrix (column-major, ld; overwritten) by Gaussian
// elimination with partial pivoting.  Returns 0, or 1 on a zero pivot.
PPG_HD inline int dense_solve(int n, double *m, int ld, double *rhs, int lane = 0, int nl = 1)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = fabs(m[c + (long)c * ld]);
        for (int r = c + 1; r < n; ++r) {
            const double v = fabs(m[r + (long)c * ld]);
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (!(best > 0.0)) return 1;
        PPG_WSYNC();
        if (piv != c) {
            for (int j = lane; j < n; j += nl) {
                const double t = m[c + (long)j * ld];
                m[c + (long)j * ld] = m[piv + (long)j * ld];
                m[piv + (long)j * ld] = t;
            }
            if (lane == 0) {
                const double t = rhs[c];
                rhs[c] = rhs[piv];
                rhs[piv] = t;
            }
        }
        PPG_WSYNC();
        const double d = m[c + (long)c * ld];
        for (int r = c + 1 + lane; r < n; r += nl) {
            const double f = m[r + (long)c * ld] / d;
            if (f == 0.0) continue;
            for (int j = c; j < n; ++j) m[r + (long)j * ld] -= f * m[c + (long)j * ld];
            rhs[r] -= f * rhs[c];
        }
        PPG_WSYNC();
    }
    if (lane == 0) {
        for (int r = n - 1; r >= 0; --r) {
            double s = rhs[r];
            for (int j = r + 1; j < n; ++j) s -= m[r + (long)j * ld] * rhs[j];
            rhs[r] = s / m[r + (long)r * ld];
        }
    }
    PPG_WSYNC();
    return 0;
}

// Harmonic Ritz values of an Arnoldi run: with H_k the leading k x k block of the
// (k+1) x k Hessenberg matrix H (column-major, ldh) and h = H[k, k-1], the eigenvalues
// of H_k + h^2 H_k^{-T} e_k e_k^T.  They are the roots of the GMRES residual polynomial
// 1 - z p(z) of the run.  work: >= k*k + k doubles (shared by the lanes).  Returns 0,
// 1 (QR failed) or 2 (H_k singular).
PPG_HD inline int harmonic_ritz(int k, const double *H, int ldh, double *wr, double *wi, double *work, int lane = 0,
                                int nl = 1)
{
    double *m = work;  // k x k, ld k
    double *f = work + k * k;
    for (int t = lane; t < k * k; t += nl) {
        const int i = t % k, j = t / k;
        m[i + j * k] = H[j + (long)i * ldh];  // H_k^T
    }
    for (int i = lane; i < k; i += nl) f[i] = (i == k - 1) ? 1.0 : 0.0;
    PPG_WSYNC();
    if (dense_solve(k, m, k, f, lane, nl)) return 2;
    const double h = H[k + (long)(k - 1) * ldh];
    for (int t = lane; t < k * k; t += nl) {
        const int i = t % k, j = t / k;
        double v = (i <= j + 1) ? H[i + (long)j * ldh] : 0.0;
        if (j == k - 1) v += h * h * f[i];
        m[i + j * k] = v;
    }
    PPG_WSYNC();
    return hess_eigs(k, m, k, wr, wi, lane, nl) ? 1 : 0;
}

// Modified Leja ordering of k roots (Reichel 1990; Baglama, Calvetti, Reichel 1998):
// start from the root of largest modulus, then repeatedly take the root that maximises
// the product of distances to those already chosen (sums of logarithms avoid overflow).
// Complex roots are taken with positive imaginary part first, immediately followed by
// their conjugate, so that real arithmetic can apply each pair at once.  order receives
// indices into (wr, wi); used: k ints; score: k doubles of scratch (all shared).
PPG_HD inline void leja_order(int k, const double *wr, const double *wi, int *order, int *used, double *score,
                              int lane = 0, int nl = 1)
{
    for (int i = lane; i < k; i += nl) {
        used[i] = 0;
        score[i] = log(hypot(wr[i], wi[i]));
    }
    PPG_WSYNC();
    int cnt = 0;
    while (cnt < k) {
        // every lane scans the scores for the best candidate (the scores are shared)
        int best = -1;
        double best_score = -INFINITY;
        for (int i = 0; i < k; ++i) {
            if (used[i] || wi[i] < 0.0) continue;  // conjugates follow their partner
            if (best < 0 || score[i] > best_score) {
                best = i;
                best_score = score[i];
            }
        }
        if (best < 0) {  // only unmatched conjugates left (should not happen): take them as they are
            for (int i = 0; i < k; ++i)
                if (!used[i]) {
                    best = i;
                    break;
                }
        }
        int partner = -1;
        if (wi[best] > 0.0) {
            double dbest = INFINITY;
            for (int i = 0; i < k; ++i) {
                if (used[i] || i == best || !(wi[i] < 0.0)) continue;
                const double dd = fabs(wr[i] - wr[best]) + fabs(wi[i] + wi[best]);
                if (dd < dbest) {
                    dbest = dd;
                    partner = i;
                }
            }
        }
        PPG_WSYNC();
        if (lane == 0) {
            used[best] = 1;
            order[cnt] = best;
            if (partner >= 0) {
                used[partner] = 1;
                order[cnt + 1] = partner;
            }
        }
        // scores: distances to the chosen points (a conjugate pair adds both)
        for (int i = lane; i < k; i += nl) {
            const double base = (cnt == 0) ? 0.0 : score[i];
            double s = base + log(hypot(wr[i] - wr[best], wi[i] - wi[best]));
            if (partner >= 0) s += log(hypot(wr[i] - wr[partner], wi[i] - wi[partner]));
            score[i] = s;
        }
        PPG_WSYNC();
        cnt += (partner >= 0) ? 2 : 1;
    }
}

}  // namespace ppg
