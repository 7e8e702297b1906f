/*
 * ppg_oracle.c -- CPU oracle for polynomial-preconditioned GMRES.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, serial, float64
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg load it; the library
 * never calls it and shares no code with it.
 *
 * What it computes (Loe, Thornquist, Boman, "Polynomial Preconditioned GMRES
 * to Reduce Communication in Parallel Computing", arXiv 1907.00072):
 *
 *   - the GMRES minimum-residual polynomial p of degree d, i.e. the p that
 *     minimises ||v0 - A p(A) v0||_2 (Section II, Eq. 1), built two ways:
 *       (a) the paper's route: power basis V = [v0, A v0, ..., A^d v0],
 *           normal equations (AV)^T (AV) y = (AV)^T v0 solved by Cholesky with
 *           the POTRF failure test (Section II, Section IV);
 *       (b) a short GMRES run: d+1 steps of modified Gram-Schmidt Arnoldi from
 *           v0 followed by the Hessenberg least-squares solve.  This defines
 *           the same p in the Arnoldi basis and stays accurate at any degree.
 *   - p(A)x in power form, p(A) = y_{d+1} A^d + ... + y_2 A + y_1 (Eq. 2),
 *     evaluated as the explicit sum of the equation, and in Arnoldi form.
 *   - restarted GMRES(m) with right preconditioning, A p(A) u = b, x = p(A) u
 *     (Section I), modified Gram-Schmidt Arnoldi, Givens rotations for the
 *     Hessenberg least-squares problem, and a true residual at every restart.
 *     Relative residual ||b - A x|| / ||b|| is the stopping measure
 *     (Section III).
 *   - the composition of Section VI: ILU(0) M = L U (no fill: L U agrees with A
 *     on A's sparsity pattern) applied on the left and the polynomial on the
 *     right, M^{-1} A p(M^{-1} A) y = M^{-1} b, x = p(M^{-1} A) y; the polynomial
 *     is then the minimum-residual polynomial of B = M^{-1} A.  Every "_lu"
 *     routine takes the factors; with lu = NULL it is the plain method.
 *   - the combination Section VII proposes: the polynomial inside an s-step
 *     (communication-avoiding) GMRES, orthogonalising once per s applications
 *     of A p(A).  The paper gives no algorithm; orc_sstep_gmres takes the
 *     standard s-step construction (Newton basis, block Gram-Schmidt, Cholesky
 *     QR, Hessenberg columns recovered from the change of basis).  It produces
 *     GMRES's iterates in exact arithmetic, and its pins are the Krylov minima
 *     of dense least squares and the dense solution.
 *
 * Every routine is written out loop by loop, in float64, one core.
 *
 * Conventions shared with the Python wrapper (oracle/__init__.py):
 *   CSR matrices: int32 row pointers (n+1) and column indices, float64 values.
 *   Dense matrices: column-major unless stated.
 *   Polynomial descriptor (ORC_POLY_*):
 *     NONE    p(z) = 1 (unpreconditioned GMRES);
 *     POWER   p(z) = sum_i coef[i] z^i, i = 0..deg (Eq. 2 with coef[i] = y_{i+1});
 *     ARNOLDI p(z) = sum_j y[j] q_j(z) with q_0 = 1/beta and
 *             q_{j}(z) = (z q_{j-1}(z) - sum_{i<j} H[i,j-1] q_i(z)) / H[j,j-1],
 *             H of size (deg+2) x (deg+1), column-major, ld = deg+2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_POLY_NONE 0
#define ORC_POLY_POWER 1
#define ORC_POLY_ARNOLDI 2

/* relative threshold for a (lucky) Arnoldi breakdown: h_{j+1,j} <= BRK * ||A p(A) v_j|| */
#define ORC_BREAKDOWN 1e-14

typedef struct {
    int64_t n;
    const int32_t *rowptr;
    const int32_t *colidx;
    const double *vals;
    const double *lu; /* ILU(0) factors on the same pattern (Section VI's left preconditioner), or NULL */
} csr_t;

typedef struct {
    int kind;
    int deg;
    const double *coef;  /* POWER */
    const double *H;     /* ARNOLDI */
    const double *y;     /* ARNOLDI */
    double beta;         /* ARNOLDI */
} poly_t;

/* ------------------------------------------------------------------ */
/* vector helpers                                                     */
/* ------------------------------------------------------------------ */

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double nrm2(int64_t n, const double *a) { return sqrt(dot(n, a, a)); }

static void axpy(int64_t n, double alpha, const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] += alpha * x[i];
}

static void scal(int64_t n, double alpha, double *x)
{
    for (int64_t i = 0; i < n; ++i) x[i] *= alpha;
}

static double *dalloc(int64_t n)
{
    double *p = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    return p;
}

/* ------------------------------------------------------------------ */
/* sparse matrix-vector product: y_i = sum_k vals[k] x[colidx[k]]      */
/* ------------------------------------------------------------------ */

static void spmv(const csr_t *A, const double *x, double *y)
{
    for (int64_t i = 0; i < A->n; ++i) {
        double s = 0.0;
        for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) s += A->vals[k] * x[A->colidx[k]];
        y[i] = s;
    }
}

void orc_spmv(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, const double *x, double *y)
{
    csr_t A = {n, rp, ci, va, NULL};
    spmv(&A, x, y);
}

/* ------------------------------------------------------------------ */
/* ILU(0): M = L U with L unit lower and U upper triangular, both on    */
/* the sparsity pattern of A (Section VI's left preconditioner)        */
/* ------------------------------------------------------------------ */

/* Incomplete LU with no fill, row by row: for row i and each of its entries k < i in
 * increasing column order, l_ik = a_ik / u_kk, then every entry j > k of row i that
 * row k also has is reduced by l_ik u_kj; entries row k has but row i lacks are
 * dropped.  lu (nnz values, A's pattern) receives L below the diagonal (its unit
 * diagonal not stored) and U on and above it.  Columns within a row must be sorted
 * and every row must hold its diagonal.  Returns 0, -(i+1) if row i has no diagonal
 * or a zero pivot, -2 on allocation failure. */
int orc_ilu0(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, double *lu)
{
    int64_t nnz = rp[n];
    memcpy(lu, va, sizeof(double) * (size_t)nnz);
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *diag = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!pos || !diag) {
        free(pos);
        free(diag);
        return -2;
    }
    for (int64_t j = 0; j < n; ++j) pos[j] = -1;
    int status = 0;
    for (int64_t i = 0; i < n && !status; ++i) {
        diag[i] = -1;
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            pos[ci[t]] = t;
            if (ci[t] == i) diag[i] = t;
        }
        if (diag[i] < 0) status = -(int)(i + 1);
        for (int32_t t = rp[i]; t < rp[i + 1] && !status; ++t) {
            int32_t k = ci[t];
            if (k >= i) break;
            double lik = lu[t] / lu[diag[k]];
            lu[t] = lik;
            for (int32_t q = diag[k] + 1; q < rp[k + 1]; ++q) {
                int32_t p = pos[ci[q]];
                if (p >= 0) lu[p] -= lik * lu[q];
            }
        }
        if (!status && !(lu[diag[i]] != 0.0)) status = -(int)(i + 1);
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) pos[ci[t]] = -1;
    }
    free(pos);
    free(diag);
    return status;
}

/* y = (L U)^{-1} x: forward substitution with the unit lower factor, then back
 * substitution with the upper one (rows sorted, diagonal present). */
static void ilu0_solve(const csr_t *A, const double *x, double *y)
{
    int64_t n = A->n;
    const int32_t *rp = A->rowptr, *ci = A->colidx;
    const double *lu = A->lu;
    for (int64_t i = 0; i < n; ++i) {
        double s = x[i];
        for (int32_t t = rp[i]; t < rp[i + 1] && ci[t] < i; ++t) s -= lu[t] * y[ci[t]];
        y[i] = s;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = y[i], d = 0.0;
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            if (ci[t] > i) s -= lu[t] * y[ci[t]];
            else if (ci[t] == i) d = lu[t];
        }
        y[i] = s / d;
    }
}

void orc_ilu0_apply(int64_t n, const int32_t *rp, const int32_t *ci, const double *lu, const double *x, double *y)
{
    csr_t A = {n, rp, ci, NULL, lu};
    ilu0_solve(&A, x, y);
}

/* the operator the Krylov methods see: y = A x, or with ILU(0) factors y = M^{-1} A x */
static void opmul(const csr_t *A, const double *x, double *y)
{
    spmv(A, x, y);
    if (A->lu) {
        double *t = dalloc(A->n);
        memcpy(t, y, sizeof(double) * (size_t)A->n);
        ilu0_solve(A, t, y);
        free(t);
    }
}

/* rows listed in `rows` only: y[t] = (A x)[rows[t]] (used to check sampled outputs) */
void orc_spmv_rows(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, const double *x,
                   int64_t nrows, const int64_t *rows, double *y)
{
    (void)n;
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t];
        double s = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s += va[k] * x[ci[k]];
        y[t] = s;
    }
}

/* transpose by counting sort; within a row of A^T the columns come out ascending */
void orc_transpose(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, int32_t *rpt, int32_t *cit,
                   double *vat)
{
    int64_t nnz = rp[n];
    for (int64_t i = 0; i <= n; ++i) rpt[i] = 0;
    for (int64_t k = 0; k < nnz; ++k) rpt[ci[k] + 1] += 1;
    for (int64_t i = 0; i < n; ++i) rpt[i + 1] += rpt[i];
    int32_t *fill = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            int32_t c = ci[k];
            int32_t dst = rpt[c] + fill[c]++;
            cit[dst] = (int32_t)i;
            vat[dst] = va[k];
        }
    }
    free(fill);
}

/* ------------------------------------------------------------------ */
/* the polynomial p(A) applied to a vector                            */
/* ------------------------------------------------------------------ */

/* Eq. 2 written out: out = sum_{i=0}^{deg} coef[i] A^i x */
static void poly_apply_power(const csr_t *A, int deg, const double *coef, const double *x, double *out,
                             double *t, double *t2)
{
    int64_t n = A->n;
    memcpy(t, x, (size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) out[i] = coef[0] * t[i];
    for (int p = 1; p <= deg; ++p) {
        opmul(A, t, t2); /* t2 = A^p x */
        memcpy(t, t2, (size_t)n * sizeof(double));
        axpy(n, coef[p], t, out);
    }
}

/* Arnoldi form: t_0 = x / beta, t_j = (A t_{j-1} - sum_{i<j} H[i,j-1] t_i) / H[j,j-1],
 * out = sum_{j=0}^{deg} y[j] t_j.  T is n x (deg+1) scratch. */
static void poly_apply_arnoldi(const csr_t *A, int deg, const double *H, const double *y, double beta,
                               const double *x, double *out, double *T)
{
    int64_t n = A->n;
    int ldh = deg + 2;
    for (int64_t i = 0; i < n; ++i) T[i] = x[i] / beta;
    for (int j = 1; j <= deg; ++j) {
        double *tj = T + (int64_t)j * n;
        opmul(A, T + (int64_t)(j - 1) * n, tj);
        for (int i = 0; i < j; ++i) axpy(n, -H[i + (int64_t)(j - 1) * ldh], T + (int64_t)i * n, tj);
        scal(n, 1.0 / H[j + (int64_t)(j - 1) * ldh], tj);
    }
    for (int64_t i = 0; i < n; ++i) out[i] = 0.0;
    for (int j = 0; j <= deg; ++j) axpy(n, y[j], T + (int64_t)j * n, out);
}

typedef struct {
    double *t, *t2, *T; /* scratch */
} poly_ws;

static int poly_ws_init(poly_ws *w, int64_t n, const poly_t *p)
{
    w->t = dalloc(n);
    w->t2 = dalloc(n);
    w->T = (p->kind == ORC_POLY_ARNOLDI) ? dalloc(n * (p->deg + 1)) : NULL;
    return (w->t && w->t2 && (p->kind != ORC_POLY_ARNOLDI || w->T)) ? 0 : -1;
}

static void poly_ws_free(poly_ws *w)
{
    free(w->t);
    free(w->t2);
    free(w->T);
}

/* out = p(A) x; returns the number of SpMVs used */
static int poly_apply(const csr_t *A, const poly_t *p, const double *x, double *out, poly_ws *w)
{
    switch (p->kind) {
    case ORC_POLY_POWER:
        poly_apply_power(A, p->deg, p->coef, x, out, w->t, w->t2);
        return p->deg;
    case ORC_POLY_ARNOLDI:
        poly_apply_arnoldi(A, p->deg, p->H, p->y, p->beta, x, out, w->T);
        return p->deg;
    default:
        memcpy(out, x, (size_t)A->n * sizeof(double));
        return 0;
    }
}

void orc_poly_apply_lu(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, const double *lu, int kind, int deg,
                    const double *coef, const double *H, const double *y, double beta, const double *x, double *out)
{
    csr_t A = {n, rp, ci, va, lu};
    poly_t p = {kind, deg, coef, H, y, beta};
    poly_ws w;
    if (poly_ws_init(&w, n, &p) == 0) poly_apply(&A, &p, x, out, &w);
    poly_ws_free(&w);
}

void orc_poly_apply(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, int kind, int deg,
                    const double *coef, const double *H, const double *y, double beta, const double *x, double *out)
{
    orc_poly_apply_lu(n, rp, ci, va, NULL, kind, deg, coef, H, y, beta, x, out);
}

/* scalar evaluation z p(z) for real z (used for the alpha p(alpha) plots of Section V) */
double orc_poly_eval_zp(int kind, int deg, const double *coef, const double *H, const double *y, double beta, double z)
{
    if (kind == ORC_POLY_POWER) {
        double s = 0.0, zp = 1.0;
        for (int i = 0; i <= deg; ++i) {
            s += coef[i] * zp;
            zp *= z;
        }
        return z * s;
    }
    if (kind == ORC_POLY_ARNOLDI) {
        int ldh = deg + 2;
        double q[128];
        if (deg + 1 > 128) return NAN;
        q[0] = 1.0 / beta;
        for (int j = 1; j <= deg; ++j) {
            double v = z * q[j - 1];
            for (int i = 0; i < j; ++i) v -= H[i + (j - 1) * ldh] * q[i];
            q[j] = v / H[j + (j - 1) * ldh];
        }
        double s = 0.0;
        for (int j = 0; j <= deg; ++j) s += y[j] * q[j];
        return z * s;
    }
    return z;
}

/* ------------------------------------------------------------------ */
/* Cholesky with the POTRF failure test                               */
/* ------------------------------------------------------------------ */

/* G (k x k, column-major, ld) = L L^T in place (lower triangle).  Returns 0, or the
 * 1-based order j of the first leading minor that is not positive definite: the
 * pivot G_jj - sum_p L_jp^2 is not > 0 (this includes NaN).  This is LAPACK
 * POTRF's `info`. */
int orc_cholesky(int k, double *G, int ld)
{
    for (int j = 0; j < k; ++j) {
        double d = G[j + j * ld];
        for (int p = 0; p < j; ++p) d -= G[j + p * ld] * G[j + p * ld];
        if (!(d > 0.0)) return j + 1;
        double ljj = sqrt(d);
        G[j + j * ld] = ljj;
        for (int i = j + 1; i < k; ++i) {
            double s = G[i + j * ld];
            for (int p = 0; p < j; ++p) s -= G[i + p * ld] * G[j + p * ld];
            G[i + j * ld] = s / ljj;
        }
    }
    return 0;
}

/* solve L L^T y = r for the leading k x k block of a factored G */
static void cholesky_solve(int k, const double *L, int ld, const double *r, double *y)
{
    for (int i = 0; i < k; ++i) { /* L z = r */
        double s = r[i];
        for (int p = 0; p < i; ++p) s -= L[i + p * ld] * y[p];
        y[i] = s / L[i + i * ld];
    }
    for (int i = k - 1; i >= 0; --i) { /* L^T y = z */
        double s = y[i];
        for (int p = i + 1; p < k; ++p) s -= L[p + i * ld] * y[p];
        y[i] = s / L[i + i * ld];
    }
}

/* ------------------------------------------------------------------ */
/* polynomial construction, route (a): Eq. 1 and Cholesky             */
/* ------------------------------------------------------------------ */

/* Builds AV = [A v0, A^2 v0, ..., A^{deg+1} v0], G = (AV)^T AV, r = (AV)^T v0 and
 * solves G y = r by Cholesky.  coef[i] = y_{i+1} multiplies A^i (Eq. 2).
 * If the factorisation fails with info = j, the leading (j-1) x (j-1) block did
 * factor, so the polynomial of degree j-2 is used (the highest degree without a
 * POTRF warning, Section IV).  Returns the degree used (-1 if even degree 0
 * fails); *info receives POTRF's info for the requested degree.  gram_out
 * (optional, (deg+1)^2, column-major) receives G before factoring and rhs_out
 * (optional) receives r. */
int orc_poly_normal_eq_lu(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, const double *lu, const double *v0, int deg,
                       double *coef, int *info, double *gram_out, double *rhs_out)
{
    csr_t A = {n, rp, ci, va, lu};
    int k = deg + 1;
    double *AV = dalloc(n * k);
    double *G = dalloc((int64_t)k * k);
    double *r = dalloc(k);
    if (!AV || !G || !r) {
        free(AV); free(G); free(r);
        return -2;
    }
    opmul(&A, v0, AV);
    for (int j = 1; j < k; ++j) opmul(&A, AV + (int64_t)(j - 1) * n, AV + (int64_t)j * n);
    for (int a = 0; a < k; ++a) {
        for (int b = 0; b < k; ++b) G[a + b * k] = dot(n, AV + (int64_t)a * n, AV + (int64_t)b * n);
        r[a] = dot(n, AV + (int64_t)a * n, v0);
    }
    if (gram_out) memcpy(gram_out, G, sizeof(double) * k * k);
    if (rhs_out) memcpy(rhs_out, r, sizeof(double) * k);
    int inf = orc_cholesky(k, G, k);
    *info = inf;
    int used = (inf == 0) ? deg : inf - 2;
    for (int i = 0; i <= deg; ++i) coef[i] = 0.0;
    if (used >= 0) cholesky_solve(used + 1, G, k, r, coef);
    free(AV);
    free(G);
    free(r);
    return used;
}

int orc_poly_normal_eq(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, const double *v0, int deg,
                       double *coef, int *info, double *gram_out, double *rhs_out)
{
    return orc_poly_normal_eq_lu(n, rp, ci, va, NULL, v0, deg, coef, info, gram_out, rhs_out);
}

/* ------------------------------------------------------------------ */
/* Arnoldi (modified Gram-Schmidt) for the operator A p(A)             */
/* ------------------------------------------------------------------ */

typedef struct {
    const csr_t *A;
    const poly_t *p;
    poly_ws ws;
    double *z;
    long spmvs;
} op_t;

/* out = A p(A) x */
static void op_apply(op_t *op, const double *x, double *out)
{
    op->spmvs += poly_apply(op->A, op->p, x, op->z, &op->ws);
    opmul(op->A, op->z, out);
    op->spmvs += 1;
}

/* One Arnoldi step on column j: w = op(V_j) is orthogonalised against V_0..V_j with
 * MGS; H[0..j+1, j] is written (column-major, ldh).  V_{j+1} = w / H[j+1,j] unless
 * the step breaks down.  Returns 1 on breakdown, 0 otherwise. */
static int arnoldi_step(op_t *op, int64_t n, double *V, int j, double *H, int ldh)
{
    double *w = V + (int64_t)(j + 1) * n;
    op_apply(op, V + (int64_t)j * n, w);
    double w0 = nrm2(n, w);
    for (int i = 0; i <= j; ++i) {
        double h = dot(n, V + (int64_t)i * n, w);
        H[i + j * ldh] = h;
        axpy(n, -h, V + (int64_t)i * n, w);
    }
    double h = nrm2(n, w);
    H[j + 1 + j * ldh] = h;
    if (!(h > ORC_BREAKDOWN * w0)) return 1;
    scal(n, 1.0 / h, w);
    return 0;
}

/* k steps of Arnoldi for A p(A) from v (normalised internally).  V: n x (k+1),
 * H: (k+1) x k column-major (ld = k+1).  Returns the number of steps completed
 * (< k only on breakdown); *beta = ||v||. */
int orc_arnoldi_lu(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, const double *lu, int kind, int deg,
                const double *coef, const double *Hp, const double *yp, double betap, const double *v, int k,
                double *V, double *H, double *beta)
{
    csr_t A = {n, rp, ci, va, lu};
    poly_t p = {kind, deg, coef, Hp, yp, betap};
    op_t op = {&A, &p, {0}, dalloc(n), 0};
    if (poly_ws_init(&op.ws, n, &p) != 0 || !op.z) {
        poly_ws_free(&op.ws);
        free(op.z);
        return -2;
    }
    memset(H, 0, sizeof(double) * (size_t)(k + 1) * (size_t)k);
    *beta = nrm2(n, v);
    for (int64_t i = 0; i < n; ++i) V[i] = v[i] / *beta;
    int done = 0;
    for (int j = 0; j < k; ++j) {
        int brk = arnoldi_step(&op, n, V, j, H, k + 1);
        done = j + 1;
        if (brk) break;
    }
    poly_ws_free(&op.ws);
    free(op.z);
    return done;
}

int orc_arnoldi(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, int kind, int deg,
                const double *coef, const double *Hp, const double *yp, double betap, const double *v, int k,
                double *V, double *H, double *beta)
{
    return orc_arnoldi_lu(n, rp, ci, va, NULL, kind, deg, coef, Hp, yp, betap, v, k, V, H, beta);
}

/* ------------------------------------------------------------------ */
/* Hessenberg least squares with Givens rotations                      */
/* ------------------------------------------------------------------ */

/* rotate rows i, i+1 of column col: (a, b) -> (c a + s b, -s a + c b) */
static void rot(double c, double s, double *a, double *b)
{
    double t = c * *a + s * *b;
    *b = -s * *a + c * *b;
    *a = t;
}

/* new rotation that zeroes b in (a, b); returns r = hypot(a, b) */
static double make_rot(double a, double b, double *c, double *s)
{
    double r = hypot(a, b);
    if (r == 0.0) {
        *c = 1.0;
        *s = 0.0;
        return 0.0;
    }
    *c = a / r;
    *s = b / r;
    return r;
}

/* Solve min || beta e1 - Hbar y || for the (k+1) x k upper Hessenberg Hbar (column-major,
 * ldh).  Returns the residual norm; y receives k entries. */
static double hess_lsq(int k, const double *H, int ldh, double beta, double *y)
{
    double *R = dalloc((int64_t)(k + 1) * k);
    double *g = dalloc(k + 1);
    double *c = dalloc(k), *s = dalloc(k);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i <= j + 1; ++i) R[i + j * (k + 1)] = H[i + j * ldh];
    g[0] = beta;
    for (int j = 0; j < k; ++j) {
        for (int i = 0; i < j; ++i) rot(c[i], s[i], &R[i + j * (k + 1)], &R[i + 1 + j * (k + 1)]);
        R[j + j * (k + 1)] = make_rot(R[j + j * (k + 1)], R[j + 1 + j * (k + 1)], &c[j], &s[j]);
        R[j + 1 + j * (k + 1)] = 0.0;
        rot(c[j], s[j], &g[j], &g[j + 1]);
    }
    for (int i = k - 1; i >= 0; --i) {
        double v = g[i];
        for (int p = i + 1; p < k; ++p) v -= R[i + p * (k + 1)] * y[p];
        y[i] = v / R[i + i * (k + 1)];
    }
    double res = fabs(g[k]);
    free(R);
    free(g);
    free(c);
    free(s);
    return res;
}

/* ------------------------------------------------------------------ */
/* polynomial construction, route (b): short GMRES run                 */
/* ------------------------------------------------------------------ */

/* deg+1 MGS Arnoldi steps with A from v0 give Hbar ((deg+2) x (deg+1), written to H with
 * ld deg+2) and V; y solves min ||beta e1 - Hbar y||, so p(A) v0 = V_{deg+1} y and
 * ||v0 - A p(A) v0|| = *resid (the GMRES residual, Section II).  On breakdown after j
 * steps the exact polynomial has degree j-1; the return value is the degree built
 * (entries of y beyond it are zero).  Returns -2 on allocation failure. */
int orc_poly_gmres_lu(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, const double *lu, const double *v0, int deg,
                   double *H, double *y, double *beta, double *resid)
{
    int k = deg + 1;
    double *V = dalloc(n * (k + 1));
    if (!V) return -2;
    int done = orc_arnoldi_lu(n, rp, ci, va, lu, ORC_POLY_NONE, 0, NULL, NULL, NULL, 1.0, v0, k, V, H, beta);
    free(V);
    if (done < 0) return done;
    for (int j = 0; j <= deg; ++j) y[j] = 0.0;
    *resid = hess_lsq(done, H, k + 1, *beta, y);
    if (done < k) *resid = 0.0; /* breakdown: v0 lies in an invariant subspace, p is exact */
    return done - 1;
}

int orc_poly_gmres(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, const double *v0, int deg,
                   double *H, double *y, double *beta, double *resid)
{
    return orc_poly_gmres_lu(n, rp, ci, va, NULL, v0, deg, H, y, beta, resid);
}

/* Power coefficients of the Arnoldi-form polynomial: K_{k} = V_k R with column j of R the
 * coordinates of A^j v0 (r_0 = beta e1, r_{j+1} = Hbar r_j), so p(A) v0 = V y = K c with
 * c = R^{-1} y.  coef[i] multiplies z^i. */
void orc_poly_arnoldi_to_power(int deg, const double *H, const double *y, double beta, double *coef)
{
    int k = deg + 1, ldh = deg + 2;
    double *R = dalloc((int64_t)k * k);
    R[0] = beta;
    for (int j = 0; j + 1 < k; ++j) {
        /* r_{j+1}[i] = sum_{l<=j} H[i,l] r_j[l], i = 0..j+1 */
        for (int i = 0; i <= j + 1; ++i) {
            double s = 0.0;
            for (int l = 0; l <= j; ++l) s += H[i + l * ldh] * R[l + j * k];
            R[i + (j + 1) * k] = s;
        }
    }
    for (int i = k - 1; i >= 0; --i) {
        double v = y[i];
        for (int p = i + 1; p < k; ++p) v -= R[i + p * k] * coef[p];
        coef[i] = v / R[i + i * k];
    }
    free(R);
}

/* ------------------------------------------------------------------ */
/* restarted, right-preconditioned GMRES(m)                            */
/* ------------------------------------------------------------------ */

/* stats layout (doubles):
 *   0 iterations  1 restarts (cycles)  2 spmvs  3 dots  4 converged (1/0)
 *   5 true relres at exit  6 last estimated relres  7 breakdowns */
#define ORC_NSTATS 8

/* Solves A x = b with x = p(A) u, A p(A) u = b.  x holds x0 on entry and the final
 * iterate on exit.  A cycle ends after m iterations, when the Givens estimate
 * |g_{j+1}| <= tol ||b||, on breakdown, or at maxit iterations; x is then updated
 * with p(A) V y and the true residual b - A x is recomputed.  The solve stops when
 * ||b - A x|| <= tol ||b|| or maxit is reached.  hist (optional, capacity hist_cap)
 * receives |g_{j+1}| / ||b|| per iteration.  Returns 0 if converged, 1 if not,
 * -2 on allocation failure.
 * With ILU(0) factors (Section VI) the system is M^{-1} A p(M^{-1} A) u = M^{-1} b:
 * each cycle starts from the preconditioned residual M^{-1} (b - A x), the Givens
 * estimate is relative to ||M^{-1} b|| (the left-preconditioned residual GMRES
 * minimises), and the stopping test stays the true ||b - A x|| <= tol ||b||. */
int orc_gmres_lu(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, const double *lu, int kind, int deg,
              const double *coef, const double *Hp, const double *yp, double betap, const double *b, double *x,
              double tol, int m, int maxit, double *stats, double *hist, int hist_cap)
{
    csr_t A = {n, rp, ci, va, lu};
    poly_t p = {kind, deg, coef, Hp, yp, betap};
    op_t op = {&A, &p, {0}, dalloc(n), 0};
    double *V = dalloc(n * (m + 1));
    double *r = dalloc(n);
    double *H = dalloc((int64_t)(m + 1) * m);
    double *cs = dalloc(m), *sn = dalloc(m), *g = dalloc(m + 1), *yv = dalloc(m);
    double *z = dalloc(n), *pz = dalloc(n);
    int ok = (poly_ws_init(&op.ws, n, &p) == 0) && op.z && V && r && H && cs && sn && g && yv && z && pz;
    for (int i = 0; i < ORC_NSTATS; ++i) stats[i] = 0.0;
    int status = -2;
    if (!ok) goto out;

    double bnorm = nrm2(n, b);
    long iters = 0, cycles = 0, dots = 0, brk_count = 0;
    int converged = 0;
    double relres = 0.0, est = 0.0;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * (size_t)n);
        converged = 1;
        goto done;
    }
    double enorm = bnorm; /* the norm the Givens estimate is relative to */
    if (lu) {
        ilu0_solve(&A, b, z);
        enorm = nrm2(n, z);
        dots += 1;
    }
    for (;;) {
        spmv(&A, x, r); /* true residual */
        op.spmvs += 1;
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double beta = nrm2(n, r);
        dots += 1;
        relres = beta / bnorm;
        if (relres <= tol) {
            converged = 1;
            break;
        }
        if (iters >= maxit) break;
        if (lu) { /* left preconditioning: the cycle's residual is M^{-1} r */
            memcpy(z, r, sizeof(double) * (size_t)n);
            ilu0_solve(&A, z, r);
            beta = nrm2(n, r);
            dots += 1;
        }
        cycles += 1;
        for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            int brk = arnoldi_step(&op, n, V, j, H, m + 1);
            dots += j + 2; /* MGS: j+1 inner products and one norm */
            double *hj = H + (int64_t)j * (m + 1);
            for (int i = 0; i < j; ++i) rot(cs[i], sn[i], &hj[i], &hj[i + 1]);
            hj[j] = make_rot(hj[j], hj[j + 1], &cs[j], &sn[j]);
            hj[j + 1] = 0.0;
            rot(cs[j], sn[j], &g[j], &g[j + 1]);
            iters += 1;
            k = j + 1;
            est = fabs(g[j + 1]) / enorm;
            if (hist && iters <= hist_cap) hist[iters - 1] = est;
            if (brk) {
                brk_count += 1;
                break;
            }
            if (est <= tol || iters >= maxit) break;
        }
        /* y = R^{-1} g (k x k upper triangle of the rotated H) */
        for (int i = k - 1; i >= 0; --i) {
            double v = g[i];
            for (int q = i + 1; q < k; ++q) v -= H[i + (int64_t)q * (m + 1)] * yv[q];
            yv[i] = v / H[i + (int64_t)i * (m + 1)];
        }
        memset(z, 0, sizeof(double) * (size_t)n);
        for (int i = 0; i < k; ++i) axpy(n, yv[i], V + (int64_t)i * n, z);
        op.spmvs += poly_apply(&A, &p, z, pz, &op.ws);
        axpy(n, 1.0, pz, x);
    }
done:
    stats[0] = (double)iters;
    stats[1] = (double)cycles;
    stats[2] = (double)op.spmvs;
    stats[3] = (double)dots;
    stats[4] = converged ? 1.0 : 0.0;
    stats[5] = relres;
    stats[6] = est;
    stats[7] = (double)brk_count;
    status = converged ? 0 : 1;
out:
    poly_ws_free(&op.ws);
    free(op.z);
    free(V);
    free(r);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(yv);
    free(z);
    free(pz);
    return status;
}

int orc_gmres(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, int kind, int deg,
              const double *coef, const double *Hp, const double *yp, double betap, const double *b, double *x,
              double tol, int m, int maxit, double *stats, double *hist, int hist_cap)
{
    return orc_gmres_lu(n, rp, ci, va, NULL, kind, deg, coef, Hp, yp, betap, b, x, tol, m, maxit, stats, hist, hist_cap);
}

/* ------------------------------------------------------------------ */
/* s-step (communication-avoiding) GMRES with the polynomial (Section VII's combination)          */
/* ------------------------------------------------------------------ */

/* The same right-preconditioned GMRES(m) iterates as orc_gmres (in exact arithmetic), built s basis
 * vectors at a time: from the last basis vector q_k, a Newton basis z_{i+1} = (B - theta I) z_i / nu_i
 * (B = A p(A), nu_i = the norm, i < s) is formed with SpMVs only; the block Z = [z_1 .. z_s] is then
 * orthogonalised against Q = [q_0 .. q_k] by block classical Gram-Schmidt twice (C = Q^T Z, Z -= Q C),
 * and within itself by Cholesky QR (Z^T Z = R^T R, Q_new = Z R^{-1}).  With U+ = [q_k, z_1 .. z_s] =
 * [Q, Q_new] S (S: column 0 = e_k, column i = [C_i; R_i]) and B U = U+ T (T: theta on the diagonal,
 * nu_i below it), the Arnoldi relation gives the block's Hessenberg columns
 *     H[:, k .. k+s-1] = (S T - [H_old S_a; 0]) S_b^{-1},
 * S_a = S's rows 0 .. k-1 and S_b its rows k .. k+s-1 (upper triangular) over columns 0 .. s-1,
 * H_old = the Hessenberg columns 0 .. k-1 (rows 0 .. k).  The columns then go through the Givens
 * rotations one by one, as in orc_gmres.  A Newton vector of norm 0 or a Cholesky pivot that is not
 * positive shortens the block to the vectors before it; an empty block is a breakdown (the cycle ends).
 * stats as orc_gmres, with stats[3] = global reductions: one per Newton norm, two block inner products
 * and one Gram matrix per block, one per true residual.  h_first (optional, (m+1) x m column-major)
 * receives the first cycle's Hessenberg matrix as built (before the rotations), its other entries zero. */
int orc_sstep_gmres(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, int kind, int deg,
                    const double *coef, const double *Hp, const double *yp, double betap, const double *b, double *x,
                    double tol, int m, int maxit, int s, double theta, double *stats, double *hist, int hist_cap,
                    double *h_first)
{
    csr_t A = {n, rp, ci, va, NULL};
    poly_t p = {kind, deg, coef, Hp, yp, betap};
    op_t op = {&A, &p, {0}, dalloc(n), 0};
    if (s < 1) s = 1;
    if (s > m) s = m;
    const int ldh = m + 1;
    double *V = dalloc(n * (m + 1));
    double *Z = dalloc(n * s);
    double *r = dalloc(n);
    double *Hraw = dalloc((int64_t)ldh * m), *R = dalloc((int64_t)ldh * m);
    double *cs = dalloc(m), *sn = dalloc(m), *g = dalloc(m + 1), *yv = dalloc(m);
    double *nu = dalloc(s), *C = dalloc((int64_t)(m + 1) * s), *C2 = dalloc((int64_t)(m + 1) * s);
    double *G = dalloc((int64_t)s * s), *S = dalloc((int64_t)(m + 1 + s) * (s + 1));
    double *Hb = dalloc((int64_t)(m + 1 + s) * s), *zc = dalloc(n), *pz = dalloc(n);
    int ok = (poly_ws_init(&op.ws, n, &p) == 0) && op.z && V && Z && r && Hraw && R && cs && sn && g && yv && nu &&
             C && C2 && G && S && Hb && zc && pz;
    for (int i = 0; i < ORC_NSTATS; ++i) stats[i] = 0.0;
    int status = -2;
    if (!ok) goto out;

    double bnorm = nrm2(n, b);
    long iters = 0, cycles = 0, dots = 0, brk_count = 0;
    int converged = 0;
    double relres = 0.0, est = 0.0;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * (size_t)n);
        converged = 1;
        goto done;
    }
    for (;;) {
        spmv(&A, x, r);
        op.spmvs += 1;
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double beta = nrm2(n, r);
        dots += 1;
        relres = beta / bnorm;
        if (relres <= tol) {
            converged = 1;
            break;
        }
        if (iters >= maxit) break;
        cycles += 1;
        for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int k = 0, stop = 0;
        while (k < m && !stop) {
            int sb = s;
            if (sb > m - k) sb = m - k;
            if (sb > maxit - iters) sb = (int)(maxit - iters);
            /* Newton basis from q_k */
            const double *zp = V + (int64_t)k * n;
            int got = 0;
            for (int i = 0; i < sb; ++i) {
                double *zi = Z + (int64_t)i * n;
                op_apply(&op, zp, zi);
                axpy(n, -theta, zp, zi);
                double v = nrm2(n, zi);
                dots += 1;
                if (!(v > 0.0) || !isfinite(v)) break;
                nu[i] = v;
                scal(n, 1.0 / v, zi);
                zp = zi;
                got = i + 1;
            }
            sb = got;
            /* block classical Gram-Schmidt, twice: C = Q^T Z, Z -= Q C */
            for (int c = 0; c <= k; ++c)
                for (int i = 0; i < sb; ++i) C[c + i * (m + 1)] = 0.0;
            for (int pass = 0; pass < 2 && sb > 0; ++pass) {
                for (int i = 0; i < sb; ++i)
                    for (int c = 0; c <= k; ++c)
                        C2[c + i * (m + 1)] = dot(n, V + (int64_t)c * n, Z + (int64_t)i * n);
                dots += 1;
                for (int i = 0; i < sb; ++i)
                    for (int c = 0; c <= k; ++c) {
                        axpy(n, -C2[c + i * (m + 1)], V + (int64_t)c * n, Z + (int64_t)i * n);
                        C[c + i * (m + 1)] += C2[c + i * (m + 1)];
                    }
            }
            /* Cholesky QR of the block: G = Z^T Z = R^T R (R upper, in G's upper triangle) */
            if (sb > 0) {
                for (int i = 0; i < sb; ++i)
                    for (int j = 0; j < sb; ++j) G[i + j * s] = dot(n, Z + (int64_t)i * n, Z + (int64_t)j * n);
                dots += 1;
                /* column-by-column Cholesky (the lower factor L = R^T, as orc_cholesky) */
                int fact = sb;
                for (int j = 0; j < sb && fact == sb; ++j) {
                    double d = G[j + j * s];
                    for (int q = 0; q < j; ++q) d -= G[j + q * s] * G[j + q * s];
                    /* the Newton vectors have norm 1 before the projections, and Z^T Z resolves a
                     * remainder's squared norm to about the unit roundoff: a pivot below the breakdown
                     * threshold (a remainder below 1e-7) means z_j lies in the span already built */
                    if (!(d > ORC_BREAKDOWN)) {
                        fact = j;
                        break;
                    }
                    d = sqrt(d);
                    G[j + j * s] = d;
                    for (int i = j + 1; i < sb; ++i) {
                        double v = G[i + j * s];
                        for (int q = 0; q < j; ++q) v -= G[i + q * s] * G[j + q * s];
                        G[i + j * s] = v / d;
                    }
                }
                sb = fact;
            }
            if (sb == 0) { /* B q_k = theta q_k + nu_0 z_1 lies in span(Q): a lucky breakdown, column k of
                            * H is theta e_k + nu_0 C[:, 0] with a zero subdiagonal entry */
                double *hc = Hraw + (int64_t)k * ldh;
                for (int i = 0; i <= m; ++i) hc[i] = 0.0;
                if (got > 0)
                    for (int c = 0; c <= k; ++c) hc[c] = nu[0] * C[c];
                hc[k] += theta;
                double *rc = R + (int64_t)k * ldh;
                for (int i = 0; i <= k + 1; ++i) rc[i] = hc[i];
                for (int i = 0; i < k; ++i) rot(cs[i], sn[i], &rc[i], &rc[i + 1]);
                rc[k] = make_rot(rc[k], rc[k + 1], &cs[k], &sn[k]);
                rc[k + 1] = 0.0;
                rot(cs[k], sn[k], &g[k], &g[k + 1]);
                iters += 1;
                k += 1;
                est = fabs(g[k]) / bnorm;
                if (hist && iters <= hist_cap) hist[iters - 1] = est;
                brk_count += 1;
                break;
            }
            /* Q_new = Z R^{-1}, R = L^T: column i of Q_new = (z_i - sum_{q<i} R[q,i] Q_new_q) / R[i,i] */
            for (int i = 0; i < sb; ++i) {
                double *qi = V + (int64_t)(k + 1 + i) * n;
                memcpy(qi, Z + (int64_t)i * n, sizeof(double) * (size_t)n);
                for (int q = 0; q < i; ++q) axpy(n, -G[i + q * s], V + (int64_t)(k + 1 + q) * n, qi);
                scal(n, 1.0 / G[i + i * s], qi);
            }
            /* S ((k+1+sb) x (sb+1)) and the block's Hessenberg columns */
            const int ns = k + 1 + sb;
            for (int i = 0; i < ns * (sb + 1); ++i) S[i] = 0.0;
            S[k] = 1.0;
            for (int i = 1; i <= sb; ++i) {
                for (int c = 0; c <= k; ++c) S[c + i * ns] = C[c + (i - 1) * (m + 1)];
                for (int q = 0; q < i; ++q) S[k + 1 + q + i * ns] = G[(i - 1) + q * s]; /* R[q, i-1] = L[i-1, q] */
            }
            /* Hb = S T - [H_old S_a; 0]   (ns x sb) */
            for (int j = 0; j < sb; ++j)
                for (int i = 0; i < ns; ++i) {
                    double v = theta * S[i + j * ns] + nu[j] * S[i + (j + 1) * ns];
                    if (i <= k)
                        for (int q = 0; q < k; ++q) v -= Hraw[i + (int64_t)q * ldh] * S[q + j * ns];
                    Hb[i + j * ns] = v;
                }
            /* Hb := Hb S_b^{-1} (S_b = S rows k .. k+sb-1, columns 0 .. sb-1, upper triangular) */
            for (int j = 0; j < sb; ++j) {
                const double d = S[k + j + j * ns];
                for (int i = 0; i < ns; ++i) {
                    double v = Hb[i + j * ns];
                    for (int q = 0; q < j; ++q) v -= Hb[i + q * ns] * S[k + q + j * ns];
                    Hb[i + j * ns] = v / d;
                }
            }
            /* the new columns through the Givens rotations, one iteration each */
            for (int j = 0; j < sb; ++j) {
                const int col = k + j;
                double *hc = Hraw + (int64_t)col * ldh, *rc = R + (int64_t)col * ldh;
                for (int i = 0; i <= m; ++i) hc[i] = 0.0;
                for (int i = 0; i <= col + 1 && i < ns; ++i) hc[i] = Hb[i + j * ns];
                for (int i = 0; i <= col + 1; ++i) rc[i] = hc[i];
                for (int i = 0; i < col; ++i) rot(cs[i], sn[i], &rc[i], &rc[i + 1]);
                rc[col] = make_rot(rc[col], rc[col + 1], &cs[col], &sn[col]);
                rc[col + 1] = 0.0;
                rot(cs[col], sn[col], &g[col], &g[col + 1]);
                iters += 1;
                est = fabs(g[col + 1]) / bnorm;
                if (hist && iters <= hist_cap) hist[iters - 1] = est;
                if (est <= tol || iters >= maxit) {
                    k = col + 1;
                    stop = 1;
                    break;
                }
            }
            if (!stop) k += sb;
        }
        if (h_first && cycles == 1) /* the first cycle's columns 0 .. k-1 as built (rows 0 .. j+1 of column j) */
            for (int j = 0; j < m; ++j)
                for (int i = 0; i <= m; ++i)
                    h_first[i + (int64_t)j * ldh] = (j < k && i <= j + 1) ? Hraw[i + (int64_t)j * ldh] : 0.0;
        /* y = R^{-1} g over the k columns, x += p(A) V y */
        for (int i = k - 1; i >= 0; --i) {
            double v = g[i];
            for (int q = i + 1; q < k; ++q) v -= R[i + (int64_t)q * ldh] * yv[q];
            yv[i] = v / R[i + (int64_t)i * ldh];
        }
        memset(zc, 0, sizeof(double) * (size_t)n);
        for (int i = 0; i < k; ++i) axpy(n, yv[i], V + (int64_t)i * n, zc);
        op.spmvs += poly_apply(&A, &p, zc, pz, &op.ws);
        axpy(n, 1.0, pz, x);
    }
done:
    stats[0] = (double)iters;
    stats[1] = (double)cycles;
    stats[2] = (double)op.spmvs;
    stats[3] = (double)dots;
    stats[4] = converged ? 1.0 : 0.0;
    stats[5] = relres;
    stats[6] = est;
    stats[7] = (double)brk_count;
    status = converged ? 0 : 1;
out:
    poly_ws_free(&op.ws);
    free(op.z);
    free(V);
    free(Z);
    free(r);
    free(Hraw);
    free(R);
    free(cs);
    free(sn);
    free(g);
    free(yv);
    free(nu);
    free(C);
    free(C2);
    free(G);
    free(S);
    free(Hb);
    free(zc);
    free(pz);
    return status;
}
