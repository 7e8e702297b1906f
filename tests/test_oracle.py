"""Pins for the CPU oracle: each test checks it against something other than itself.

The pins are closed forms, library routines (dense solves, least squares,
LAPACK's POTRF), invariants of Arnoldi and GMRES, and the values the paper
prints for its Section V Laplacian example (tests/golden/).
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg.lapack as lapack

import oracle
import workloads as w

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rand_dd(n, seed, shift=0.5, per_row=5):
    return w.random_csr(n, per_row, seed, diag_shift=shift)


# ---------------------------------------------------------------- SpMV / transpose


def test_spmv_matches_dense_product():
    a = _rand_dd(300, 11)
    x = w.uniform(12, a.n)
    np.testing.assert_allclose(oracle.spmv(a, x), a.to_dense() @ x, rtol=1e-14, atol=1e-13)


def test_spmv_rows_matches_full_product():
    a = w.c1_matrix()
    x = w.uniform(13, a.n)
    rows = np.array([0, 1, 63, 64, 2047, 4095])
    np.testing.assert_array_equal(oracle.spmv_rows(a, x, rows), oracle.spmv(a, x)[rows])


def test_transpose_matches_scipy():
    a = _rand_dd(257, 14)
    t = oracle.transpose(a)
    ref = a.to_scipy().T.tocsr()
    ref.sort_indices()
    np.testing.assert_array_equal(t.rowptr, ref.indptr)
    np.testing.assert_array_equal(t.colidx, ref.indices)
    np.testing.assert_array_equal(t.vals, ref.data)


# ---------------------------------------------------------------- Cholesky (POTRF semantics)


def test_cholesky_matches_lapack_on_spd():
    rng = np.random.default_rng(0)
    for k in (1, 2, 5, 11, 41):
        b = rng.standard_normal((k, k))
        g = b @ b.T + k * np.eye(k)
        l, info = oracle.cholesky(g)
        assert info == 0
        np.testing.assert_allclose(l, np.linalg.cholesky(g), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("j", [1, 2, 4, 7, 10])
def test_cholesky_info_matches_lapack(j):
    rng = np.random.default_rng(j)
    k = 10
    b = rng.standard_normal((k, k))
    g = b @ b.T + np.eye(k)
    # make the leading minor of order j indefinite: shrink its last diagonal entry
    # below the Schur complement of the leading (j-1) block
    g[j - 1, j - 1] -= 1.5 * g[j - 1, j - 1]
    _, info_lapack = lapack.dpotrf(g, lower=1)
    _, info = oracle.cholesky(g)
    assert info_lapack == j
    assert info == info_lapack


def test_cholesky_info_on_nan():
    g = np.eye(4)
    g[2, 2] = np.nan
    _, info = oracle.cholesky(g)
    assert info == 3


# ---------------------------------------------------------------- the polynomial: closed form


def _elementary_symmetric(vals):
    """e_0..e_k of vals (coefficients of prod (1 + v t))."""
    e = np.zeros(len(vals) + 1)
    e[0] = 1.0
    for v in vals:
        e[1:] = e[1:] + v * e[:-1]
    return e


def _diag_matrix(lams, reps):
    d = np.repeat(np.asarray(lams, dtype=np.float64), reps)
    n = len(d)
    return w.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d, "diag")


@pytest.mark.parametrize("lams", [[2.0, 5.0], [1.0, 3.0, 4.5], [0.5, 1.5, 2.5, 7.0], [1.0, 2.0, 3.0, 5.0, 8.0]])
def test_poly_is_exact_interpolant_when_degree_reaches_spectrum(lams):
    """With d+1 distinct eigenvalues, 1 - z p(z) = prod (1 - z/lambda_i) exactly, so
    coef[j] = (-1)^j e_{j+1}(1/lambda) and p(A) = A^{-1} (Section II, Eqs. 1-2)."""
    d = len(lams) - 1
    a = _diag_matrix(lams, 7)
    v0 = w.uniform(21, a.n)
    e = _elementary_symmetric(1.0 / np.asarray(lams))
    expect = np.array([(-1.0) ** j * e[j + 1] for j in range(d + 1)])

    pn = oracle.poly_normal_eq(a, v0, d)
    assert pn.info == 0 and pn.used == d
    # the normal equations square the power basis' condition number: allow for it
    np.testing.assert_allclose(pn.coef, expect, rtol=1e-6)

    pg = oracle.poly_gmres(a, v0, d)
    assert pg.deg == d
    assert pg.resid < 1e-10 * np.linalg.norm(v0)
    np.testing.assert_allclose(oracle.arnoldi_to_power(pg), expect, rtol=1e-9)

    x = w.uniform(22, a.n)
    exact = x / a.vals
    np.testing.assert_allclose(oracle.poly_apply(a, pn, x), exact, rtol=1e-6)
    np.testing.assert_allclose(oracle.poly_apply(a, pg, x), exact, rtol=1e-9)
    # scalar evaluation: alpha p(alpha) = 1 at every eigenvalue
    np.testing.assert_allclose(oracle.poly_eval_zp(pn, lams), 1.0, rtol=1e-6)
    np.testing.assert_allclose(oracle.poly_eval_zp(pg, lams), 1.0, rtol=1e-9)


def test_poly_breakdown_gives_exact_lower_degree():
    """Asking for a higher degree than the spectrum supports: the Arnoldi run breaks down
    and the exact polynomial of lower degree is returned."""
    lams = [1.0, 4.0]
    a = _diag_matrix(lams, 5)
    v0 = w.uniform(23, a.n)
    pg = oracle.poly_gmres(a, v0, 4)
    assert pg.deg == 1
    np.testing.assert_allclose(oracle.arnoldi_to_power(pg), [1.25, -0.25], rtol=1e-9)


# ---------------------------------------------------------------- the polynomial: optimality


@pytest.mark.parametrize("deg", [1, 2, 3, 4, 5])
def test_poly_minimises_residual_like_least_squares(deg):
    """||v0 - A p(A) v0|| is the least-squares minimum over the Krylov space (Eq. 1)."""
    a = _rand_dd(80, 31, shift=1.0)
    ad = a.to_dense()
    v0 = w.uniform(32, a.n)
    K = np.empty((a.n, deg + 1))
    t = v0.copy()
    for j in range(deg + 1):
        t = ad @ t
        K[:, j] = t
    c, *_ = np.linalg.lstsq(K, v0, rcond=None)
    best = np.linalg.norm(v0 - K @ c)

    pg = oracle.poly_gmres(a, v0, deg)
    assert abs(pg.resid - best) <= 1e-10 * np.linalg.norm(v0)
    r_arn = np.linalg.norm(v0 - oracle.spmv(a, oracle.poly_apply(a, pg, v0)))
    assert abs(r_arn - best) <= 1e-10 * np.linalg.norm(v0)

    pn = oracle.poly_normal_eq(a, v0, deg)
    r_ne = np.linalg.norm(v0 - oracle.spmv(a, oracle.poly_apply(a, pn, v0)))
    assert r_ne >= best * (1 - 1e-12)
    assert r_ne <= best * (1 + 1e-6)
    if deg <= 3:
        np.testing.assert_allclose(pn.coef, c, rtol=1e-7)
        np.testing.assert_allclose(oracle.arnoldi_to_power(pg), c, rtol=1e-7)


def test_power_and_arnoldi_forms_apply_the_same_polynomial():
    a = w.c1_matrix()
    v0 = w.v0(a.n)
    x = w.uniform(41, a.n)
    for deg in (2, 5, 8):
        pg = oracle.poly_gmres(a, v0, deg)
        pp = oracle.Poly(oracle.POLY_POWER, deg, oracle.arnoldi_to_power(pg))
        ya = oracle.poly_apply(a, pg, x)
        yp = oracle.poly_apply(a, pp, x)
        assert np.linalg.norm(ya - yp) <= 1e-7 * np.linalg.norm(ya)


def test_power_basis_degree_limit_section4():
    """Section IV: POTRF warns (info > 0) from about degree 10-12 on; the degree used is
    the largest one whose Gram matrix still factors, and its coefficients equal those of
    a direct construction at that degree."""
    a = w.c1_matrix()
    v0 = w.v0(a.n)
    first_fail = None
    for deg in range(4, 20):
        p = oracle.poly_normal_eq(a, v0, deg)
        if p.info > 0:
            first_fail = deg
            assert p.used == p.info - 2
            direct = oracle.poly_normal_eq(a, v0, p.used)
            np.testing.assert_array_equal(direct.coef, p.coef)
            break
    assert first_fail is not None and 8 <= first_fail <= 14


# ---------------------------------------------------------------- Arnoldi


def test_arnoldi_relation_and_orthogonality():
    a = w.c1_matrix()
    pg = oracle.poly_gmres(a, w.v0(a.n), 5)
    b = w.rhs(a.n)
    k = 30
    V, H, beta, done = oracle.arnoldi(a, pg, b, k)
    assert done == k
    AV = np.column_stack([oracle.spmv(a, oracle.poly_apply(a, pg, V[:, j])) for j in range(k)])
    rel = np.linalg.norm(AV - V @ H) / np.linalg.norm(H)
    assert rel <= 1e-12
    # modified Gram-Schmidt keeps orthogonality only to O(u * cond), not to u
    assert np.linalg.norm(np.eye(k + 1) - V.T @ V) <= 1e-8
    assert np.allclose(np.tril(H, -2), 0.0)


# ---------------------------------------------------------------- GMRES


def _dense_solve(a, b):
    return np.linalg.solve(a.to_dense(), b)


@pytest.mark.parametrize("case", ["convdiff", "random"])
def test_gmres_matches_dense_solve(case):
    a = w.convdiff(14, 2, 10.0) if case == "convdiff" else _rand_dd(200, 51, shift=0.2)
    b = w.rhs(a.n)
    xd = _dense_solve(a, b)
    v0 = w.v0(a.n)
    polys = [oracle.IDENTITY, oracle.poly_normal_eq(a, v0, 3), oracle.poly_gmres(a, v0, 8)]
    for p in polys:
        r = oracle.gmres(a, b, p, tol=1e-12, m=20, maxit=2000)
        assert r.converged
        assert np.linalg.norm(r.x - xd) <= 1e-10 * np.linalg.norm(xd)
        assert r.relres <= 1e-12


def test_gmres_first_cycle_residuals_are_krylov_minima():
    """Iteration k's estimate equals min ||b - M K_k c|| over the Krylov space of M = A p(A)."""
    a = _rand_dd(120, 61, shift=0.3)
    b = w.rhs(a.n)
    for p in (oracle.IDENTITY, oracle.poly_gmres(a, w.v0(a.n), 3)):
        M = np.column_stack([oracle.spmv(a, oracle.poly_apply(a, p, e)) for e in np.eye(a.n)])
        r = oracle.gmres(a, b, p, tol=1e-14, m=30, maxit=6)
        t = b.copy()
        K = []
        for k in range(1, 7):
            K.append(t)
            Kk = np.column_stack(K)
            Q, _ = np.linalg.qr(Kk)
            MQ = M @ Q
            c, *_ = np.linalg.lstsq(MQ, b, rcond=None)
            best = np.linalg.norm(b - MQ @ c) / np.linalg.norm(b)
            assert abs(r.hist[k - 1] - best) <= 1e-9 * max(best, 1e-3)
            t = M @ t


def test_degree_zero_is_unpreconditioned_gmres():
    """Section III: degree 0 means no preconditioning (a scalar p leaves GMRES unchanged)."""
    a = w.c1_matrix()
    b = w.rhs(a.n)
    p0 = oracle.poly_normal_eq(a, w.v0(a.n), 0)
    r0 = oracle.gmres(a, b, p0, tol=1e-8, m=50, maxit=3000)
    ri = oracle.gmres(a, b, oracle.IDENTITY, tol=1e-8, m=50, maxit=3000)
    assert r0.iters == ri.iters
    assert np.linalg.norm(r0.x - ri.x) <= 1e-7 * np.linalg.norm(ri.x)


def test_gmres_zero_rhs_and_converged_start():
    a = w.c1_matrix()
    r = oracle.gmres(a, np.zeros(a.n), oracle.IDENTITY, tol=1e-8, m=10, maxit=10)
    assert r.converged and r.iters == 0 and not r.x.any()
    b = w.rhs(a.n)
    xd = _dense_solve(a, b)
    r = oracle.gmres(a, b, oracle.IDENTITY, tol=1e-8, m=10, maxit=10, x0=xd)
    assert r.converged and r.iters == 0


def test_gmres_maxit_stops_unconverged():
    a = w.c1_matrix()
    r = oracle.gmres(a, w.rhs(a.n), oracle.IDENTITY, tol=1e-8, m=50, maxit=7)
    assert not r.converged and r.iters == 7 and r.relres > 1e-8


def test_transposed_solve_matches_dense():
    a = w.convdiff(12, 2, 30.0)
    g = w.uniform(71, a.n)
    at = oracle.transpose(a)
    p = oracle.poly_gmres(a, w.v0(a.n), 4)
    r = oracle.gmres(at, g, p, tol=1e-12, m=30, maxit=2000)
    lam = np.linalg.solve(a.to_dense().T, g)
    assert np.linalg.norm(r.x - lam) <= 1e-10 * np.linalg.norm(lam)


def test_dense_gradient_formula_matches_finite_differences():
    """L = ||x - x_t||^2 with A x = b: dL/db = lambda, dL/dA_ij = -lambda_i x_j where
    A^T lambda = 2 (x - x_t).  Central differences on a tiny dense problem."""
    a = w.convdiff(5, 2, 20.0)
    A = a.to_dense()
    b = w.rhs(a.n)
    xt = w.uniform(w.SEED_XTARGET, a.n)

    def loss(A_, b_):
        x_ = np.linalg.solve(A_, b_)
        return float(np.sum((x_ - xt) ** 2))

    x = np.linalg.solve(A, b)
    lam = np.linalg.solve(A.T, 2 * (x - xt))
    h = 1e-6
    for i in (0, 7, 24):
        e = np.zeros(a.n)
        e[i] = h
        fd = (loss(A, b + e) - loss(A, b - e)) / (2 * h)
        assert abs(fd - lam[i]) <= 1e-6 * max(1.0, abs(lam[i]))
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    for kk in (0, 13, 40, a.nnz - 1):
        i, j = rows[kk], a.colidx[kk]
        E = np.zeros_like(A)
        E[i, j] = h
        fd = (loss(A + E, b) - loss(A - E, b)) / (2 * h)
        assert abs(fd - (-lam[i] * x[j])) <= 1e-6 * max(1.0, abs(lam[i] * x[j]))


# ---------------------------------------------------------------- the paper's examples


@pytest.fixture(scope="module")
def lap5():
    return w.laplacian2d(201)


def test_laplacian_random_v0_iterations(lap5, golden_dir):
    """Section V: random v0, degree 5, GMRES(50) converges in 148 iterations."""
    gold = json.load(open(os.path.join(golden_dir, "laplacian_section5.json")))
    a = lap5
    assert a.n == 40401
    b = np.ones(a.n)
    p = oracle.poly_normal_eq(a, w.v0(a.n), gold["degree"])
    r = oracle.gmres(a, b, p, tol=gold["tol"], m=gold["restart"], maxit=2000)
    g = gold["random_v0_iterations"]
    assert r.converged
    assert abs(r.iters - g["value"]) <= g["tolerance"]
    bulk = gold["random_v0_bulk_range"]
    zs = np.linspace(bulk["alpha_lo"], bulk["alpha_hi"], 200)
    vals = oracle.poly_eval_zp(p, zs)
    assert vals.min() >= bulk["lo"] and vals.max() <= bulk["hi"]


def test_laplacian_v0_b_polynomial_maps_8_near_minus_1400(lap5, golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "laplacian_section5.json")))
    a = lap5
    b = np.ones(a.n)
    p = oracle.poly_normal_eq(a, b, gold["degree"])
    g = gold["v0_is_b_alpha_p_alpha_at_8"]
    val = oracle.poly_eval_zp(p, 8.0)[0]
    assert abs(val - g["value"]) <= g["rel_tolerance"] * abs(g["value"])


@pytest.mark.slow
def test_laplacian_v0_b_stalls_at_0856(lap5, golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "laplacian_section5.json")))
    a = lap5
    b = np.ones(a.n)
    p = oracle.poly_normal_eq(a, b, gold["degree"])
    r = oracle.gmres(a, b, p, tol=gold["tol"], m=gold["restart"], maxit=2550)
    g = gold["v0_is_b_relres_after_2550"]
    assert not r.converged and r.iters == 2550
    assert abs(r.relres - g["value"]) <= g["tolerance"]


@pytest.mark.parametrize("name", ["BiDiag1", "BiDiag2"])
def test_bidiag_matrices_converge(name, golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "bidiag_section4.json")))
    a = w.bidiag1() if name == "BiDiag1" else w.bidiag2()
    assert a.n == gold[name]["n"]
    xs = w.uniform(81, a.n)
    b = oracle.spmv(a, xs)
    for deg in gold["degrees"]:
        p = oracle.poly_normal_eq(a, b, deg)
        r = oracle.gmres(a, b, p, tol=1e-8, m=50, maxit=20000)
        assert r.converged
        true = np.linalg.norm(b - a.to_scipy() @ r.x) / np.linalg.norm(b)
        assert true <= 1e-8


# ---------------------------------------------------------------- ILU(0) on the left (Section VI)


def _lu_dense(a, lu):
    """Dense unit-lower L and upper U from the oracle's ILU(0) array on a's pattern."""
    L = np.eye(a.n)
    U = np.zeros((a.n, a.n))
    for i in range(a.n):
        for t in range(a.rowptr[i], a.rowptr[i + 1]):
            j = a.colidx[t]
            if j < i:
                L[i, j] = lu[t]
            else:
                U[i, j] = lu[t]
    return L, U


def test_ilu0_is_the_exact_lu_without_fill():
    """A tridiagonal matrix has no fill, so ILU(0) is its exact LU factorisation: L U = A."""
    a = w.convdiff(60, 1, 20.0)
    lu = oracle.ilu0(a)
    L, U = _lu_dense(a, lu)
    np.testing.assert_allclose(L @ U, a.to_dense(), rtol=0, atol=1e-13 * np.abs(a.vals).max())
    # then M^{-1} A = I: GMRES with ILU(0) on the left converges in one iteration
    b = w.rhs(a.n)
    r = oracle.gmres(a, b, oracle.IDENTITY, tol=1e-12, m=20, lu=lu)
    assert r.converged and r.iters == 1


@pytest.mark.parametrize("case", ["convdiff2d", "random"])
def test_ilu0_reproduces_a_on_its_pattern(case):
    """The defining property of ILU(0): (L U)_ij = a_ij wherever a has an entry (the products that
    fall outside the pattern are the dropped fill, which is not zero here)."""
    a = w.convdiff(12, 2, 30.0) if case == "convdiff2d" else _rand_dd(150, 71, shift=3.0)
    lu = oracle.ilu0(a)
    L, U = _lu_dense(a, lu)
    P = L @ U
    ad = a.to_dense()
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    scale = np.abs(a.vals).max()
    assert np.abs(P[rows, a.colidx] - a.vals).max() <= 1e-12 * scale
    mask = np.ones_like(ad, dtype=bool)
    mask[rows, a.colidx] = False
    assert np.abs(P[mask]).max() > 1e-6 * scale  # fill was dropped: M is not A


def test_ilu0_apply_inverts_lu():
    a = w.convdiff(12, 2, 30.0)
    lu = oracle.ilu0(a)
    L, U = _lu_dense(a, lu)
    x = w.uniform(72, a.n)
    y = oracle.ilu0_apply(a, lu, x)
    np.testing.assert_allclose(L @ (U @ y), x, rtol=0, atol=1e-12 * np.abs(x).max())


@pytest.mark.parametrize("deg", [1, 3, 5])
def test_poly_of_the_ilu_preconditioned_operator_is_minimal(deg):
    """With ILU(0) the polynomial is the minimum-residual polynomial of B = M^{-1} A: ||v0 - B p(B) v0|| is
    the least-squares minimum over B's Krylov space, and the three routes agree."""
    a = _rand_dd(90, 73, shift=2.0)
    lu = oracle.ilu0(a)
    L, U = _lu_dense(a, lu)
    B = np.linalg.solve(U, np.linalg.solve(L, a.to_dense()))
    v0 = w.uniform(74, a.n)
    K = np.empty((a.n, deg + 1))
    t = v0.copy()
    for j in range(deg + 1):
        t = B @ t
        K[:, j] = t
    c, *_ = np.linalg.lstsq(K, v0, rcond=None)
    best = np.linalg.norm(v0 - K @ c)
    pg = oracle.poly_gmres(a, v0, deg, lu=lu)
    assert abs(pg.resid - best) <= 1e-10 * np.linalg.norm(v0)
    px = oracle.poly_apply(a, pg, v0, lu=lu)
    assert abs(np.linalg.norm(v0 - B @ px) - best) <= 1e-10 * np.linalg.norm(v0)
    pn = oracle.poly_normal_eq(a, v0, deg, lu=lu)
    if pn.info == 0:  # the power basis of B ~ I is ill-conditioned early: a clamped degree is checked below
        assert np.linalg.norm(v0 - B @ oracle.poly_apply(a, pn, v0, lu=lu)) <= best * (1 + 1e-6)
    else:
        assert pn.deg == pn.info - 2 < deg


def test_gmres_with_ilu_left_and_poly_right():
    """Section VI's composition: the solution solves A x = b (true residual), and the first cycle's
    estimates are the Krylov minima of M^{-1} A p(M^{-1} A) for the preconditioned residual M^{-1} b,
    relative to ||M^{-1} b||."""
    a = _rand_dd(120, 75, shift=0.8)
    lu = oracle.ilu0(a)
    L, U = _lu_dense(a, lu)
    Minv = lambda v: np.linalg.solve(U, np.linalg.solve(L, v))  # noqa: E731
    b = w.rhs(a.n)
    p = oracle.poly_gmres(a, w.v0(a.n), 3, lu=lu)
    r = oracle.gmres(a, b, p, tol=1e-10, m=40, maxit=500, lu=lu)
    assert r.converged
    np.testing.assert_allclose(a.to_dense() @ r.x, b, rtol=0, atol=1e-9 * np.linalg.norm(b))
    Bop = np.column_stack([Minv(a.to_dense() @ oracle.poly_apply(a, p, e, lu=lu)) for e in np.eye(a.n)])
    rb = Minv(b)
    h = oracle.gmres(a, b, p, tol=1e-14, m=30, maxit=5, lu=lu).hist
    assert len(h) >= 3
    t = rb.copy()
    Kl = []
    for k in range(1, len(h) + 1):
        Kl.append(t)
        Q, _ = np.linalg.qr(np.column_stack(Kl))
        BQ = Bop @ Q
        c, *_ = np.linalg.lstsq(BQ, rb, rcond=None)
        best = np.linalg.norm(rb - BQ @ c) / np.linalg.norm(rb)
        assert abs(h[k - 1] - best) <= 1e-9 * max(best, 1e-3)
        t = Bop @ t


# ---------------------------------------------------------------- s-step GMRES with the polynomial


def test_sstep_first_cycle_residuals_are_krylov_minima():
    """Each iteration of the s-step solver still minimises ||b - M c|| over the Krylov space of
    M = A p(A), checked by dense least squares on an orthonormal basis of that space, for blocks of
    1, 3 and 4 (the last one ragged against the 6 iterations)."""
    a = _rand_dd(120, 62, shift=0.3)
    b = w.rhs(a.n)
    p = oracle.poly_gmres(a, w.v0(a.n), 3)
    M = np.column_stack([oracle.spmv(a, oracle.poly_apply(a, p, e)) for e in np.eye(a.n)])
    best = []
    t, K = b.copy(), []
    for k in range(1, 7):
        K.append(t)
        Q, _ = np.linalg.qr(np.column_stack(K))
        c, *_ = np.linalg.lstsq(M @ Q, b, rcond=None)
        best.append(np.linalg.norm(b - M @ Q @ c) / np.linalg.norm(b))
        t = M @ t
    for s in (1, 3, 4):
        r, brk = oracle.sstep_gmres(a, b, p, s=s, theta=1.0, tol=1e-14, m=30, maxit=6)
        assert r.iters == 6 and brk == 0
        for k in range(6):
            assert abs(r.hist[k] - best[k]) <= 1e-9 * max(best[k], 1e-3), (s, k)


@pytest.mark.parametrize("s,theta", [(1, 0.0), (2, 1.0), (5, 1.0), (7, 0.5)])
def test_sstep_matches_dense_solve_and_standard_gmres(s, theta):
    """Restarted s-step GMRES (blocks that do not divide the restart length included) reaches the dense
    solution, with the iteration count of standard GMRES."""
    a = w.convdiff(12, 3, 20.0)
    b = w.rhs(a.n)
    xd = _dense_solve(a, b)
    p = oracle.poly_gmres(a, w.v0(a.n), 6)
    r, brk = oracle.sstep_gmres(a, b, p, s=s, theta=theta, tol=1e-10, m=9, maxit=2000)
    assert r.converged and brk == 0 and r.relres <= 1e-10
    assert np.linalg.norm(r.x - xd) <= 1e-8 * np.linalg.norm(xd)
    ref = oracle.gmres(a, b, p, tol=1e-10, m=9, maxit=2000)
    assert r.iters == ref.iters and r.restarts == ref.restarts


def test_sstep_reductions_per_block():
    """One global reduction per Newton norm, three per block (two Gram-Schmidt passes and the Gram
    matrix), one per true residual: 11 iterations in blocks of 5 with GMRES(30) are 3 blocks of 5 Newton
    vectors, 15 + 9 + 2 = 26 reductions."""
    a = w.convdiff(12, 3, 20.0)
    b = w.rhs(a.n)
    p = oracle.poly_gmres(a, w.v0(a.n), 6)
    r, _ = oracle.sstep_gmres(a, b, p, s=5, theta=1.0, tol=1e-10, m=30, maxit=2000)
    assert r.iters == 11 and r.restarts == 1 and r.dots == 26


def test_sstep_exhausted_krylov_space_is_a_lucky_breakdown():
    """A diagonal matrix with three distinct eigenvalues and no polynomial: the Krylov space has
    dimension 3, so the first block of 5 Newton vectors is rank 3 (a Cholesky pivot vanishes) and the
    solver stops after 3 iterations with the exact solution."""
    d = np.array([1.0, 2.0, 4.0] * 20)
    n = d.size
    a = w.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    b = w.rhs(n)
    r, _ = oracle.sstep_gmres(a, b, oracle.IDENTITY, s=5, theta=0.5, tol=1e-12, m=30, maxit=100)
    assert r.converged and r.iters == 3
    np.testing.assert_allclose(r.x, b / d, rtol=1e-10)


def test_sstep_zero_rhs_and_maxit():
    a = w.c1_matrix()
    r, _ = oracle.sstep_gmres(a, np.zeros(a.n), oracle.IDENTITY, s=4, tol=1e-8, m=10, maxit=10)
    assert r.converged and r.iters == 0 and not r.x.any()
    r, _ = oracle.sstep_gmres(a, w.rhs(a.n), oracle.IDENTITY, s=4, theta=1.0, tol=1e-8, m=50, maxit=7)
    assert not r.converged and r.iters == 7
    ref = oracle.gmres(a, w.rhs(a.n), oracle.IDENTITY, tol=1e-8, m=50, maxit=7)
    np.testing.assert_allclose(r.hist, ref.hist, rtol=1e-8)


def _dense_arnoldi_reorth(M, v, k):
    """k Arnoldi steps with the dense operator M from v, classical Gram-Schmidt applied twice (numpy)."""
    n = len(v)
    V = np.zeros((n, k + 1))
    H = np.zeros((k + 1, k))
    V[:, 0] = v / np.linalg.norm(v)
    for j in range(k):
        w_ = M @ V[:, j]
        for _ in range(2):
            h = V[:, : j + 1].T @ w_
            w_ = w_ - V[:, : j + 1] @ h
            H[: j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w_)
        V[:, j + 1] = w_ / H[j + 1, j]
    return H


@pytest.mark.parametrize("s,theta", [(1, 1.0), (3, 1.0), (4, 0.5), (7, 1.0)])
def test_sstep_hessenberg_equals_arnoldis(s, theta):
    """The first cycle's Hessenberg matrix recovered block by block from the change of basis equals the
    one Arnoldi builds from b with the explicit dense operator A p(A) and reorthogonalisation (both
    bases are orthonormal with positive subdiagonal entries, so unique), for blocks that do and do not
    divide the 9 columns; and the oracle's own MGS Arnoldi's, whose orthogonality loss grows about tenfold
    per column here (1e-9 by the ninth).  Blocks of 1 and 3 agree with the dense reference to 1e-13;
    larger blocks to about 1e-10, the precision Cholesky QR of a Newton block keeps (kappa(Z)^2 u)."""
    a = w.convdiff(10, 3, 20.0)
    b = w.rhs(a.n)
    p = oracle.poly_gmres(a, w.v0(a.n), 5)
    M = np.column_stack([oracle.spmv(a, oracle.poly_apply(a, p, e)) for e in np.eye(a.n)])
    k = 9
    _, _, H_s = oracle.sstep_gmres(a, b, p, s=s, theta=theta, tol=1e-15, m=k, maxit=k, want_h=True)
    H_d = _dense_arnoldi_reorth(M, b, k)
    _, H_a, _, steps = oracle.arnoldi(a, p, b, k)
    assert steps == k and H_s.shape == H_d.shape == H_a.shape == (k + 1, k)
    scale = np.abs(H_d).max()
    np.testing.assert_allclose(H_s, H_d, rtol=0, atol=(1e-12 if s <= 3 else 1e-9) * scale)
    np.testing.assert_allclose(H_s, H_a, rtol=0, atol=1e-8 * scale)
