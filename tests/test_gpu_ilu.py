"""ILU(0) on the left of the polynomial (Section VI) on the GPU, against the oracle.

The factors are compared bit for bit (both evaluate the same row-by-row loops in float64 without
fused multiply-adds); the composed operator's polynomial application and the composed solve
M^{-1} A p(M^{-1} A) u = M^{-1} b are compared with the oracle's: true relative residual <= 1e-8,
solution within 1e-6 of the oracle's, iterations within max(5%, 1) in float64.
"""
import numpy as np
import pytest

import oracle
import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="no CUDA device")]

import paper_1907_00072_gb300 as ppg  # noqa: E402

DEV = "cuda:0"

MATS = {
    "c1": w.c1_matrix,
    "3d_7pt_21": lambda: w.convdiff(21, 3, 50.0),
    "27pt_12": lambda: w.stencil27_perturbed(12),
    "random": lambda: w.random_csr(3001, 6, 17, diag_shift=2.0),
}


def _T(a, dt=None):
    a = np.asarray(a)
    if dt is None:
        dt = torch.float64 if a.dtype.kind == "f" else torch.int32
    return torch.as_tensor(a, dtype=dt, device=DEV)


def _solver(a):
    return ppg.Solver(_T(a.rowptr, torch.int32), _T(a.colidx, torch.int32), _T(a.vals))


def _relres(a, b, x):
    return np.linalg.norm(b - oracle.spmv(a, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("mat", list(MATS))
def test_ilu0_factors_equal_the_oracles(mat):
    a = MATS[mat]()
    s = _solver(a)
    lu = s.set_left_ilu0(1, want_factors=True).cpu().numpy()
    np.testing.assert_array_equal(lu, oracle.ilu0(a))
    # ppg_spmv keeps computing A x with ILU(0) on
    x = w.uniform(81, a.n)
    y = s.spmv(_T(x)).cpu().numpy()
    np.testing.assert_allclose(y, oracle.spmv(a, x), rtol=1e-13, atol=1e-13 * np.abs(y).max())
    s.close()


@pytest.mark.parametrize("mat", ["c1", "3d_7pt_21", "27pt_12"])
@pytest.mark.parametrize("deg", [0, 5, 12])
def test_composed_solve_matches_the_oracle(mat, deg):
    a = MATS[mat]()
    b = w.rhs(a.n)
    v0 = w.v0(a.n)
    lu = oracle.ilu0(a)
    s = _solver(a)
    s.set_left_ilu0(1)
    used, _ = s.build_poly(deg, ppg.PPG_BASIS_ROOTS, v0=_T(v0))
    assert used == deg
    p = oracle.poly_gmres(a, v0, deg, lu=lu)
    # p(M^{-1} A) applied
    x = w.uniform(82, a.n)
    y = s.apply_poly(_T(x)).cpu().numpy()
    ref = oracle.poly_apply(a, p, x, lu=lu)
    assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(ref)
    # the composed solve
    r = oracle.gmres(a, b, p, tol=1e-8, m=50, maxit=3000, lu=lu)
    assert r.converged
    xg, info = s.solve(_T(b), tol=1e-8, restart=50, maxit=3000)
    xg = xg.cpu().numpy()
    it = info.stats["iterations"]
    assert info.status == ppg.PPG_OK and _relres(a, b, xg) <= 1e-8
    assert np.linalg.norm(xg - r.x) <= 1e-6 * np.linalg.norm(r.x)
    assert abs(it - r.iters) <= max(1, 0.05 * r.iters), (it, r.iters)
    # float32 inner solve with float64 refinement (the standard form runs with ILU(0))
    x32, i32 = s.solve(_T(b), tol=1e-8, restart=50, maxit=3000, precision=ppg.PPG_F32)
    x32 = x32.cpu().numpy()
    assert i32.status == ppg.PPG_OK and _relres(a, b, x32) <= 1e-8
    assert np.linalg.norm(x32 - r.x) <= 1e-6 * np.linalg.norm(r.x)
    s.close()


def test_polynomial_reduces_iterations_with_ilu_as_in_section6():
    """Section VI's observation on a smaller convection-diffusion problem: ILU(0) plus a degree-12
    polynomial needs far fewer iterations (and dot products) than ILU(0) alone."""
    a = w.convdiff(32, 3, 200.0)
    b = w.rhs(a.n)
    s = _solver(a)
    s.set_left_ilu0(1)
    s.build_poly(0, ppg.PPG_BASIS_ROOTS, v0=_T(w.v0(a.n)))
    _, i0 = s.solve(_T(b), tol=1e-8, restart=50, maxit=5000)
    s.build_poly(12, ppg.PPG_BASIS_ROOTS, v0=_T(w.v0(a.n)))
    _, i12 = s.solve(_T(b), tol=1e-8, restart=50, maxit=5000)
    assert i0.status == i12.status == ppg.PPG_OK
    assert i12.stats["iterations"] * 4 <= i0.stats["iterations"]
    assert i12.stats["dots"] * 4 <= i0.stats["dots"]
    s.close()


def test_ilu_switch_drops_the_polynomial_and_guards_other_entry_points():
    a = w.c1_matrix()
    s = _solver(a)
    s.build_poly(5, ppg.PPG_BASIS_ROOTS, v0=_T(w.v0(a.n)))
    s.set_left_ilu0(1)
    with pytest.raises(ppg.PPGError) as e:
        s.apply_poly(_T(w.uniform(3, a.n)))
    assert e.value.status == ppg.PPG_ERR_NO_POLY
    with pytest.raises(ppg.PPGError):
        s.solve_transpose(_T(w.rhs(a.n)))
    s.set_left_ilu0(0)
    s.build_poly(5, ppg.PPG_BASIS_ROOTS, v0=_T(w.v0(a.n)))
    x, info = s.solve(_T(w.rhs(a.n)), tol=1e-8)
    ref = oracle.gmres(a, w.rhs(a.n), oracle.poly_gmres(a, w.v0(a.n), 5), tol=1e-8, m=50)
    assert info.status == ppg.PPG_OK and abs(info.stats["iterations"] - ref.iters) <= 1
    s.close()


def test_ilu_rejects_unsorted_rows():
    a = w.c1_matrix()
    ci = a.colidx.copy()
    vals = a.vals.copy()
    r0, r1 = a.rowptr[100], a.rowptr[101]
    ci[r0:r1] = ci[r0:r1][::-1].copy()
    vals[r0:r1] = vals[r0:r1][::-1].copy()
    s = ppg.Solver(_T(a.rowptr, torch.int32), _T(ci, torch.int32), _T(vals))
    with pytest.raises(ppg.PPGError) as e:
        s.set_left_ilu0(1)
    assert e.value.status == ppg.PPG_ERR_INVALID_ARG and "sorted" in str(e.value)
    s.close()


@pytest.mark.parametrize("n", [1, 2, 3])
def test_ilu_on_dense_tiny_matrices_is_exact(n):
    """On a dense matrix ILU(0) has no fill to drop: M = L U = A, M^{-1} A = I, and the composed solve
    gives the exact solution at once."""
    rng = np.random.default_rng(10 + n)
    dense = rng.uniform(-1, 1, (n, n)) + np.diag(np.full(n, n + 2.0))
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    a = w.CSR(n, rp, ci, dense.reshape(-1), f"dense{n}")
    s = _solver(a)
    lu = s.set_left_ilu0(1, want_factors=True).cpu().numpy()
    np.testing.assert_array_equal(lu, oracle.ilu0(a))
    s.build_poly(4, ppg.PPG_BASIS_ROOTS, v0=_T(w.uniform(4, n)))
    b = w.uniform(3, n)
    x, info = s.solve(_T(b), tol=1e-10, restart=10, maxit=50)
    assert info.status == ppg.PPG_OK and info.stats["iterations"] <= 2
    np.testing.assert_allclose(x.cpu().numpy(), np.linalg.solve(dense, b), rtol=1e-10, atol=1e-13)
    s.close()
