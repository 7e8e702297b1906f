"""s-step PP-GMRES on the GPU (Section VII's combination of the polynomial with an s-step method)
against the oracle's s-step solver and the library's standard solve.

Blocks of s Newton vectors (A p(A) - theta I)^i q_k are orthogonalised together (block classical
Gram-Schmidt twice, Cholesky QR); in exact arithmetic the iterates are GMRES's.  Tolerances: the
float64 solve follows the oracle's iteration count within max(1, 5%) and its solution within 1e-6
(relative), like the standard solve's parity tests; the float32 solve (float64 refinement; the
flexible form by default, Z = P M from the chains' p(A) u_i, and the standard form) reaches the true
relative residual asked for and the oracle's solution.
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


def T(a, dt=None):
    a = np.asarray(a)
    if dt is None:
        dt = torch.float64 if a.dtype.kind == "f" else torch.int32
    return torch.as_tensor(a, dtype=dt, device=DEV)


def solver_for(a):
    return ppg.Solver(T(a.rowptr, torch.int32), T(a.colidx, torch.int32), T(a.vals))


def relres(a, b, x):
    return np.linalg.norm(b - oracle.spmv(a, x)) / np.linalg.norm(b)


MATS = {
    "convdiff3d": lambda: w.convdiff(17, 3, 20.0),  # n = 4913: 20 row tiles of 256, a ragged last one
    "c1": w.c1_matrix,
}


@pytest.mark.parametrize("mat", list(MATS))
@pytest.mark.parametrize("s,theta,deg", [(1, 1.0, 6), (4, 1.0, 6), (5, 1.0, 10), (8, 1.0, 6), (5, 0.5, 6),
                                         (3, 1.0, 0)])
def test_sstep_f64_matches_oracle(mat, s, theta, deg):
    a = MATS[mat]()
    b = w.rhs(a.n)
    v0 = w.v0(a.n)
    sol = solver_for(a)
    if deg:
        sol.build_poly(deg, ppg.PPG_BASIS_ROOTS, v0=T(v0))
        p = oracle.poly_gmres(a, v0, deg)
    else:
        p = oracle.IDENTITY
    ref, _ = oracle.sstep_gmres(a, b, p, s=s, theta=theta, tol=1e-8, m=30, maxit=5000)
    x, info = sol.solve(T(b), tol=1e-8, restart=30, maxit=5000, sstep=s, sstep_shift=theta)
    xg = x.cpu().numpy()
    assert ref.converged
    assert info.status == ppg.PPG_OK, info.stats
    assert relres(a, b, xg) <= 1e-8
    assert abs(info.stats["relres_true"] - relres(a, b, xg)) <= 1e-10
    assert np.linalg.norm(xg - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
    assert abs(info.stats["iterations"] - ref.iters) <= max(1, 0.05 * ref.iters), (info.stats["iterations"], ref.iters)
    sol.close()


@pytest.mark.parametrize("s", [2, 5, 8])
def test_sstep_f64_follows_the_standard_solve(s):
    """The same polynomial and restart length: the s-step solve and the standard one stop within one
    iteration of each other at the same solution, with fewer global reductions (3 per block instead of
    3 per iteration)."""
    a = w.convdiff(17, 3, 20.0)
    b = w.rhs(a.n)
    sol = solver_for(a)
    sol.build_poly(8, ppg.PPG_BASIS_ROOTS, v0=T(w.v0(a.n)))
    xs, i_std = sol.solve(T(b), tol=1e-10, restart=40, maxit=5000)
    xb, i_blk = sol.solve(T(b), tol=1e-10, restart=40, maxit=5000, sstep=s, sstep_shift=1.0)
    assert i_std.status == ppg.PPG_OK and i_blk.status == ppg.PPG_OK
    assert abs(i_std.stats["iterations"] - i_blk.stats["iterations"]) <= 1
    xs, xb = xs.cpu().numpy(), xb.cpu().numpy()
    assert np.linalg.norm(xb - xs) <= 1e-8 * np.linalg.norm(xs)
    if s > 2:
        assert i_blk.stats["dots"] < i_std.stats["dots"]
    sol.close()


@pytest.mark.parametrize("form", [ppg.PPG_F32_FLEXIBLE, ppg.PPG_F32_STANDARD])
@pytest.mark.parametrize("s", [4, 8])
def test_sstep_f32_reaches_the_oracles_solution(s, form):
    """Float32 blocks with float64 refinement, in the flexible form (Z = P M) and the standard form,
    reach the float64 oracle's solution."""
    a = w.convdiff(17, 3, 20.0)
    b = w.rhs(a.n)
    v0 = w.v0(a.n)
    sol = solver_for(a)
    sol.build_poly(10, ppg.PPG_BASIS_ROOTS, v0=T(v0))
    ref = oracle.gmres(a, b, oracle.poly_gmres(a, v0, 10), tol=1e-8, m=50, maxit=5000)
    x, info = sol.solve(T(b), tol=1e-8, restart=50, maxit=5000, precision=ppg.PPG_F32, sstep=s, sstep_shift=1.0,
                        f32_form=form)
    xg = x.cpu().numpy()
    assert info.status == ppg.PPG_OK, info.stats
    assert relres(a, b, xg) <= 1e-8
    assert np.linalg.norm(xg - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
    sol.close()


@pytest.mark.parametrize("prec", [ppg.PPG_F64, ppg.PPG_F32])
def test_sstep_lucky_breakdown_on_an_exhausted_krylov_space(prec):
    """b in a 3-dimensional invariant subspace: the first block of 5 Newton vectors has rank 3, its
    Cholesky QR stops at the dependent vector and the block's last column has a zero subdiagonal
    entry, so the cycle ends after 3 iterations with the exact solution."""
    lams = np.repeat([1.0, 2.0, 5.0], 100)
    n = len(lams)
    a = w.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), lams, "diag")
    b = w.uniform(9, n)
    sol = solver_for(a)
    x, info = sol.solve(T(b), tol=1e-12 if prec == ppg.PPG_F64 else 1e-9, restart=20, maxit=100, precision=prec,
                        sstep=5, sstep_shift=0.5)
    ref, brk = oracle.sstep_gmres(a, b, oracle.IDENTITY, s=5, theta=0.5, tol=1e-12, m=20, maxit=100)
    assert info.status == ppg.PPG_OK, info.stats
    assert brk >= 1 and ref.iters == 3
    if prec == ppg.PPG_F64:
        assert info.stats["iterations"] == 3 and info.stats["breakdowns"] >= 1
        np.testing.assert_allclose(x.cpu().numpy(), b / lams, rtol=1e-10)
    else:
        np.testing.assert_allclose(x.cpu().numpy(), b / lams, rtol=1e-7)
    sol.close()


@pytest.mark.parametrize("prec", [ppg.PPG_F64, ppg.PPG_F32])
def test_sstep_largest_blocks_and_restart(prec):
    """restart 64 with blocks of 8 (the largest basis the block passes stage: 64 + 8 columns per tile,
    144 KB of float64) and blocks of 7 that do not divide it: the solve converges to the oracle's
    solution."""
    a = w.convdiff(17, 3, 20.0)
    b = w.rhs(a.n)
    v0 = w.v0(a.n)
    sol = solver_for(a)
    sol.build_poly(4, ppg.PPG_BASIS_ROOTS, v0=T(v0))
    ref = oracle.gmres(a, b, oracle.poly_gmres(a, v0, 4), tol=1e-10, m=64, maxit=5000)
    for s in (8, 7):
        x, info = sol.solve(T(b), tol=1e-10 if prec == ppg.PPG_F64 else 1e-8, restart=64, maxit=5000, precision=prec,
                            sstep=s, sstep_shift=1.0)
        xg = x.cpu().numpy()
        assert info.status == ppg.PPG_OK, (s, info.stats)
        assert np.linalg.norm(xg - ref.x) <= (1e-8 if prec == ppg.PPG_F64 else 1e-6) * np.linalg.norm(ref.x)
    sol.close()


def test_sstep_zero_rhs_exact_start_and_maxit():
    a = w.c1_matrix()
    sol = solver_for(a)
    sol.build_poly(5, ppg.PPG_BASIS_ROOTS, v0=T(w.v0(a.n)))
    b = w.rhs(a.n)
    x, info = sol.solve(T(np.zeros(a.n)), tol=1e-8, restart=20, sstep=4)
    assert info.status == ppg.PPG_OK and info.stats["iterations"] == 0 and not x.any()
    xd = np.linalg.solve(a.to_dense(), b)
    x, info = sol.solve(T(b), x=T(xd), tol=1e-8, restart=20, sstep=4)
    assert info.status == ppg.PPG_OK and info.stats["iterations"] == 0
    x, info = sol.solve(T(b), tol=1e-14, restart=20, maxit=7, sstep=4)
    assert info.status == ppg.PPG_ERR_NOT_CONVERGED and info.stats["iterations"] == 7
    ref, _ = oracle.sstep_gmres(a, b, oracle.poly_gmres(a, w.v0(a.n), 5), s=4, theta=1.0, tol=1e-14, m=20, maxit=7)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    sol.close()


def test_sstep_rejects_bad_arguments():
    a = w.c1_matrix()
    sol = solver_for(a)
    b = T(w.rhs(a.n))
    for kw in (dict(sstep=9), dict(sstep=-1), dict(sstep=4, restart=65), dict(sstep=4, sstep_shift=float("nan"))):
        args = dict(tol=1e-8, restart=20)
        args.update(kw)
        with pytest.raises(ppg.PPGError) as e:
            sol.solve(b, **args)
        assert e.value.status == ppg.PPG_ERR_INVALID_ARG
    sol.set_left_ilu0(1)
    with pytest.raises(ppg.PPGError) as e:
        sol.solve(b, tol=1e-8, restart=20, sstep=4)
    assert e.value.status == ppg.PPG_ERR_INVALID_ARG
    sol.close()


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_sstep_tiny_systems(n):
    """Degenerate sizes: the Krylov space has at most n dimensions, so a block of 4 Newton vectors is
    rank-deficient from n = 1 on (the block ends in a lucky breakdown); blocks larger than the restart
    length (restart 2 with blocks of 4) shrink to it.  Every solve reaches the dense solution."""
    rng = np.random.default_rng(n)
    dense = rng.uniform(-1, 1, (n, n)) + np.diag(np.full(n, n + 2.0))
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    a = w.CSR(n, rp, ci, dense.reshape(-1), f"dense{n}")
    b = w.uniform(3, n)
    xd = np.linalg.solve(dense, b)
    sol = solver_for(a)
    for poly in (False, True):
        if poly:
            sol.build_poly(10, ppg.PPG_BASIS_ROOTS, v0=T(w.uniform(4, n)))
        for prec in (ppg.PPG_F64, ppg.PPG_F32):
            for restart in (2, 10):
                x, info = sol.solve(T(b), tol=1e-10, restart=restart, maxit=200, precision=prec, sstep=4,
                                    sstep_shift=1.0)
                assert info.status == ppg.PPG_OK, (poly, prec, restart, info.stats)
                np.testing.assert_allclose(x.cpu().numpy(), xd, rtol=1e-8, atol=1e-12)
    sol.close()

