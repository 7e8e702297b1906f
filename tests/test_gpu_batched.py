"""The batched persistent solver: every system matches an independent single-system solve.

Each system of the batch builds its polynomial from the SplitMix64 stream seed + i; the single
solve is given the same stream, so both build the same minimum-residual polynomial and run the
same float32 PP-GMRES with float64 refinement (flexible form with the restart projection).  Solutions must agree to 1e-6 relative, both must
reach a true relative residual of 1e-8 (checked on the host with the oracle's SpMV), and their
iteration counts must agree within 5%.
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


def _T(a, dt):
    return torch.as_tensor(np.asarray(a), dtype=dt, device=DEV)


def _relres(a, b, x):
    return np.linalg.norm(b - oracle.spmv(a, x)) / np.linalg.norm(b)


def _batch(specs):
    mats, systems = [], []
    for i, (side, pe) in enumerate(specs):
        a, b = w.batch_system(i, side, pe)
        mats.append((a, b))
        systems.append((_T(a.rowptr, torch.int32), _T(a.colidx, torch.int32), _T(a.vals, torch.float64),
                        _T(b, torch.float64), torch.zeros(a.n, dtype=torch.float64, device=DEV)))
    return mats, systems


@pytest.mark.parametrize("degree,restart", [(15, 30), (5, 20), (0, 30)])
def test_batched_matches_single_solves(degree, restart):
    specs = [(32, 6.4), (48, 57.9), (40, 97.6), (100, 5.1), (71, 33.3), (64, 80.0)]
    mats, systems = _batch(specs)
    seed = 11
    status, stats = ppg.ppg_solve_batched(systems, degree=degree, tol=1e-8, restart=restart, maxit=20000, seed=seed)
    assert status == ppg.PPG_OK
    for i, ((a, b), sysi, st) in enumerate(zip(mats, systems, stats)):
        xb = sysi[4].cpu().numpy()
        assert st["converged"] == 1 and st["degree_used"] == degree
        assert _relres(a, b, xb) <= 1e-8
        s = ppg.Solver(sysi[0], sysi[1], sysi[2])
        s.build_poly(degree, ppg.PPG_BASIS_ROOTS, v0=None, seed=seed + i)
        xs, info = s.solve(sysi[3], tol=1e-8, restart=restart, maxit=20000, precision=ppg.PPG_F32)
        xs = xs.cpu().numpy()
        assert info.status == ppg.PPG_OK and _relres(a, b, xs) <= 1e-8
        assert np.linalg.norm(xb - xs) <= 1e-6 * np.linalg.norm(xs)
        assert abs(st["iterations"] - info.stats["iterations"]) <= max(2, 0.05 * info.stats["iterations"])
        s.close()


def test_batched_at_the_configuration_extremes():
    """Grid sides 32 and 448 (n = 1,024 and 200,704) with Peclet 1 and 100, degree 15, GMRES(30), in one
    launch with a few systems between: every system converges to 1e-8 and matches its single solve
    (solution within 1e-6, iterations within max(2, 5%)); the smallest is checked against the oracle."""
    specs = [(448, 100.0), (448, 1.0), (200, 50.0), (90, 20.0), (32, 100.0), (32, 1.0)]
    mats, systems = _batch(specs)
    seed = 21
    status, stats = ppg.ppg_solve_batched(systems, degree=15, tol=1e-8, restart=30, maxit=20000, seed=seed)
    assert status == ppg.PPG_OK
    assert stats[0]["ctas_per_system"] in (4, 8, 16)
    for i, ((a, b), sysi, st) in enumerate(zip(mats, systems, stats)):
        assert st["ctas_per_system"] in (1, 2, 4, 8, 16) and st["spmv_lanes"] in (1, 2, 4, 8)
        xb = sysi[4].cpu().numpy()
        assert st["converged"] == 1 and st["degree_used"] == 15
        assert _relres(a, b, xb) <= 1e-8
        s = ppg.Solver(sysi[0], sysi[1], sysi[2])
        s.build_poly(15, ppg.PPG_BASIS_ROOTS, v0=None, seed=seed + i)
        xs, info = s.solve(sysi[3], tol=1e-8, restart=30, maxit=20000, precision=ppg.PPG_F32)
        xs = xs.cpu().numpy()
        assert info.status == ppg.PPG_OK
        assert np.linalg.norm(xb - xs) <= 1e-6 * np.linalg.norm(xs), i
        assert abs(st["iterations"] - info.stats["iterations"]) <= max(2, 0.05 * info.stats["iterations"]), i
        s.close()
    a, b = mats[-1]
    ref = oracle.gmres(a, b, oracle.poly_gmres(a, w.uniform(seed + len(specs) - 1, a.n), 15), tol=1e-8, m=30,
                       maxit=20000)
    xb = systems[-1][4].cpu().numpy()
    assert ref.converged
    assert np.linalg.norm(xb - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
    assert abs(stats[-1]["iterations"] - ref.iters) <= max(2, 0.05 * ref.iters)


def test_batched_tuning_keeps_the_callers_x_and_is_cached():
    """The autotuner's trial solves run on scratch copies of x: a second call with the same shape starts
    from the caller's x0 again and gives the same result bit for bit (the choice is cached)."""
    specs = [(64, 10.0), (40, 60.0), (33, 90.0)]
    mats, systems = _batch(specs)
    x0 = [torch.full_like(sy[4], 0.25) for sy in systems]
    for sy, x in zip(systems, x0):
        sy[4].copy_(x)
    st1, s1 = ppg.ppg_solve_batched(systems, degree=8, tol=1e-9, restart=20, seed=5)
    r1 = [sy[4].clone() for sy in systems]
    for sy, x in zip(systems, x0):
        sy[4].copy_(x)
    st2, s2 = ppg.ppg_solve_batched(systems, degree=8, tol=1e-9, restart=20, seed=5)
    assert st1 == st2 == ppg.PPG_OK
    for a, b in zip(r1, systems):
        assert torch.equal(a, b[4])
    assert [q["iterations"] for q in s1] == [q["iterations"] for q in s2]


def test_batched_matches_oracle_on_a_small_system():
    specs = [(24, 40.0)]
    mats, systems = _batch(specs)
    status, stats = ppg.ppg_solve_batched(systems, degree=10, tol=1e-10, restart=30, maxit=5000, seed=3)
    (a, b), = mats
    v0 = w.uniform(3, a.n)  # the SplitMix64 stream the batch uses for system 0
    ref = oracle.gmres(a, b, oracle.poly_gmres(a, v0, 10), tol=1e-10, m=30, maxit=5000)
    xb = systems[0][4].cpu().numpy()
    assert status == ppg.PPG_OK and ref.converged
    assert np.linalg.norm(xb - ref.x) <= 1e-7 * np.linalg.norm(ref.x)


def test_batched_zero_rhs_and_initial_guess():
    specs = [(32, 10.0), (36, 20.0)]
    mats, systems = _batch(specs)
    systems[0][3].zero_()  # b = 0: x must come back 0
    systems[0][4].fill_(1.0)
    a1, b1 = mats[1]
    systems[1][4].copy_(_T(np.linalg.solve(a1.to_dense(), b1), torch.float64))  # exact start
    status, stats = ppg.ppg_solve_batched(systems, degree=8, tol=1e-8, restart=30, seed=4)
    assert status == ppg.PPG_OK
    assert stats[1]["iterations"] == 0
    assert stats[0]["converged"] == 1


def test_batched_rejects_bad_arguments():
    specs = [(32, 10.0)]
    _, systems = _batch(specs)
    with pytest.raises(ppg.PPGError):
        ppg.ppg_solve_batched(systems, degree=40)
    with pytest.raises(ppg.PPGError):
        ppg.ppg_solve_batched(systems, restart=41)


@pytest.mark.parametrize("config", ["16,4,16384", "8,4,4000", "4,16,16384", "16,8,16384,512", "8,8,0,512", "16,1,4000",
                                    "2,2,0"])
def test_batched_split_launches_match_single_solves(config, monkeypatch):
    """The configurations the tuner can choose, forced through PPG_BATCH_CONFIG: the large systems in
    one launch and the others in a concurrent second launch with another cluster size (or one launch).
    Every system reports its cluster size and matches its single solve."""
    monkeypatch.setenv("PPG_BATCH_CONFIG", config)
    c1, c2, big = (int(v) for v in config.split(",")[:3])
    if big == 0:
        c2 = c1
    specs = [(200, 50.0), (150, 20.0), (90, 20.0), (64, 80.0), (32, 100.0), (40, 1.0)]
    mats, systems = _batch(specs)
    seed = 31
    status, stats = ppg.ppg_solve_batched(systems, degree=10, tol=1e-8, restart=30, maxit=20000, seed=seed)
    assert status == ppg.PPG_OK
    for i, ((a, b), sysi, st) in enumerate(zip(mats, systems, stats)):
        assert st["ctas_per_system"] == (c1 if a.n >= big else c2)
        xb = sysi[4].cpu().numpy()
        assert st["converged"] == 1 and _relres(a, b, xb) <= 1e-8
        s = ppg.Solver(sysi[0], sysi[1], sysi[2])
        s.build_poly(10, ppg.PPG_BASIS_ROOTS, v0=None, seed=seed + i)
        xs, info = s.solve(sysi[3], tol=1e-8, restart=30, maxit=20000, precision=ppg.PPG_F32)
        xs = xs.cpu().numpy()
        assert info.status == ppg.PPG_OK
        assert np.linalg.norm(xb - xs) <= 1e-6 * np.linalg.norm(xs), i
        assert abs(st["iterations"] - info.stats["iterations"]) <= max(2, 0.05 * info.stats["iterations"]), i
        s.close()


def test_batched_config_override_is_checked(monkeypatch):
    monkeypatch.setenv("PPG_BATCH_CONFIG", "5,4,100")
    mats, systems = _batch([(32, 10.0)])
    with pytest.raises(ppg.PPGError) as e:
        ppg.ppg_solve_batched(systems, degree=5, tol=1e-8, restart=20, seed=1)
    assert e.value.status == ppg.PPG_ERR_INVALID_ARG


def test_batched_degenerate_sizes():
    """Systems of 1, 4 and 9 rows (grid sides 1, 2, 3) in a batch with an ordinary one: most CTAs of a
    tiny system's cluster own no rows, and its Krylov space is exhausted before the degree asked for;
    every system still matches a dense solve."""
    specs = [(1, 10.0), (2, 50.0), (3, 5.0), (40, 20.0)]
    mats, systems = _batch(specs)
    status, stats = ppg.ppg_solve_batched(systems, degree=8, tol=1e-10, restart=20, maxit=2000, seed=7)
    assert status == ppg.PPG_OK
    for (a, b), sysi, st in zip(mats, systems, stats):
        xb = sysi[4].cpu().numpy()
        xd = np.linalg.solve(a.to_dense(), b)
        assert st["converged"] == 1 and _relres(a, b, xb) <= 1e-10
        assert np.linalg.norm(xb - xd) <= 1e-6 * np.linalg.norm(xd)
