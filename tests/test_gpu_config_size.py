"""Parity with the oracle at the benchmark configurations' full sizes.

The 128^3 convection-diffusion system (n = 2,097,152, GMRES(50), degrees 10 and 25) and the
perturbed 27-point 100^3 system (n = 1,000,000, degree 25) are solved on the GPU through the C
ABI and by the oracle (its own polynomial construction from the same seeded v0, MGS Arnoldi,
float64), and compared:
  * true relative residual ||b - A x|| / ||b|| <= 1e-8, recomputed on the host (Section III's test);
  * ||x - x_oracle|| <= 1e-6 ||x_oracle||;
  * iteration counts: within 5% for the float64 solve.  The float32 solve with float64 refinement
    reaches about 1e-7 in one float32 cycle, so a 1e-8 target always takes a second refinement
    step; with the restart projection that step costs one basis vector, and the count is held to
    max(5%, one iteration) of the oracle's.
The oracle solves run in spawned worker processes (tests/_oracle_jobs.py) while the GPU works.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import _oracle_jobs
import oracle
import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="no CUDA device")]

import paper_1907_00072_gb300 as ppg  # noqa: E402

DEV = "cuda:0"
CASES = [("c2", 10), ("c2", 25), ("c3", 25)]


@pytest.fixture(scope="module")
def oracle_runs():
    ex = cf.ProcessPoolExecutor(max_workers=len(CASES), mp_context=mp.get_context("spawn"))
    futs = {key: ex.submit(_oracle_jobs.solve, *key) for key in CASES}
    yield futs
    ex.shutdown(wait=True, cancel_futures=True)


_mats = {}


def _matrix(config):
    if config not in _mats:
        _mats.clear()  # one full-size matrix at a time
        _mats[config] = _oracle_jobs.matrix(config)
    return _mats[config]


def _T(a, dt=torch.float64):
    return torch.as_tensor(np.asarray(a), dtype=dt, device=DEV)


def _gpu_solve(config, degree, precision, **kw):
    a = _matrix(config)
    b = w.rhs(a.n)
    s = ppg.Solver(_T(a.rowptr, torch.int32), _T(a.colidx, torch.int32), _T(a.vals))
    used, _ = s.build_poly(degree, ppg.PPG_BASIS_ROOTS, v0=_T(w.v0(a.n)))
    assert used == degree
    x, info = s.solve(_T(b), tol=1e-8, restart=50, maxit=5000, precision=precision, **kw)
    xs = x.cpu().numpy()
    s.close()
    relres = np.linalg.norm(b - oracle.spmv(a, xs)) / np.linalg.norm(b)
    return xs, info, relres


def _check(config, degree, precision, ref):
    xs, info, relres = _gpu_solve(config, degree, precision)
    it, it_ref = info.stats["iterations"], ref["iters"]
    err = np.linalg.norm(xs - ref["x"]) / np.linalg.norm(ref["x"])
    msg = (f"{config} degree {degree}: GPU {it} iterations, relres {relres:.3e}, |x - x_oracle|/|x_oracle| "
           f"{err:.3e}; oracle {it_ref} iterations, relres {ref['relres']:.3e}")
    assert ref["converged"], msg
    assert info.status == ppg.PPG_OK, msg
    assert relres <= 1e-8, msg
    assert abs(info.stats["relres_true"] - relres) <= 1e-3 * relres, msg
    assert err <= 1e-6, msg
    if precision == ppg.PPG_F64:
        assert abs(it - it_ref) <= 0.05 * it_ref, msg
    else:
        assert abs(it - it_ref) <= max(0.05 * it_ref, 1), msg
    print(msg)


def test_c2_degree10_float64_matches_oracle(oracle_runs):
    _check("c2", 10, ppg.PPG_F64, oracle_runs[("c2", 10)].result())


@pytest.mark.parametrize("degree", [10, 25])
def test_c2_float32_refined_matches_oracle(oracle_runs, degree):
    _check("c2", degree, ppg.PPG_F32, oracle_runs[("c2", degree)].result())


def test_c3_degree25_float32_refined_matches_oracle(oracle_runs):
    _check("c3", 25, ppg.PPG_F32, oracle_runs[("c3", 25)].result())


def test_c2_degree10_sstep_float64_matches_oracle(oracle_runs):
    """s-step blocks of 5 (Section VII's combination) in float64: in exact arithmetic GMRES's iterates,
    so the standard oracle's solution and iteration count (within 5%) hold."""
    ref = oracle_runs[("c2", 10)].result()
    xs, info, relres = _gpu_solve("c2", 10, ppg.PPG_F64, sstep=5, sstep_shift=1.0)
    err = np.linalg.norm(xs - ref["x"]) / np.linalg.norm(ref["x"])
    msg = f"s-step float64: {info.stats['iterations']} iterations (oracle {ref['iters']}), relres {relres:.3e}, err {err:.3e}"
    assert info.status == ppg.PPG_OK and relres <= 1e-8 and err <= 1e-6, msg
    assert abs(info.stats["iterations"] - ref["iters"]) <= 0.05 * ref["iters"], msg
    assert info.stats["dots"] < 0.3 * 3 * ref["iters"], msg  # 3 reductions per block of 5, not 3 per iteration
    print(msg)


@pytest.mark.parametrize("form", [ppg.PPG_F32_FLEXIBLE, ppg.PPG_F32_STANDARD])
def test_c2_degree10_sstep_float32_matches_oracle(oracle_runs, form):
    """s-step blocks of 4 in float32 with float64 refinement: the oracle's solution, and the iteration
    count of the library's float32 solve without blocks in the same form, within one; the flexible form
    (Z = P M from the chains' p(A) u_i) also holds the oracle's count to max(5%, 1)."""
    ref = oracle_runs[("c2", 10)].result()
    xs, info, relres = _gpu_solve("c2", 10, ppg.PPG_F32, sstep=4, sstep_shift=1.0, f32_form=form)
    _, info_nb, _ = _gpu_solve("c2", 10, ppg.PPG_F32, f32_form=form)
    err = np.linalg.norm(xs - ref["x"]) / np.linalg.norm(ref["x"])
    it, it_nb = info.stats["iterations"], info_nb.stats["iterations"]
    msg = (f"s-step float32 (form {form}): {it} iterations (without blocks {it_nb}, oracle {ref['iters']}), "
           f"relres {relres:.3e}, err {err:.3e}")
    assert info.status == ppg.PPG_OK and relres <= 1e-8 and err <= 1e-6, msg
    assert abs(it - it_nb) <= 1, msg
    if form == ppg.PPG_F32_FLEXIBLE:
        assert abs(it - ref["iters"]) <= max(0.05 * ref["iters"], 1), msg
    print(msg)
