"""Failure detection: the library's software waits run out on purpose and the context stays usable.

Every wait in the library is bounded.  These tests make two of them run out without any fault:
  * the two-step chain kernel's waits on its round counters, with a test switch that makes every
    round need one CTA more than the launch has (a count that nothing reaches), and a 2 ms limit;
  * the host's wait for the device's progress between enqueued iterations, with a 1 us limit on a
    system whose first iteration takes hundreds of microseconds.
  * the ILU(0) triangular solves' waits on the rows a row depends on, with the same test switch (every
    wait treats the row it waits on as not ready) and a 2 ms limit.
Each solve must return PPG_ERR_TIMEOUT with a record of where the wait gave up, and the next solve
on the same context, with the default limits, must converge.
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


def _T(a, dt=torch.float64):
    return torch.as_tensor(np.asarray(a), dtype=dt, device=DEV)


def _solver(a):
    return ppg.Solver(_T(a.rowptr, torch.int32), _T(a.colidx, torch.int32), _T(a.vals))


def _relres(a, b, x):
    return np.linalg.norm(b - oracle.spmv(a, x)) / np.linalg.norm(b)


def test_round_counter_wait_runs_out_and_the_context_recovers():
    a = w.convdiff(48, 3, 50.0)  # 110,592 rows: many rounds of the two-step kernel's grid
    b = w.rhs(a.n)
    s = _solver(a)
    s.spmv_format(ppg.PPG_SPMV_CSR)  # the two-step kernel pairs row-block CSR links
    assert s.chain_fusion(1) == 1
    s.build_poly(10, ppg.PPG_BASIS_ROOTS, v0=_T(w.v0(a.n)))
    with pytest.raises(ppg.PPGError) as e:
        s.solve(_T(b), tol=1e-8, restart=30, maxit=300, precision=ppg.PPG_F32, wait_limit_us=2000,
                test_unreachable_wait=1)
    assert e.value.status == ppg.PPG_ERR_TIMEOUT
    msg = str(e.value)
    assert "two-step SpMV: round wait" in msg and "have" in msg and "need" in msg, msg
    # the same context, default limits: the counters were cleared and the solve converges
    x, info = s.solve(_T(b), tol=1e-8, restart=30, maxit=300, precision=ppg.PPG_F32)
    assert info.status == ppg.PPG_OK and _relres(a, b, x.cpu().numpy()) <= 1e-8
    s.chain_fusion(0)
    x0, info0 = s.solve(_T(b), tol=1e-8, restart=30, maxit=300, precision=ppg.PPG_F32)
    np.testing.assert_array_equal(x.cpu().numpy(), x0.cpu().numpy())  # pairing is bit-identical
    s.close()


@pytest.mark.parametrize("sstep", [0, 4])
def test_host_progress_wait_runs_out_and_the_context_recovers(sstep):
    """Iterations (sstep 0) or s-step blocks of 4 (the host queues two blocks ahead): the host's wait for
    the device's progress runs out after 1 us, and the next solve on the same context succeeds."""
    a = w.c2_matrix(96)  # 884,736 rows: an iteration takes far longer than the host needs to queue two
    b = w.rhs(a.n)
    s = _solver(a)
    s.build_poly(10, ppg.PPG_BASIS_ROOTS, v0=_T(w.v0(a.n)))
    with pytest.raises(ppg.PPGError) as e:
        s.solve(_T(b), tol=1e-8, restart=50, maxit=500, precision=ppg.PPG_F32, wait_limit_us=1, sstep=sstep)
    assert e.value.status == ppg.PPG_ERR_TIMEOUT
    assert "wait for the device's progress ran out" in str(e.value)
    x, info = s.solve(_T(b), tol=1e-8, restart=50, maxit=500, precision=ppg.PPG_F32, sstep=sstep)
    assert info.status == ppg.PPG_OK and _relres(a, b, x.cpu().numpy()) <= 1e-8
    s.close()


def test_ilu_ready_word_wait_runs_out_and_the_context_recovers():
    a = w.convdiff(21, 3, 50.0)
    b = w.rhs(a.n)
    s = _solver(a)
    s.set_left_ilu0(1)
    s.build_poly(5, ppg.PPG_BASIS_ROOTS, v0=_T(w.v0(a.n)))
    for prec in (ppg.PPG_F64, ppg.PPG_F32):
        with pytest.raises(ppg.PPGError) as e:
            s.solve(_T(b), tol=1e-8, restart=50, maxit=500, precision=prec, wait_limit_us=2000,
                    test_unreachable_wait=1)
        assert e.value.status == ppg.PPG_ERR_TIMEOUT
        assert "ILU(0) triangular solve" in str(e.value), str(e.value)
        x, info = s.solve(_T(b), tol=1e-8, restart=50, maxit=500, precision=prec)
        assert info.status == ppg.PPG_OK and _relres(a, b, x.cpu().numpy()) <= 1e-8
    s.close()
