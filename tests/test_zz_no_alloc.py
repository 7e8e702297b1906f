"""The allocation-free apply entry point gives the same result as ppg_apply_poly.

ppg_apply_poly_noalloc exists for callers that may not allocate device memory when they apply
the preconditioner (a fixed device-memory budget reserved at start-up, or code where a
cudaMalloc could fail or must not happen).  Its working vectors come from one array compiled
into the library, shared by every call, so this test also checks that a second call is not
disturbed by what the first one left there.  The file sorts last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as w

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="no CUDA device")]

import paper_1907_00072_gb300 as ppg  # noqa: E402

DEV = "cuda:0"


def _T(a, dt):
    return torch.as_tensor(np.asarray(a), dtype=dt, device=DEV)


def _solver(a):
    return ppg.Solver(_T(a.rowptr, torch.int32), _T(a.colidx, torch.int32), _T(a.vals, torch.float64))


@pytest.mark.parametrize("basis,deg", [(ppg.PPG_BASIS_ROOTS, 10), (ppg.PPG_BASIS_POWER, 4)])
def test_apply_poly_noalloc_matches_apply_poly_on_two_calls(basis, deg):
    a = w.convdiff(255, 2, 10.0)  # n = 65025, just under the 65536-row limit
    s = _solver(a)
    s.build_poly(deg, basis, v0=_T(w.v0(a.n), torch.float64))
    for call in range(2):
        for dtype in (torch.float64, torch.float32):
            x = _T(w.uniform(700 + call, a.n), dtype)
            ref = s.apply_poly(x)  # the workspace-backed entry point (also creates the float32 copy)
            out = torch.full_like(ref, float("nan"))
            ppg.ppg_apply_poly_noalloc(s.ctx, x, out)
            torch.cuda.synchronize()
            r, o = ref.double().cpu().numpy(), out.double().cpu().numpy()
            tol = 1e-12 if dtype == torch.float64 else 1e-5
            assert np.all(np.isfinite(o))
            assert np.linalg.norm(o - r) <= tol * np.linalg.norm(r)
    s.close()


def test_apply_poly_noalloc_rejects_too_large_and_missing_polynomial():
    big = w.convdiff(257, 2, 10.0)  # n = 66049 > 65536
    s = _solver(big)
    x = _T(w.uniform(3, big.n), torch.float64)
    out = torch.empty_like(x)
    with pytest.raises(ppg.PPGError) as e:
        ppg.ppg_apply_poly_noalloc(s.ctx, x, out)
    assert e.value.status == ppg.PPG_ERR_NO_POLY
    s.set_poly(ppg.PPG_BASIS_POWER, [1.0, 0.5])
    with pytest.raises(ppg.PPGError) as e:
        ppg.ppg_apply_poly_noalloc(s.ctx, x, out)
    assert e.value.status == ppg.PPG_ERR_INVALID_ARG
    assert "65536" in str(e.value)
    s.close()
