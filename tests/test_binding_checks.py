"""The Python binding checks every tensor before its pointer reaches the C ABI.

The C entry points take bare device pointers and no lengths, so a vector of the
wrong length, type or device would make a kernel read or write outside its
buffer.  These tests run on the CPU: each call below is rejected by the binding
before the library is called (a fake context handle stands in for a real one,
and no call here ever passes every check).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_00072_gb300 as ppg  # noqa: E402

N, NNZ = 8, 20


@pytest.fixture
def ctx():
    c = ppg.Context(0x1000)  # never dereferenced: every call below fails a check first
    c.n, c.nnz, c.device = N, NNZ, torch.device("cpu")
    return c


def f64(n=N):
    return torch.zeros(n, dtype=torch.float64)


def f32(n=N):
    return torch.zeros(n, dtype=torch.float32)


@pytest.mark.parametrize("fn", [ppg.ppg_apply_poly, ppg.ppg_apply_poly_noalloc, ppg.ppg_spmv])
def test_vector_pairs_are_checked(ctx, fn):
    with pytest.raises(TypeError):
        fn(ctx, f64(), f32())  # float64 input, float32 output: the kernel would write 8n bytes into 4n
    with pytest.raises(TypeError):
        fn(ctx, f32(), f64())
    with pytest.raises(ValueError):
        fn(ctx, f64(N + 1), f64())  # wrong length
    with pytest.raises(ValueError):
        fn(ctx, f64(), f64(N - 1))
    with pytest.raises(ValueError):
        fn(ctx, f64(2 * N)[::2], f64())  # not contiguous
    with pytest.raises(ValueError):
        fn(ctx, f64().reshape(2, N // 2), f64())  # not 1-D
    with pytest.raises(ValueError):
        fn(ctx, torch.zeros(N, dtype=torch.float64, device="meta"), f64())  # another device
    with pytest.raises(TypeError):
        fn(ctx, torch.zeros(N, dtype=torch.int32), torch.zeros(N, dtype=torch.int32))
    with pytest.raises(TypeError):
        fn(ctx, np.zeros(N), f64())  # not a tensor
    v = f64()
    with pytest.raises(ValueError):
        fn(ctx, v, v)  # in place: input and output overlap


def test_closed_or_foreign_context_is_rejected():
    c = ppg.Context()
    with pytest.raises(ValueError):
        ppg.ppg_apply_poly(c, f64(), f64())
    with pytest.raises(ValueError):
        ppg.ppg_apply_poly(0x1000, f64(), f64())  # a bare integer is not a context


def test_solve_vectors_are_checked(ctx):
    for fn in (ppg.ppg_solve, ppg.ppg_solve_transpose):
        with pytest.raises(TypeError):
            fn(ctx, f32(), f64())  # solves take float64 b and x
        with pytest.raises(TypeError):
            fn(ctx, f64(), f32())
        with pytest.raises(ValueError):
            fn(ctx, f64(N + 1), f64())
        x = f64()
        with pytest.raises(ValueError):
            fn(ctx, x, x)


def test_other_entry_points_are_checked(ctx):
    with pytest.raises(ValueError):
        ppg.ppg_csr_outer(ctx, f64(), f64(), 1.0, f64(N))  # out has nnz entries, not n
    with pytest.raises(TypeError):
        ppg.ppg_csr_outer(ctx, f64(), f32(), 1.0, f64(NNZ))
    with pytest.raises(TypeError):
        ppg.ppg_build_poly(ctx, 3, v0=f32())
    with pytest.raises(ValueError):
        ppg.ppg_build_poly(ctx, 3, v0=f64(N + 2))
    with pytest.raises(ValueError):
        ppg.ppg_arnoldi(ctx, f64(), 3, V=torch.zeros(3 * N, dtype=torch.float64))  # needs (k+1) n
    with pytest.raises(TypeError):
        ppg.ppg_fill_uniform(ctx, f32(), 1)
    with pytest.raises(ValueError):
        ppg.ppg_hessenberg_eigs(ctx, torch.zeros(4, 3, dtype=torch.float64), f64(4), f64(4))  # ld < k
    with pytest.raises(ValueError):
        ppg.ppg_set_workspace(ctx, torch.zeros(64, dtype=torch.uint8, device="meta"))


def test_create_checks_the_csr_tensors():
    rp = torch.tensor([0, 1, 2], dtype=torch.int32)
    ci = torch.tensor([0, 1], dtype=torch.int32)
    va = torch.tensor([1.0, 2.0], dtype=torch.float64)
    with pytest.raises(ValueError):
        ppg.ppg_create(rp, ci, va)  # CPU tensors: the library takes device memory
    with pytest.raises(TypeError):
        ppg.ppg_create(rp.long(), ci, va)
    with pytest.raises(TypeError):
        ppg.ppg_create(rp, ci, va.float())
    m = lambda t: t.to("meta")  # noqa: E731
    with pytest.raises(ValueError):
        ppg.ppg_create(m(rp), m(ci), m(torch.ones(3, dtype=torch.float64)))  # colidx and vals differ in length
    with pytest.raises(ValueError):
        ppg.ppg_create(m(rp), m(ci), m(torch.ones(4, dtype=torch.float64))[::2])
    with pytest.raises(ValueError):
        ppg.ppg_create(m(torch.tensor([0], dtype=torch.int32)), m(ci[:0]), m(va[:0]))  # n = 0


def test_batched_systems_are_checked():
    rp = torch.tensor([0, 1, 2], dtype=torch.int32)
    ci = torch.tensor([0, 1], dtype=torch.int32)
    va = torch.tensor([1.0, 2.0], dtype=torch.float64)
    with pytest.raises(ValueError):
        ppg.ppg_solve_batched([(rp, ci, va, f64(2), f64(2))])  # CPU tensors
    m = lambda t: t.to("meta")  # noqa: E731
    with pytest.raises(ValueError):
        ppg.ppg_solve_batched([(m(rp), m(ci), m(va), m(f64(3)), m(f64(2)))])  # b of the wrong length
    with pytest.raises(ValueError):
        ppg.ppg_solve_batched([(m(rp), m(ci), m(va), m(f32(2)), m(f64(2)))])


def _fake_solver(vals):
    s = object.__new__(ppg.Solver)
    s.ctx = None
    s.vals = vals
    s._vals_key = (vals.data_ptr(), vals._version)
    return s


def test_differentiable_solve_takes_only_the_solvers_values():
    vals = torch.ones(NNZ, dtype=torch.float64)
    s = _fake_solver(vals)
    with pytest.raises(ValueError, match="not the tensor"):
        ppg.solve(s, torch.ones(NNZ, dtype=torch.float64), f64())  # equal values, another tensor
    vals.mul_(2.0)  # written in place after the context copied the old values
    with pytest.raises(ValueError, match="modified"):
        ppg.solve(s, vals, f64())
