"""GB300 polynomial-preconditioned GMRES (Loe, Thornquist, Boman, arXiv 1907.00072).

Python binding of ``libppg.so`` (C ABI in ``include/ppg.h``).  This module only
marshals arguments: torch tensors supply device memory and the CUDA stream,
and every step of the method runs in the library's CUDA kernels.  There is no
CPU path: if the compiled library is missing, importing the binding's entry
points raises.

Low-level functions keep the C names (``ppg_create``, ``ppg_build_poly``,
``ppg_apply_poly``, ``ppg_solve``, ...).  ``Solver`` bundles a context with a
torch-allocated workspace, and ``solve`` is a differentiable solve whose
backward pass is the hand-written adjoint (a transposed PP-GMRES solve with
p(A^T) = p(A)^T and the CSR-pattern outer product for the matrix values).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libppg.so")

PPG_OK = 0
PPG_WARN_DEGREE_CLAMPED = 1
PPG_ERR_NOT_CONVERGED = 2
PPG_ERR_INVALID_ARG = -1
PPG_ERR_CUDA = -2
PPG_ERR_POLY_BREAKDOWN = -3
PPG_ERR_NONFINITE = -4
PPG_ERR_TIMEOUT = -5
PPG_ERR_OOM = -6
PPG_ERR_NO_POLY = -7

PPG_BASIS_POWER = 0
PPG_BASIS_ROOTS = 1
PPG_F64 = 0
PPG_F32 = 1
PPG_F32_FLEXIBLE = 0
PPG_F32_STANDARD = 1
PPG_SPMV_QUERY = -1
PPG_SPMV_AUTO = 0
PPG_SPMV_CSR = 1
PPG_SPMV_SELL = 2
PPG_SPMV_STAGED = 3

# every symbol include/ppg.h declares
EXPORTED = (
    "ppg_create", "ppg_destroy", "ppg_set_stream", "ppg_workspace_bytes", "ppg_set_workspace", "ppg_spmv",
    "ppg_spmv_format", "ppg_chain_fusion", "ppg_build_poly", "ppg_set_poly", "ppg_get_poly", "ppg_apply_poly", "ppg_apply_poly_noalloc", "ppg_solve",
    "ppg_solve_transpose",
    "ppg_csr_outer", "ppg_arnoldi", "ppg_hessenberg_eigs", "ppg_gram_solve", "ppg_fill_uniform", "ppg_solve_batched",
    "ppg_set_left_ilu0",
    "ppg_status_string", "ppg_last_error", "ppg_version",
)


class ppg_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("inner_rtol", ctypes.c_double), ("use_graph", ctypes.c_int),
                ("profile", ctypes.c_int), ("f32_form", ctypes.c_int), ("wait_limit_us", ctypes.c_int),
                ("test_unreachable_wait", ctypes.c_int), ("sstep", ctypes.c_int), ("sstep_shift", ctypes.c_double)]


class ppg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("restarts", ctypes.c_int64), ("spmvs", ctypes.c_int64),
                ("dots", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("relres_true", ctypes.c_double),
                ("relres_est", ctypes.c_double), ("degree_used", ctypes.c_int), ("converged", ctypes.c_int),
                ("breakdowns", ctypes.c_int), ("ctas_per_system", ctypes.c_int), ("spmv_lanes", ctypes.c_int),
                ("time_ms", ctypes.c_double),
                ("spmv_ms", ctypes.c_double), ("spmv_bytes", ctypes.c_double), ("spmv_segments", ctypes.c_int64),
                ("gs_ms", ctypes.c_double), ("gs_bytes", ctypes.c_double), ("gs_segments", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ppg_batch_system(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("x", ctypes.c_void_p)]


class PPGError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libppg.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, I, I64, D, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
    sig = {
        "ppg_create": (I, [ctypes.POINTER(P), I64, I64, P, P, P, P]),
        "ppg_destroy": (None, [P]),
        "ppg_set_stream": (I, [P, P]),
        "ppg_workspace_bytes": (I, [P, I, I, I, ctypes.POINTER(ctypes.c_size_t)]),
        "ppg_set_workspace": (I, [P, P, ctypes.c_size_t]),
        "ppg_spmv": (I, [P, P, P, I]),
        "ppg_spmv_format": (I, [P, I, ctypes.POINTER(I)]),
        "ppg_chain_fusion": (I, [P, I, ctypes.POINTER(I)]),
        "ppg_build_poly": (I, [P, I, I, P, U64, ctypes.POINTER(I)]),
        "ppg_set_poly": (I, [P, I, I, P]),
        "ppg_get_poly": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), P, I, ctypes.POINTER(D)]),
        "ppg_apply_poly": (I, [P, P, P, I]),
        "ppg_apply_poly_noalloc": (I, [P, P, P, I]),
        "ppg_solve": (I, [P, P, P, D, I, I, ctypes.POINTER(ppg_opts), ctypes.POINTER(ppg_stats)]),
        "ppg_solve_transpose": (I, [P, P, P, D, I, I, ctypes.POINTER(ppg_opts), ctypes.POINTER(ppg_stats)]),
        "ppg_csr_outer": (I, [P, P, P, D, P]),
        "ppg_arnoldi": (I, [P, P, I, P, P, ctypes.POINTER(I)]),
        "ppg_hessenberg_eigs": (I, [P, I, P, I, P, P]),
        "ppg_gram_solve": (I, [P, I, P, P, P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "ppg_set_left_ilu0": (I, [P, I, P]),
        "ppg_fill_uniform": (I, [P, P, I64, U64]),
        "ppg_solve_batched": (I, [I, ctypes.POINTER(ppg_batch_system), I, D, I, I, U64, P,
                                  ctypes.POINTER(ppg_stats)]),
        "ppg_status_string": (ctypes.c_char_p, [I]),
        "ppg_last_error": (ctypes.c_char_p, []),
        "ppg_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, where):
    if status < 0:
        lib = load_library()
        raise PPGError(status, where, lib.ppg_last_error().decode())
    return status


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Context(ctypes.c_void_p):
    """Handle of a library context (``ppg_ctx *``) that also remembers the matrix order ``n``, the
    number of stored entries ``nnz`` and the torch device the context was created on, so the bindings
    can check every vector before its pointer reaches the C ABI (which takes no lengths)."""

    n = 0
    nnz = 0
    device = None


def _tensor(t, where, name):
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{where}: {name} must be a torch tensor, got {type(t).__name__}")
    return t


def _vec(ctx, t, where, name, dtype=None, length=None):
    """Checks that t is a contiguous 1-D tensor of `length` (default: the matrix order) elements on the
    context's device, of `dtype` (default: float64 or float32).  Returns its precision code."""
    import torch

    _tensor(t, where, name)
    length = ctx.n if length is None else length
    if ctx.device is not None and t.device != ctx.device:
        raise ValueError(f"{where}: {name} is on {t.device}, the context on {ctx.device}")
    if t.dim() != 1 or t.numel() != length:
        raise ValueError(f"{where}: {name} must be a 1-D tensor of {length} elements, got shape {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{where}: {name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{where}: {name} must be {dtype}, got {t.dtype}")
    if t.dtype not in (torch.float64, torch.float32):
        raise TypeError(f"{where}: {name} must be float64 or float32, got {t.dtype}")
    return PPG_F64 if t.dtype == torch.float64 else PPG_F32


def _pair(ctx, src, dst, where, names=("v", "out")):
    """Input/output vector pair of one precision: same dtype, both of the matrix order, no overlap."""
    prec = _vec(ctx, src, where, names[0])
    _vec(ctx, dst, where, names[1], dtype=src.dtype)
    if _overlap(src, dst):
        raise ValueError(f"{where}: {names[0]} and {names[1]} must not overlap")
    return prec


def _overlap(a, b):
    a0, b0 = a.data_ptr(), b.data_ptr()
    a1 = a0 + a.numel() * a.element_size()
    b1 = b0 + b.numel() * b.element_size()
    return a0 < b1 and b0 < a1


def _f64(ctx, t, where, name, length=None):
    import torch

    return _vec(ctx, t, where, name, dtype=torch.float64, length=length)


def _ctx(ctx, where):
    if not isinstance(ctx, Context) or not ctx.value:
        raise ValueError(f"{where}: not an open context (create one with ppg_create)")
    return ctx


def _stream_ptr(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# --------------------------------------------------------------------------- C-named entry points


def ppg_create(rowptr, colidx, vals, stream=None):
    """Context for the CSR matrix given as CUDA tensors (int32 rowptr[n+1], int32 colidx[nnz], float64
    vals[nnz], contiguous, one device).  Returns a ``Context``."""
    import torch

    where = "ppg_create"
    for name, t, dt in (("rowptr", rowptr, torch.int32), ("colidx", colidx, torch.int32), ("vals", vals, torch.float64)):
        _tensor(t, where, name)
        if t.dtype != dt:
            raise TypeError(f"{where}: {name} must be {dt}, got {t.dtype}")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"{where}: {name} must be a contiguous 1-D tensor")
    if colidx.device != rowptr.device or vals.device != rowptr.device:
        raise ValueError(f"{where}: rowptr, colidx and vals must be on one device")
    if rowptr.numel() < 2:
        raise ValueError(f"{where}: rowptr must have n + 1 >= 2 entries")
    if colidx.numel() != vals.numel():
        raise ValueError(f"{where}: colidx has {colidx.numel()} entries, vals {vals.numel()}")
    if not rowptr.is_cuda:
        raise ValueError(f"{where}: the CSR tensors must be CUDA tensors, got {rowptr.device}")
    lib = load_library()
    ctx = Context()
    n = rowptr.numel() - 1
    _check(lib.ppg_create(ctypes.byref(ctx), n, vals.numel(), _ptr(rowptr), _ptr(colidx), _ptr(vals),
                          _stream_ptr(stream)), where)
    ctx.n, ctx.nnz, ctx.device = n, vals.numel(), vals.device
    return ctx


def ppg_destroy(ctx):
    if isinstance(ctx, Context) and ctx.value:
        load_library().ppg_destroy(ctx)
        ctx.value = None


def ppg_set_stream(ctx, stream=None):
    return _check(load_library().ppg_set_stream(_ctx(ctx, "ppg_set_stream"), _stream_ptr(stream)), "ppg_set_stream")


def ppg_workspace_bytes(ctx, restart, degree, precision=PPG_F64):
    out = ctypes.c_size_t(0)
    _check(load_library().ppg_workspace_bytes(_ctx(ctx, "ppg_workspace_bytes"), restart, degree, precision,
                                              ctypes.byref(out)), "ppg_workspace_bytes")
    return out.value


def ppg_set_workspace(ctx, ws):
    where = "ppg_set_workspace"
    _ctx(ctx, where)
    if ws is not None:
        _tensor(ws, where, "ws")
        if ws.device != ctx.device or not ws.is_contiguous():
            raise ValueError(f"{where}: ws must be a contiguous tensor on {ctx.device}")
    return _check(load_library().ppg_set_workspace(ctx, _ptr(ws), 0 if ws is None else ws.numel() * ws.element_size()),
                  where)


def ppg_spmv(ctx, x, y):
    prec = _pair(_ctx(ctx, "ppg_spmv"), x, y, "ppg_spmv", ("x", "y"))
    return _check(load_library().ppg_spmv(ctx, _ptr(x), _ptr(y), prec), "ppg_spmv")


def ppg_spmv_format(ctx, request=PPG_SPMV_QUERY):
    """Selects (or with PPG_SPMV_QUERY reports) the sparse format the SpMV kernels read; returns the one in effect."""
    out = ctypes.c_int(0)
    _check(load_library().ppg_spmv_format(_ctx(ctx, "ppg_spmv_format"), request, ctypes.byref(out)),
           "ppg_spmv_format")
    return out.value


def ppg_chain_fusion(ctx, request=-1):
    """Turns pairing of the p(A) chain's links on (1) or off (0), or queries it (-1); returns whether
    float32 chains of this matrix are paired."""
    out = ctypes.c_int(0)
    _check(load_library().ppg_chain_fusion(_ctx(ctx, "ppg_chain_fusion"), request, ctypes.byref(out)),
           "ppg_chain_fusion")
    return out.value


def ppg_build_poly(ctx, degree, basis=PPG_BASIS_ROOTS, v0=None, seed=2):
    where = "ppg_build_poly"
    _ctx(ctx, where)
    if v0 is not None:
        _f64(ctx, v0, where, "v0")
    used = ctypes.c_int(0)
    st = _check(load_library().ppg_build_poly(ctx, degree, basis, _ptr(v0), seed, ctypes.byref(used)), where)
    return used.value, st


def ppg_set_poly(ctx, basis, coef):
    """coef: power coefficients (degree + 1) or roots as (re, im) pairs (2 (degree + 1)) on the host."""
    import numpy as np

    c = np.ascontiguousarray(coef, dtype=np.float64)
    deg = (len(c) - 1) if basis == PPG_BASIS_POWER else (len(c) // 2 - 1)
    return _check(load_library().ppg_set_poly(_ctx(ctx, "ppg_set_poly"), basis, deg,
                                              c.ctypes.data_as(ctypes.c_void_p)), "ppg_set_poly")


def ppg_get_poly(ctx):
    import numpy as np

    b, d, r = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
    buf = np.zeros(256)
    _check(load_library().ppg_get_poly(_ctx(ctx, "ppg_get_poly"), ctypes.byref(b), ctypes.byref(d),
                                       buf.ctypes.data_as(ctypes.c_void_p), 256, ctypes.byref(r)), "ppg_get_poly")
    cnt = d.value + 1 if b.value == PPG_BASIS_POWER else 2 * (d.value + 1)
    return b.value, d.value, buf[:cnt].copy(), r.value


def ppg_apply_poly(ctx, v, out):
    prec = _pair(_ctx(ctx, "ppg_apply_poly"), v, out, "ppg_apply_poly")
    return _check(load_library().ppg_apply_poly(ctx, _ptr(v), _ptr(out), prec), "ppg_apply_poly")


def ppg_apply_poly_noalloc(ctx, v, out):
    """ppg_apply_poly without any device allocation (n <= 65536; see include/ppg.h)."""
    prec = _pair(_ctx(ctx, "ppg_apply_poly_noalloc"), v, out, "ppg_apply_poly_noalloc")
    return _check(load_library().ppg_apply_poly_noalloc(ctx, _ptr(v), _ptr(out), prec), "ppg_apply_poly_noalloc")


def _opts(precision=PPG_F64, inner_rtol=0.0, use_graph=-1, profile=0, f32_form=PPG_F32_FLEXIBLE, wait_limit_us=0,
          test_unreachable_wait=0, sstep=0, sstep_shift=1.0):
    o = ppg_opts()
    o.sstep = sstep
    o.sstep_shift = sstep_shift
    o.precision = precision
    o.inner_rtol = inner_rtol
    o.use_graph = use_graph
    o.profile = profile
    o.f32_form = f32_form
    o.wait_limit_us = wait_limit_us
    o.test_unreachable_wait = test_unreachable_wait
    return o


def _solve_args(ctx, b, x, where, names):
    _ctx(ctx, where)
    _f64(ctx, b, where, names[0])
    _f64(ctx, x, where, names[1])
    if _overlap(b, x):
        raise ValueError(f"{where}: {names[0]} and {names[1]} must not overlap")


def ppg_solve(ctx, b, x, tol=1e-8, restart=50, maxit=10000, precision=PPG_F64, inner_rtol=0.0, use_graph=-1,
              profile=0, f32_form=PPG_F32_FLEXIBLE, wait_limit_us=0, test_unreachable_wait=0, sstep=0,
              sstep_shift=1.0):
    """Solves A x = b in place (x holds x0).  Returns (status, stats dict).  sstep in 1..8 builds the basis
    in s-step blocks with the Newton shift sstep_shift (ppg_opts.sstep)."""
    _solve_args(ctx, b, x, "ppg_solve", ("b", "x"))
    st = ppg_stats()
    o = _opts(precision, inner_rtol, use_graph, profile, f32_form, wait_limit_us, test_unreachable_wait, sstep,
              sstep_shift)
    s = _check(load_library().ppg_solve(ctx, _ptr(b), _ptr(x), float(tol), int(restart), int(maxit),
                                        ctypes.byref(o), ctypes.byref(st)), "ppg_solve")
    return s, st.as_dict()


def ppg_solve_transpose(ctx, g, lam, tol=1e-8, restart=50, maxit=10000, precision=PPG_F64, inner_rtol=0.0,
                        use_graph=-1, f32_form=PPG_F32_FLEXIBLE):
    _solve_args(ctx, g, lam, "ppg_solve_transpose", ("g", "lam"))
    st = ppg_stats()
    o = _opts(precision, inner_rtol, use_graph, 0, f32_form)
    s = _check(load_library().ppg_solve_transpose(ctx, _ptr(g), _ptr(lam), float(tol), int(restart), int(maxit),
                                                  ctypes.byref(o), ctypes.byref(st)), "ppg_solve_transpose")
    return s, st.as_dict()


def ppg_csr_outer(ctx, u, v, alpha, out):
    where = "ppg_csr_outer"
    _ctx(ctx, where)
    _f64(ctx, u, where, "u")
    _f64(ctx, v, where, "v")
    _f64(ctx, out, where, "out", length=ctx.nnz)
    if _overlap(out, u) or _overlap(out, v):
        raise ValueError(f"{where}: out must not overlap u or v")
    return _check(load_library().ppg_csr_outer(ctx, _ptr(u), _ptr(v), float(alpha), _ptr(out)), where)


def ppg_arnoldi(ctx, v, k, V=None):
    """k Arnoldi steps of A p(A) from v; returns (steps, H as a (k+1, k) numpy array).  V (optional):
    float64 (k+1, n) tensor receiving the basis, column j of the method in row j."""
    import numpy as np
    import torch

    where = "ppg_arnoldi"
    _ctx(ctx, where)
    _f64(ctx, v, where, "v")
    if V is not None:
        _tensor(V, where, "V")
        if V.dtype != torch.float64 or V.device != ctx.device or not V.is_contiguous() or \
                V.numel() != (int(k) + 1) * ctx.n:
            raise ValueError(f"{where}: V must be a contiguous float64 tensor of (k+1) x n elements on {ctx.device}")
    H = np.zeros((k + 1) * k)
    steps = ctypes.c_int(0)
    _check(load_library().ppg_arnoldi(ctx, _ptr(v), int(k), _ptr(V), H.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(steps)), where)
    return steps.value, H.reshape(k, k + 1).T.copy()


def ppg_hessenberg_eigs(ctx, H, wr, wi):
    """Eigenvalues of the k x k upper Hessenberg matrix stored column-major in H (a float64 tensor of
    shape (k, ld) whose row j holds column j, ld >= k)."""
    import torch

    where = "ppg_hessenberg_eigs"
    _ctx(ctx, where)
    _tensor(H, where, "H")
    if H.dim() != 2 or H.dtype != torch.float64 or H.device != ctx.device or not H.is_contiguous():
        raise ValueError(f"{where}: H must be a contiguous 2-D float64 tensor on {ctx.device}")
    k, ld = H.shape[0], H.shape[1]
    if ld < k:
        raise ValueError(f"{where}: H must have at least as many entries per column as columns")
    _f64(ctx, wr, where, "wr", length=k)
    _f64(ctx, wi, where, "wi", length=k)
    return _check(load_library().ppg_hessenberg_eigs(ctx, k, _ptr(H), ld, _ptr(wr), _ptr(wi)), where)


def ppg_gram_solve(ctx, G, r):
    """Solves G y = r (Eq. 1's normal equations) with the device Cholesky and Section IV's degree rule.
    G: (d+1, d+1) and r: (d+1,) host arrays.  Returns (y, info, degree_used, status)."""
    import numpy as np

    where = "ppg_gram_solve"
    _ctx(ctx, where)
    Gf = np.asfortranarray(G, dtype=np.float64)
    rf = np.ascontiguousarray(r, dtype=np.float64)
    kk = Gf.shape[0]
    if Gf.ndim != 2 or Gf.shape[1] != kk or rf.shape != (kk,):
        raise ValueError(f"{where}: G must be square and r of its order")
    y = np.zeros(kk)
    info, used = ctypes.c_int(0), ctypes.c_int(0)
    st = _check(load_library().ppg_gram_solve(ctx, kk - 1, Gf.ctypes.data_as(ctypes.c_void_p),
                                              rf.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.byref(info), ctypes.byref(used)), where)
    return y, info.value, used.value, st


def ppg_set_left_ilu0(ctx, enable=1, lu_out=None):
    """ILU(0) on the left of the polynomial (Section VI) on or off; lu_out (float64 tensor of nnz, optional)
    receives the factors on A's pattern."""
    where = "ppg_set_left_ilu0"
    _ctx(ctx, where)
    if lu_out is not None:
        _f64(ctx, lu_out, where, "lu_out", length=ctx.nnz)
    return _check(load_library().ppg_set_left_ilu0(ctx, int(enable), _ptr(lu_out)), where)


def ppg_fill_uniform(ctx, out, seed):
    where = "ppg_fill_uniform"
    _ctx(ctx, where)
    _f64(ctx, out, where, "out", length=out.numel() if hasattr(out, "numel") else None)
    return _check(load_library().ppg_fill_uniform(ctx, _ptr(out), out.numel(), int(seed)), where)


def ppg_solve_batched(systems, degree=15, tol=1e-8, restart=30, maxit=10000, seed=2, stream=None):
    """systems: list of (rowptr, colidx, vals, b, x) CUDA tensors (x: initial guess, overwritten).
    Returns (status, list of per-system stats dicts)."""
    import torch

    where = "ppg_solve_batched"
    n = len(systems)
    arr = (ppg_batch_system * n)()
    dev = None
    for i, (rp, ci, va, b, x) in enumerate(systems):
        for name, t, dt in (("rowptr", rp, torch.int32), ("colidx", ci, torch.int32), ("vals", va, torch.float64),
                            ("b", b, torch.float64), ("x", x, torch.float64)):
            _tensor(t, where, f"system {i} {name}")
            if t.dtype != dt or t.dim() != 1 or not t.is_contiguous() or not t.is_cuda:
                raise ValueError(f"{where}: system {i} {name} must be a contiguous 1-D CUDA tensor of {dt}")
            dev = t.device if dev is None else dev
            if t.device != dev:
                raise ValueError(f"{where}: every tensor of the batch must be on one device")
        m = rp.numel() - 1
        if m < 1 or ci.numel() != va.numel() or b.numel() != m or x.numel() != m:
            raise ValueError(f"{where}: system {i} has inconsistent sizes")
        arr[i].n = m
        arr[i].nnz = va.numel()
        arr[i].rowptr = rp.data_ptr()
        arr[i].colidx = ci.data_ptr()
        arr[i].vals = va.data_ptr()
        arr[i].b = b.data_ptr()
        arr[i].x = x.data_ptr()
    stats = (ppg_stats * n)()
    st = _check(load_library().ppg_solve_batched(n, arr, int(degree), float(tol), int(restart), int(maxit),
                                                 int(seed), _stream_ptr(stream), stats), where)
    return st, [stats[i].as_dict() for i in range(n)]


def ppg_status_string(status):
    return load_library().ppg_status_string(int(status)).decode()


def ppg_version():
    return load_library().ppg_version().decode()


# --------------------------------------------------------------------------- convenience layer


@dataclass
class SolveInfo:
    status: int
    stats: dict


class Solver:
    """A context plus a torch-allocated workspace for one CSR matrix.

    ``Solver(rowptr, colidx, vals)`` takes CUDA tensors; ``build_poly`` builds
    the minimum-residual polynomial, ``apply_poly`` applies it, ``solve`` runs
    PP-GMRES(m).  The workspace is a torch uint8 tensor sized by the library.
    """

    def __init__(self, rowptr, colidx, vals, stream=None):
        import torch

        self.n = rowptr.numel() - 1
        self.nnz = vals.numel()
        self.device = vals.device
        self.ctx = ppg_create(rowptr, colidx, vals, stream)
        # the values the context copied: solve() accepts only this tensor, unmodified since
        self.vals = vals
        self._vals_key = (vals.data_ptr(), vals._version)
        self._ws = None
        self._ws_key = None
        self._torch = torch

    def close(self):
        if getattr(self, "ctx", None) is not None:
            ppg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _workspace(self, restart, degree, precision=PPG_F64):
        need = ppg_workspace_bytes(self.ctx, restart, degree, precision)
        if self._ws is None or self._ws.numel() < need:
            self._ws = self._torch.empty(need + 256, dtype=self._torch.uint8, device=self.device)
            ppg_set_workspace(self.ctx, self._ws)

    def set_stream(self, stream=None):
        ppg_set_stream(self.ctx, stream)

    def spmv(self, x, y=None):
        y = self._torch.empty_like(x) if y is None else y
        ppg_spmv(self.ctx, x, y)
        return y

    def set_left_ilu0(self, enable=1, want_factors=False):
        """ILU(0) on the left (Section VI); returns the factors (float64, nnz) when want_factors."""
        lu = self._torch.empty(self.nnz, dtype=self._torch.float64, device=self.device) if want_factors else None
        ppg_set_left_ilu0(self.ctx, enable, lu)
        return lu

    def spmv_format(self, request=PPG_SPMV_QUERY):
        return ppg_spmv_format(self.ctx, request)

    def chain_fusion(self, request=-1):
        return ppg_chain_fusion(self.ctx, request)

    def build_poly(self, degree, basis=PPG_BASIS_ROOTS, v0=None, seed=2):
        self._workspace(1, max(degree, 30) if degree < 0 else degree)
        return ppg_build_poly(self.ctx, degree, basis, v0, seed)

    def set_poly(self, basis, coef):
        return ppg_set_poly(self.ctx, basis, coef)

    def get_poly(self):
        return ppg_get_poly(self.ctx)

    def apply_poly(self, v, out=None):
        self._workspace(1, 0, PPG_F32 if v.dtype == self._torch.float32 else PPG_F64)
        out = self._torch.empty_like(v) if out is None else out
        ppg_apply_poly(self.ctx, v, out)
        return out

    def solve(self, b, x=None, tol=1e-8, restart=50, maxit=10000, precision=PPG_F64, inner_rtol=0.0, use_graph=-1,
              profile=0, f32_form=PPG_F32_FLEXIBLE, wait_limit_us=0, test_unreachable_wait=0, sstep=0,
              sstep_shift=1.0):
        self._workspace(restart, 0, precision)
        x = self._torch.zeros_like(b) if x is None else x
        status, stats = ppg_solve(self.ctx, b, x, tol, restart, maxit, precision, inner_rtol, use_graph, profile,
                                  f32_form, wait_limit_us, test_unreachable_wait, sstep, sstep_shift)
        return x, SolveInfo(status, stats)

    def solve_transpose(self, g, lam=None, tol=1e-8, restart=50, maxit=10000, precision=PPG_F64, inner_rtol=0.0):
        lam = self._torch.zeros_like(g) if lam is None else lam
        status, stats = ppg_solve_transpose(self.ctx, g, lam, tol, restart, maxit, precision, inner_rtol)
        return lam, SolveInfo(status, stats)

    def csr_outer(self, u, v, alpha=1.0, out=None):
        out = self._torch.empty(self.nnz, dtype=self._torch.float64, device=self.device) if out is None else out
        ppg_csr_outer(self.ctx, u, v, alpha, out)
        return out

    def arnoldi(self, v, k, want_V=False):
        self._workspace(k, 0)
        V = self._torch.zeros((k + 1, self.n), dtype=self._torch.float64, device=self.device) if want_V else None
        steps, H = ppg_arnoldi(self.ctx, v, k, V)
        return steps, H, V


def solve(solver: Solver, vals, b, tol=1e-10, restart=50, maxit=10000, precision=PPG_F64):
    """Differentiable x = A^{-1} b for the solver's matrix with values ``vals``.

    The forward pass is PP-GMRES with the solver's polynomial; the backward pass
    solves A^T lambda = dL/dx with p(A^T) = p(A)^T and returns dL/db = lambda and
    dL/dvals_k = -lambda_{row(k)} x_{col(k)}.  ``vals`` must be the tensor the
    solver was created with, unmodified since (the context holds a copy of those
    values, so other values would give a wrong solve and wrong gradients): any
    other tensor, or the same one written in place, raises ValueError.  A forward
    or adjoint solve that fails or stops at ``maxit`` without meeting ``tol``
    raises PPGError.
    """
    import torch

    if vals is not solver.vals and (vals.data_ptr(), vals._version) != solver._vals_key:
        raise ValueError("solve: vals is not the tensor the solver was created with")
    if (vals.data_ptr(), vals._version) != solver._vals_key:
        raise ValueError("solve: vals was modified after the solver was created (the context holds the old values)")

    def _require(info, where):
        if info.status < 0 or info.status == PPG_ERR_NOT_CONVERGED:
            raise PPGError(info.status, where,
                           f"{ppg_status_string(info.status)} after {info.stats['iterations']} iterations "
                           f"(true relative residual {info.stats['relres_true']:.3e}, tol {tol:g})")

    class _Solve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, vals_, b_):
            x, info = solver.solve(b_.detach().contiguous(), tol=tol, restart=restart, maxit=maxit,
                                   precision=precision)
            _require(info, "solve")
            ctx.save_for_backward(x)
            ctx.info = info
            return x

        @staticmethod
        def backward(ctx, gx):
            (x,) = ctx.saved_tensors
            lam, info = solver.solve_transpose(gx.contiguous(), tol=tol, restart=restart, maxit=maxit,
                                               precision=precision)
            _require(info, "solve_transpose")
            gvals = solver.csr_outer(lam, x, -1.0)
            return gvals, lam

    return _Solve.apply(vals, b)
