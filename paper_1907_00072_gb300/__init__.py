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
    "ppg_csr_outer", "ppg_arnoldi", "ppg_hessenberg_eigs", "ppg_fill_uniform", "ppg_solve_batched",
    "ppg_status_string", "ppg_last_error", "ppg_version",
)


class ppg_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("inner_rtol", ctypes.c_double), ("use_graph", ctypes.c_int),
                ("profile", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class ppg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("restarts", ctypes.c_int64), ("spmvs", ctypes.c_int64),
                ("dots", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("relres_true", ctypes.c_double),
                ("relres_est", ctypes.c_double), ("degree_used", ctypes.c_int), ("converged", ctypes.c_int),
                ("breakdowns", ctypes.c_int), ("ctas_per_system", ctypes.c_int), ("time_ms", ctypes.c_double),
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


def _stream_ptr(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _prec_of(t):
    import torch

    if t.dtype == torch.float64:
        return PPG_F64
    if t.dtype == torch.float32:
        return PPG_F32
    raise TypeError("vectors must be float64 or float32")


# --------------------------------------------------------------------------- C-named entry points


def ppg_create(rowptr, colidx, vals, stream=None):
    """Context for the CSR matrix given as CUDA tensors (int32, int32, float64)."""
    import torch

    assert rowptr.is_cuda and rowptr.dtype == torch.int32 and colidx.dtype == torch.int32
    assert vals.dtype == torch.float64
    lib = load_library()
    ctx = ctypes.c_void_p()
    n = rowptr.numel() - 1
    _check(lib.ppg_create(ctypes.byref(ctx), n, vals.numel(), _ptr(rowptr), _ptr(colidx), _ptr(vals),
                          _stream_ptr(stream)), "ppg_create")
    return ctx


def ppg_destroy(ctx):
    load_library().ppg_destroy(ctx)


def ppg_set_stream(ctx, stream=None):
    return _check(load_library().ppg_set_stream(ctx, _stream_ptr(stream)), "ppg_set_stream")


def ppg_workspace_bytes(ctx, restart, degree, precision=PPG_F64):
    out = ctypes.c_size_t(0)
    _check(load_library().ppg_workspace_bytes(ctx, restart, degree, precision, ctypes.byref(out)),
           "ppg_workspace_bytes")
    return out.value


def ppg_set_workspace(ctx, ws):
    return _check(load_library().ppg_set_workspace(ctx, _ptr(ws), 0 if ws is None else ws.numel() * ws.element_size()),
                  "ppg_set_workspace")


def ppg_spmv(ctx, x, y):
    return _check(load_library().ppg_spmv(ctx, _ptr(x), _ptr(y), _prec_of(x)), "ppg_spmv")


def ppg_spmv_format(ctx, request=PPG_SPMV_QUERY):
    """Selects (or with PPG_SPMV_QUERY reports) the sparse format the SpMV kernels read; returns the one in effect."""
    out = ctypes.c_int(0)
    _check(load_library().ppg_spmv_format(ctx, request, ctypes.byref(out)), "ppg_spmv_format")
    return out.value


def ppg_chain_fusion(ctx, request=-1):
    """Turns pairing of the p(A) chain's links on (1) or off (0), or queries it (-1); returns whether
    float32 chains of this matrix are paired."""
    out = ctypes.c_int(0)
    _check(load_library().ppg_chain_fusion(ctx, request, ctypes.byref(out)), "ppg_chain_fusion")
    return out.value


def ppg_build_poly(ctx, degree, basis=PPG_BASIS_ROOTS, v0=None, seed=2):
    used = ctypes.c_int(0)
    st = _check(load_library().ppg_build_poly(ctx, degree, basis, _ptr(v0), seed, ctypes.byref(used)),
                "ppg_build_poly")
    return used.value, st


def ppg_set_poly(ctx, basis, coef):
    """coef: power coefficients (degree + 1) or roots as (re, im) pairs (2 (degree + 1)) on the host."""
    import numpy as np

    c = np.ascontiguousarray(coef, dtype=np.float64)
    deg = (len(c) - 1) if basis == PPG_BASIS_POWER else (len(c) // 2 - 1)
    return _check(load_library().ppg_set_poly(ctx, basis, deg, c.ctypes.data_as(ctypes.c_void_p)), "ppg_set_poly")


def ppg_get_poly(ctx):
    import numpy as np

    b, d, r = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
    buf = np.zeros(256)
    _check(load_library().ppg_get_poly(ctx, ctypes.byref(b), ctypes.byref(d), buf.ctypes.data_as(ctypes.c_void_p),
                                       256, ctypes.byref(r)), "ppg_get_poly")
    cnt = d.value + 1 if b.value == PPG_BASIS_POWER else 2 * (d.value + 1)
    return b.value, d.value, buf[:cnt].copy(), r.value


def ppg_apply_poly(ctx, v, out):
    return _check(load_library().ppg_apply_poly(ctx, _ptr(v), _ptr(out), _prec_of(v)), "ppg_apply_poly")


def ppg_apply_poly_noalloc(ctx, v, out):
    """ppg_apply_poly without any device allocation (n <= 65536; see include/ppg.h)."""
    return _check(load_library().ppg_apply_poly_noalloc(ctx, _ptr(v), _ptr(out), _prec_of(v)),
                  "ppg_apply_poly_noalloc")


def _opts(precision=PPG_F64, inner_rtol=0.0, use_graph=-1, profile=0):
    o = ppg_opts()
    o.precision = precision
    o.inner_rtol = inner_rtol
    o.use_graph = use_graph
    o.profile = profile
    return o


def ppg_solve(ctx, b, x, tol=1e-8, restart=50, maxit=10000, precision=PPG_F64, inner_rtol=0.0, use_graph=-1,
              profile=0):
    """Solves A x = b in place (x holds x0).  Returns (status, stats dict)."""
    st = ppg_stats()
    o = _opts(precision, inner_rtol, use_graph, profile)
    s = _check(load_library().ppg_solve(ctx, _ptr(b), _ptr(x), float(tol), int(restart), int(maxit),
                                        ctypes.byref(o), ctypes.byref(st)), "ppg_solve")
    return s, st.as_dict()


def ppg_solve_transpose(ctx, g, lam, tol=1e-8, restart=50, maxit=10000, precision=PPG_F64, inner_rtol=0.0,
                        use_graph=-1):
    st = ppg_stats()
    o = _opts(precision, inner_rtol, use_graph)
    s = _check(load_library().ppg_solve_transpose(ctx, _ptr(g), _ptr(lam), float(tol), int(restart), int(maxit),
                                                  ctypes.byref(o), ctypes.byref(st)), "ppg_solve_transpose")
    return s, st.as_dict()


def ppg_csr_outer(ctx, u, v, alpha, out):
    return _check(load_library().ppg_csr_outer(ctx, _ptr(u), _ptr(v), float(alpha), _ptr(out)), "ppg_csr_outer")


def ppg_arnoldi(ctx, v, k, V=None):
    """k Arnoldi steps of A p(A) from v; returns (steps, H as a (k+1, k) numpy array)."""
    import numpy as np

    H = np.zeros((k + 1) * k)
    steps = ctypes.c_int(0)
    _check(load_library().ppg_arnoldi(ctx, _ptr(v), int(k), _ptr(V), H.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(steps)), "ppg_arnoldi")
    return steps.value, H.reshape(k, k + 1).T.copy()


def ppg_hessenberg_eigs(ctx, H, wr, wi):
    k = H.shape[1]
    ld = H.shape[0]
    return _check(load_library().ppg_hessenberg_eigs(ctx, k, _ptr(H), ld, _ptr(wr), _ptr(wi)), "ppg_hessenberg_eigs")


def ppg_fill_uniform(ctx, out, seed):
    return _check(load_library().ppg_fill_uniform(ctx, _ptr(out), out.numel(), int(seed)), "ppg_fill_uniform")


def ppg_solve_batched(systems, degree=15, tol=1e-8, restart=30, maxit=10000, seed=2, stream=None):
    """systems: list of (rowptr, colidx, vals, b, x) CUDA tensors (x: initial guess, overwritten).
    Returns (status, list of per-system stats dicts)."""
    n = len(systems)
    arr = (ppg_batch_system * n)()
    for i, (rp, ci, va, b, x) in enumerate(systems):
        arr[i].n = rp.numel() - 1
        arr[i].nnz = va.numel()
        arr[i].rowptr = rp.data_ptr()
        arr[i].colidx = ci.data_ptr()
        arr[i].vals = va.data_ptr()
        arr[i].b = b.data_ptr()
        arr[i].x = x.data_ptr()
    stats = (ppg_stats * n)()
    st = _check(load_library().ppg_solve_batched(n, arr, int(degree), float(tol), int(restart), int(maxit),
                                                 int(seed), _stream_ptr(stream), stats), "ppg_solve_batched")
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
        self._workspace(1, 0, _prec_of(v))
        out = self._torch.empty_like(v) if out is None else out
        ppg_apply_poly(self.ctx, v, out)
        return out

    def solve(self, b, x=None, tol=1e-8, restart=50, maxit=10000, precision=PPG_F64, inner_rtol=0.0, use_graph=-1,
              profile=0):
        self._workspace(restart, 0, precision)
        x = self._torch.zeros_like(b) if x is None else x
        status, stats = ppg_solve(self.ctx, b, x, tol, restart, maxit, precision, inner_rtol, use_graph, profile)
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
    dL/dvals_k = -lambda_{row(k)} x_{col(k)}.  ``vals`` must be the values the
    solver was created with (they enter only through the gradient).
    """
    import torch

    class _Solve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, vals_, b_):
            x, info = solver.solve(b_.detach().contiguous(), tol=tol, restart=restart, maxit=maxit,
                                   precision=precision)
            if info.status < 0:
                raise PPGError(info.status, "solve", "forward solve failed")
            ctx.save_for_backward(x)
            ctx.info = info
            return x

        @staticmethod
        def backward(ctx, gx):
            (x,) = ctx.saved_tensors
            lam, info = solver.solve_transpose(gx.contiguous(), tol=tol, restart=restart, maxit=maxit,
                                               precision=precision)
            if info.status < 0:
                raise PPGError(info.status, "solve_transpose", "adjoint solve failed")
            gvals = solver.csr_outer(lam, x, -1.0)
            return gvals, lam

    return _Solve.apply(vals, b)
