"""CPU oracle for polynomial-preconditioned GMRES (test infrastructure only).

A thin ctypes wrapper around ``ppg_oracle.c``: plain serial float64 C code
that the CUDA library is checked against.  Only the tests, the smoke check
and the benchmark's CPU-baseline leg import this package; the library never
does, and the two share no code.

The C source states, routine by routine, which part of the paper (Loe,
Thornquist, Boman, arXiv 1907.00072) it follows: Eq. 1 (power basis and
normal equations), Eq. 2 (the polynomial's power form), Section IV (the
POTRF-based degree limit) and Sections I/III (right-preconditioned GMRES(m)
with a relative-residual stopping test).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppg_oracle.c")
_LIB = os.path.join(_HERE, "libppg_oracle.so")

POLY_NONE, POLY_POWER, POLY_ARNOLDI = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, strict IEEE: no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        d = ctypes.c_double
        i64 = ctypes.c_int64
        ci = ctypes.c_int
        p = ctypes.c_void_p
        _lib.orc_spmv.argtypes = [i64, p, p, p, p, p]
        _lib.orc_spmv_rows.argtypes = [i64, p, p, p, p, i64, p, p]
        _lib.orc_transpose.argtypes = [i64, p, p, p, p, p, p]
        _lib.orc_poly_apply.argtypes = [i64, p, p, p, ci, ci, p, p, p, d, p, p]
        _lib.orc_poly_eval_zp.argtypes = [ci, ci, p, p, p, d, d]
        _lib.orc_poly_eval_zp.restype = d
        _lib.orc_cholesky.argtypes = [ci, p, ci]
        _lib.orc_cholesky.restype = ci
        _lib.orc_poly_normal_eq.argtypes = [i64, p, p, p, p, ci, p, p, p, p]
        _lib.orc_poly_normal_eq.restype = ci
        _lib.orc_arnoldi.argtypes = [i64, p, p, p, ci, ci, p, p, p, d, p, ci, p, p, p]
        _lib.orc_arnoldi.restype = ci
        _lib.orc_poly_gmres.argtypes = [i64, p, p, p, p, ci, p, p, p, p]
        _lib.orc_poly_gmres.restype = ci
        _lib.orc_poly_arnoldi_to_power.argtypes = [ci, p, p, d, p]
        _lib.orc_gmres.argtypes = [i64, p, p, p, ci, ci, p, p, p, d, p, p, d, ci, ci, p, p, ci]
        _lib.orc_gmres.restype = ci
        # the same routines with ILU(0) factors on the left (Section VI); lu = NULL is the plain method
        _lib.orc_ilu0.argtypes = [i64, p, p, p, p]
        _lib.orc_ilu0.restype = ci
        _lib.orc_ilu0_apply.argtypes = [i64, p, p, p, p, p]
        _lib.orc_poly_apply_lu.argtypes = [i64, p, p, p, p, ci, ci, p, p, p, d, p, p]
        _lib.orc_poly_normal_eq_lu.argtypes = [i64, p, p, p, p, p, ci, p, p, p, p]
        _lib.orc_poly_normal_eq_lu.restype = ci
        _lib.orc_arnoldi_lu.argtypes = [i64, p, p, p, p, ci, ci, p, p, p, d, p, ci, p, p, p]
        _lib.orc_arnoldi_lu.restype = ci
        _lib.orc_poly_gmres_lu.argtypes = [i64, p, p, p, p, p, ci, p, p, p, p]
        _lib.orc_poly_gmres_lu.restype = ci
        _lib.orc_gmres_lu.argtypes = [i64, p, p, p, p, ci, ci, p, p, p, d, p, p, d, ci, ci, p, p, ci]
        _lib.orc_gmres_lu.restype = ci
        # s-step GMRES with the polynomial (Newton basis, block CGS2, Cholesky QR)
        _lib.orc_sstep_gmres.argtypes = [i64, p, p, p, ci, ci, p, p, p, d, p, p, d, ci, ci, ci, d, p, p, ci, p]
        _lib.orc_sstep_gmres.restype = ci
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _csr(a):
    return a.n, _i32(a.rowptr), _i32(a.colidx), _f64(a.vals)


@dataclass
class Poly:
    """The GMRES minimum-residual polynomial in one of the oracle's representations."""

    kind: int
    deg: int
    coef: np.ndarray | None = None  # POWER: coef[i] multiplies A^i
    H: np.ndarray | None = None  # ARNOLDI: (deg+2) x (deg+1) column-major
    y: np.ndarray | None = None
    beta: float = 1.0
    info: int = 0  # POTRF info of the normal-equations route
    resid: float = float("nan")  # ||v0 - A p(A) v0|| where known

    def args(self):
        return (
            self.kind,
            self.deg,
            _ptr(self.coef),
            _ptr(self.H),
            _ptr(self.y),
            float(self.beta),
        )

    def _keep(self):
        return (self.coef, self.H, self.y)


IDENTITY = Poly(POLY_NONE, 0)


def spmv(a, x):
    lib = _load()
    n, rp, ci, va = _csr(a)
    x = _f64(x)
    y = np.empty(n)
    lib.orc_spmv(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(x), _ptr(y))
    return y


def spmv_rows(a, x, rows):
    lib = _load()
    n, rp, ci, va = _csr(a)
    x = _f64(x)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(len(rows))
    lib.orc_spmv_rows(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(x), len(rows), _ptr(rows), _ptr(y))
    return y


def _lu(lu):
    return None if lu is None else _f64(lu)


def ilu0(a):
    """ILU(0) factors of a (columns sorted within rows, diagonal present): one array on a's pattern
    with the unit lower factor L below the diagonal and U on and above it (Section VI's M = L U)."""
    lib = _load()
    n, rp, ci, va = _csr(a)
    lu = np.empty(len(va))
    st = lib.orc_ilu0(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(lu))
    if st == -2:
        raise MemoryError("oracle allocation failed")
    if st < 0:
        raise ValueError(f"ILU(0) breaks down at row {-st - 1} (no diagonal or a zero pivot)")
    return lu


def ilu0_apply(a, lu, x):
    """(L U)^{-1} x for the factors of ilu0."""
    lib = _load()
    n, rp, ci, _ = _csr(a)
    lu, x = _f64(lu), _f64(x)
    y = np.empty(n)
    lib.orc_ilu0_apply(n, _ptr(rp), _ptr(ci), _ptr(lu), _ptr(x), _ptr(y))
    return y


def transpose(a):
    import workloads

    lib = _load()
    n, rp, ci, va = _csr(a)
    nnz = int(rp[-1])
    rpt = np.empty(n + 1, np.int32)
    cit = np.empty(nnz, np.int32)
    vat = np.empty(nnz)
    lib.orc_transpose(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(rpt), _ptr(cit), _ptr(vat))
    return workloads.CSR(n, rpt, cit, vat, a.name + "^T")


def cholesky(G):
    """Returns (L, info) with POTRF semantics (info = 1-based failing order, 0 if none)."""
    lib = _load()
    k = G.shape[0]
    a = np.asfortranarray(G, dtype=np.float64).copy(order="F")
    info = lib.orc_cholesky(k, _ptr(a), k)
    return np.tril(a), info


def poly_normal_eq(a, v0, deg, lu=None):
    """The paper's construction (Eq. 1 + Cholesky); degree clamped per Section IV.  With lu (ILU(0)
    factors, see ilu0) the polynomial is that of M^{-1} A."""
    lib = _load()
    n, rp, ci, va = _csr(a)
    v0 = _f64(v0)
    coef = np.zeros(deg + 1)
    info = ctypes.c_int(0)
    gram = np.zeros((deg + 1) * (deg + 1))
    rhs = np.zeros(deg + 1)
    used = lib.orc_poly_normal_eq_lu(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(_lu(lu)), _ptr(v0), deg, _ptr(coef),
                                     ctypes.byref(info), _ptr(gram), _ptr(rhs))
    if used == -2:
        raise MemoryError("oracle allocation failed")
    p = Poly(POLY_POWER, max(used, 0), coef[: max(used, 0) + 1].copy(), info=info.value)
    p.gram = gram.reshape(deg + 1, deg + 1, order="F")
    p.rhs = rhs
    p.used = used
    return p


def poly_gmres(a, v0, deg, lu=None):
    """Minimum-residual polynomial from deg+1 MGS Arnoldi steps (Arnoldi form); with lu, of M^{-1} A."""
    lib = _load()
    n, rp, ci, va = _csr(a)
    v0 = _f64(v0)
    H = np.zeros((deg + 2) * (deg + 1))
    y = np.zeros(deg + 1)
    beta = ctypes.c_double(0)
    resid = ctypes.c_double(0)
    built = lib.orc_poly_gmres_lu(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(_lu(lu)), _ptr(v0), deg, _ptr(H), _ptr(y),
                                  ctypes.byref(beta), ctypes.byref(resid))
    if built == -2:
        raise MemoryError("oracle allocation failed")
    if built < deg:  # breakdown: keep the exact lower-degree polynomial
        Hc = H.reshape(deg + 2, deg + 1, order="F")[: built + 2, : built + 1].copy(order="F").ravel(order="F")
        return Poly(POLY_ARNOLDI, built, None, Hc, y[: built + 1].copy(), beta.value, resid=resid.value)
    return Poly(POLY_ARNOLDI, deg, None, H, y, beta.value, resid=resid.value)


def arnoldi_to_power(p: Poly) -> np.ndarray:
    lib = _load()
    coef = np.zeros(p.deg + 1)
    lib.orc_poly_arnoldi_to_power(p.deg, _ptr(p.H), _ptr(p.y), float(p.beta), _ptr(coef))
    return coef


def poly_apply(a, p: Poly, x, lu=None):
    """p(A) x, or p(M^{-1} A) x with ILU(0) factors lu."""
    lib = _load()
    n, rp, ci, va = _csr(a)
    x = _f64(x)
    out = np.empty(n)
    keep = p._keep()  # noqa: F841 (arrays must outlive the call)
    lu = _lu(lu)
    lib.orc_poly_apply_lu(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(lu), *p.args(), _ptr(x), _ptr(out))
    return out


def poly_eval_zp(p: Poly, z):
    """alpha p(alpha) at real points (Section V's plots)."""
    lib = _load()
    keep = p._keep()  # noqa: F841
    return np.array([lib.orc_poly_eval_zp(*p.args(), float(t)) for t in np.atleast_1d(z)])


def arnoldi(a, p: Poly, v, k, lu=None):
    """k MGS Arnoldi steps of A p(A) (with lu: B p(B), B = M^{-1} A) from v: returns (V n x (k+1),
    Hbar (k+1) x k, beta, steps)."""
    lib = _load()
    n, rp, ci, va = _csr(a)
    v = _f64(v)
    V = np.zeros((k + 1) * n)
    H = np.zeros((k + 1) * k)
    beta = ctypes.c_double(0)
    keep = p._keep()  # noqa: F841
    lu = _lu(lu)
    done = lib.orc_arnoldi_lu(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(lu), *p.args(), _ptr(v), k, _ptr(V), _ptr(H),
                              ctypes.byref(beta))
    return V.reshape(k + 1, n).T, H.reshape(k, k + 1).T, beta.value, done


@dataclass
class SolveResult:
    x: np.ndarray
    converged: bool
    iters: int
    restarts: int
    spmvs: int
    dots: int
    relres: float
    est: float
    hist: np.ndarray


def gmres(a, b, p: Poly = IDENTITY, tol=1e-8, m=50, maxit=10000, x0=None, lu=None):
    """Right-preconditioned restarted GMRES(m) with MGS Arnoldi; with lu (ILU(0) factors) the
    composition of Section VI, M^{-1} A p(M^{-1} A) u = M^{-1} b with x = p(M^{-1} A) u."""
    lib = _load()
    n, rp, ci, va = _csr(a)
    b = _f64(b)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    stats = np.zeros(8)
    hist = np.zeros(maxit)
    keep = p._keep()  # noqa: F841
    lu = _lu(lu)
    st = lib.orc_gmres_lu(n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(lu), *p.args(), _ptr(b), _ptr(x), float(tol), int(m),
                          int(maxit), _ptr(stats), _ptr(hist), int(maxit))
    if st == -2:
        raise MemoryError("oracle allocation failed")
    it = int(stats[0])
    return SolveResult(x, bool(stats[4]), it, int(stats[1]), int(stats[2]), int(stats[3]), float(stats[5]),
                       float(stats[6]), hist[:it].copy())


def sstep_gmres(a, b, p: Poly = IDENTITY, s=5, theta=0.0, tol=1e-8, m=50, maxit=10000, x0=None, want_h=False):
    """s-step GMRES(m) with right preconditioning A p(A) u = b: per block, s Newton vectors
    (B - theta I) z / ||.|| from the last basis vector (B = A p(A)), block classical Gram-Schmidt twice
    against the basis, Cholesky QR within the block, and the block's Hessenberg columns recovered from
    the change of basis.  The same iterates as gmres() in exact arithmetic.  Returns (SolveResult,
    number of breakdowns), and with want_h the first cycle's Hessenberg matrix ((m+1) x m, as built)."""
    lib = _load()
    n, rp, ci, va = _csr(a)
    b = _f64(b)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    stats = np.zeros(8)
    hist = np.zeros(maxit)
    keep = p._keep()  # noqa: F841
    h = np.zeros((int(m), int(m) + 1)) if want_h else None  # column-major (m+1) x m, as rows of a (m, m+1) array
    st = lib.orc_sstep_gmres(n, _ptr(rp), _ptr(ci), _ptr(va), *p.args(), _ptr(b), _ptr(x), float(tol), int(m),
                             int(maxit), int(s), float(theta), _ptr(stats), _ptr(hist), int(maxit), _ptr(h))
    if st == -2:
        raise MemoryError("oracle allocation failed")
    it = int(stats[0])
    res = SolveResult(x, bool(stats[4]), it, int(stats[1]), int(stats[2]), int(stats[3]), float(stats[5]),
                      float(stats[6]), hist[:it].copy())
    if want_h:
        return res, int(stats[7]), h.T.copy()
    return res, int(stats[7])
