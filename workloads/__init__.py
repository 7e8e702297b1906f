"""Seeded synthetic inputs for the polynomial-preconditioned GMRES workloads.

This module only *generates* inputs: sparse matrices in CSR form (int32
row pointers and column indices, float64 values) and seeded vectors.  It
holds none of the solver's arithmetic, so both the CPU oracle and the CUDA
path can take their inputs from here without sharing any method code.

Random numbers come from a counter-based SplitMix64 generator (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
output ``i`` of stream ``seed`` is ``mix(mix(seed) + (i + 1) * GAMMA)``,
where ``mix`` is the SplitMix64 finaliser, and a uniform double in [0, 1)
is the top 53 bits times 2**-53.  Because element ``i`` depends only on
(seed, i), any slice of a stream can be regenerated independently.

Matrices (the paper's workloads are Matrix Market and Firedrake matrices
that are not available here; these stencils have the same structure):

* ``convdiff``: convection-diffusion ``-eps*lap(u) + w.grad(u)`` on the unit
  square/cube, interior ``N^dim`` grid, h = 1/(N+1), homogeneous Dirichlet
  boundaries, lexicographic ordering with x fastest.  Central differences for
  diffusion, first-order upwind for convection, every row scaled by h^2:
  diagonal ``2*dim*eps + h*sum|w_d|``, upwind neighbour ``-eps - h|w_d|``,
  downwind neighbour ``-eps``.  eps = 1 and |w|_2 = Pe (global Peclet number).
* ``stencil27_perturbed``: 27-point stencil whose off-diagonals are ``-1``
  times independent U[0.5, 1.5] factors (nonsymmetric), with diagonal
  ``a_ii = sum_j |a_ij| + delta`` so that every Gershgorin disc lies in Re > 0.
* ``laplacian2d``: the 5-point Laplacian (diagonal 4, off-diagonals -1) used
  in the paper's Section V example (n = 40401 for a 201 x 201 grid).
* ``bidiag1`` / ``bidiag2``: the upper bidiagonal test matrices of Section IV.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seeds used by every workload (one per role).
SEED_B = 1
SEED_V0 = 2
SEED_XTARGET = 3
SEED_PERTURB = 4
SEED_BATCH = 5
SEED_BATCH_B0 = 1000  # system i of the batch uses seed 1000 + i for b


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, index) -> np.ndarray:
    """Counter-based SplitMix64 output for (seed, index); index may be an array."""
    idx = np.asarray(index, dtype=np.uint64)
    base = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    with np.errstate(over="ignore"):
        state = base + (idx + np.uint64(1)) * GAMMA
    return _mix(state)


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1): element i is stream position offset + i."""
    bits = splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64))
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, n: int, lo: float = -1.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [lo, hi)."""
    return lo + (hi - lo) * uniform01(seed, n, offset)


@dataclass
class CSR:
    """A square sparse matrix in CSR form (rows sorted, columns sorted within a row)."""

    n: int
    rowptr: np.ndarray  # int32, n + 1
    colidx: np.ndarray  # int32, nnz
    vals: np.ndarray  # float64, nnz
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.vals, self.colidx, self.rowptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        np.add.at(a, (rows, self.colidx), self.vals)
        return a


def _assemble(n: int, offsets: list[int], valid: np.ndarray, vals: np.ndarray, name: str) -> CSR:
    """Build CSR from per-row stencil slots.

    ``offsets`` are column offsets sorted ascending, ``valid`` and ``vals`` are
    (n, len(offsets)) arrays.  Row-major compression keeps columns sorted.
    """
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32")
    cols = np.arange(n, dtype=np.int64)[:, None] + np.asarray(offsets, dtype=np.int64)[None, :]
    colidx = cols[valid].astype(np.int32)
    v = vals[valid].astype(np.float64)
    return CSR(n, rowptr.astype(np.int32), colidx, v, name)


def convdiff(N: int, dim: int, pe: float, wind=None, eps: float = 1.0) -> CSR:
    """Upwind convection-diffusion on an interior N^dim grid (see module docstring)."""
    if wind is None:
        wind = (1.0, 0.5) if dim == 2 else (1.0, 0.5, 0.25)
    w = np.asarray(wind, dtype=np.float64)[:dim]
    w = w / np.linalg.norm(w) * pe
    h = 1.0 / (N + 1)
    n = N**dim
    idx = np.arange(n, dtype=np.int64)
    coords = [(idx // N**d) % N for d in range(dim)]  # d = 0 is x (fastest)
    offsets, valid_cols, val_cols = [], [], []
    # neighbours in order of increasing column offset: -N^(dim-1) ... -1, 0, +1 ... +N^(dim-1)
    for d in reversed(range(dim)):
        stride = N**d
        upwind_lo = w[d] > 0  # flow in +x_d: the lower neighbour is upwind
        coef = -eps - (h * abs(w[d]) if upwind_lo else 0.0)
        offsets.append(-stride)
        valid_cols.append(coords[d] > 0)
        val_cols.append(np.full(n, coef))
    offsets.append(0)
    valid_cols.append(np.ones(n, dtype=bool))
    val_cols.append(np.full(n, 2.0 * dim * eps + h * float(np.abs(w).sum())))
    for d in range(dim):
        stride = N**d
        upwind_hi = w[d] < 0
        coef = -eps - (h * abs(w[d]) if upwind_hi else 0.0)
        offsets.append(stride)
        valid_cols.append(coords[d] < N - 1)
        val_cols.append(np.full(n, coef))
    valid = np.stack(valid_cols, axis=1)
    vals = np.stack(val_cols, axis=1)
    return _assemble(n, offsets, valid, vals, f"convdiff{dim}d_N{N}_Pe{pe:g}")


def laplacian2d(N: int) -> CSR:
    """5-point Laplacian on an N x N interior grid: 4 on the diagonal, -1 off it."""
    n = N * N
    idx = np.arange(n, dtype=np.int64)
    x, y = idx % N, idx // N
    offsets = [-N, -1, 0, 1, N]
    valid = np.stack([y > 0, x > 0, np.ones(n, bool), x < N - 1, y < N - 1], axis=1)
    vals = np.tile(np.array([-1.0, -1.0, 4.0, -1.0, -1.0]), (n, 1))
    return _assemble(n, offsets, valid, vals, f"laplacian2d_N{N}")


def stencil27_perturbed(N: int, seed: int = SEED_PERTURB, delta: float = 0.05) -> CSR:
    """27-point stencil with off-diagonals -U[0.5,1.5] and diagonal sum|a_ij| + delta."""
    n = N**3
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % N, (idx // N) % N, idx // (N * N)
    offsets, valid_cols = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                offsets.append(dz * N * N + dy * N + dx)
                ok = np.ones(n, dtype=bool)
                for c, dc in ((x, dx), (y, dy), (z, dz)):
                    if dc < 0:
                        ok &= c > 0
                    elif dc > 0:
                        ok &= c < N - 1
                valid_cols.append(ok)
    valid = np.stack(valid_cols, axis=1)
    # one random factor per (row, slot): stream position row*27 + slot
    factors = uniform(seed, n * 27, 0.5, 1.5).reshape(n, 27)
    vals = -factors
    centre = offsets.index(0)
    vals[:, centre] = 0.0
    offdiag_abs = np.where(valid, np.abs(vals), 0.0).sum(axis=1)
    vals[:, centre] = offdiag_abs + delta
    return _assemble(n, offsets, valid, vals, f"stencil27_N{N}_delta{delta:g}")


def bidiag(diag: np.ndarray, sup: float, name: str) -> CSR:
    n = len(diag)
    offsets = [0, 1]
    valid = np.stack([np.ones(n, bool), np.arange(n) < n - 1], axis=1)
    vals = np.stack([np.asarray(diag, dtype=np.float64), np.full(n, sup)], axis=1)
    return _assemble(n, offsets, valid, vals, name)


def bidiag1() -> CSR:
    """n = 2000: diagonal 1, 2, ..., 2000; 0.05 on the superdiagonal (Section IV)."""
    return bidiag(np.arange(1, 2001, dtype=np.float64), 0.05, "BiDiag1")


def bidiag2() -> CSR:
    """n = 5000: diagonal 0.1, ..., 0.9, 1, 2, ..., 4991; 0.2 on the superdiagonal (Section IV)."""
    d = np.concatenate([np.arange(1, 10) / 10.0, np.arange(1, 4992, dtype=np.float64)])
    return bidiag(d, 0.2, "BiDiag2")


def random_csr(n: int, nnz_per_row: int, seed: int, diag_shift: float = 0.0, max_row: int | None = None) -> CSR:
    """Random nonsymmetric CSR with a nonzero diagonal (ragged row lengths).

    Row i gets between 1 and 2*nnz_per_row entries (or up to ``max_row``);
    off-diagonal values are U[-1, 1]; the diagonal is sum|off| + diag_shift.
    """
    u = uniform01(seed, 4 * n * (2 * nnz_per_row + 2))
    pos = 0
    rows, cols, vals = [], [], []
    cap = max_row if max_row is not None else 2 * nnz_per_row
    for i in range(n):
        k = 1 + int(u[pos] * cap)
        pos += 1
        c = set()
        for _ in range(k - 1):
            c.add(int(u[pos] * n))
            pos += 1
        c.discard(i)
        c = sorted(c)
        off = [2.0 * u[pos + t] - 1.0 for t in range(len(c))]
        pos += len(c)
        d = float(np.sum(np.abs(off))) + diag_shift
        entries = sorted(list(zip(c, off)) + [(i, d if d != 0 else 1.0)])
        for cc, vv in entries:
            rows.append(i)
            cols.append(cc)
            vals.append(vv)
    rows = np.asarray(rows, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr.astype(np.int32), np.asarray(cols, dtype=np.int32), np.asarray(vals), f"random_n{n}")


# ---------------------------------------------------------------------------
# The five workload configurations of the polynomial-preconditioned GMRES study
# ---------------------------------------------------------------------------


def c1_matrix() -> CSR:
    """2D 64x64 upwind convection-diffusion, Pe 10, wind (1, 0.5): n = 4096."""
    return convdiff(64, 2, 10.0, (1.0, 0.5))


def c2_matrix(N: int = 128) -> CSR:
    """3D 128^3 7-point convection-diffusion, Pe 50, wind (1, 0.5, 0.25): n = 2,097,152."""
    return convdiff(N, 3, 50.0, (1.0, 0.5, 0.25))


def c3_matrix(N: int = 100) -> CSR:
    """Perturbed 27-point stencil on 100^3: n = 1,000,000, nnz 26,463,592."""
    return stencil27_perturbed(N, SEED_PERTURB, 0.05)


def c5_matrix(N: int = 64) -> CSR:
    """3D 64^3 7-point convection-diffusion, Pe 50 (adjoint workload)."""
    return convdiff(N, 3, 50.0, (1.0, 0.5, 0.25))


def batch_specs(count: int = 256, seed: int = SEED_BATCH, lo: int = 32, hi: int = 448):
    """Grid sides log-uniform in [lo, hi] and Peclet numbers U[1, 100] for the batch."""
    u = uniform01(seed, 2 * count)
    sides = np.rint(np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u[:count])).astype(int)
    pes = 1.0 + 99.0 * u[count:]
    return [(int(s), float(p)) for s, p in zip(sides, pes)]


def batch_system(i: int, side: int, pe: float):
    """System i of the batch: 2D convection-diffusion and its seeded right-hand side."""
    a = convdiff(side, 2, pe, (1.0, 0.5))
    b = uniform(SEED_BATCH_B0 + i, a.n)
    return a, b


def rhs(n: int, seed: int = SEED_B) -> np.ndarray:
    return uniform(seed, n)


def v0(n: int, seed: int = SEED_V0) -> np.ndarray:
    return uniform(seed, n)


def expected_nnz_convdiff(N: int, dim: int) -> int:
    return N**dim * (2 * dim + 1) - 2 * dim * N ** (dim - 1)


def describe(a: CSR) -> str:
    return f"{a.name}: n={a.n} nnz={a.nnz} nnz/row={a.nnz / max(a.n, 1):.2f}"


__all__ = [
    "CSR",
    "splitmix64",
    "uniform01",
    "uniform",
    "convdiff",
    "laplacian2d",
    "stencil27_perturbed",
    "bidiag1",
    "bidiag2",
    "random_csr",
    "c1_matrix",
    "c2_matrix",
    "c3_matrix",
    "c5_matrix",
    "batch_specs",
    "batch_system",
    "rhs",
    "v0",
    "describe",
    "math",
]
