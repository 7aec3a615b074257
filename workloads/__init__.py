"""Seeded synthetic inputs shared by the oracle and the GPU path.

This module holds no arithmetic of the solver: it only writes down PDE-shaped
sparse matrices (CSR), grid coordinates for the recursive bisection, and
right-hand sides drawn from a counter-based generator.  Both sides of every
parity test (the CPU oracle and the CUDA library) take their inputs from here.

Matrices (the stencils the paper benchmarks, Sec. 5):
  * 2D 5-point Poisson, Dirichlet: diagonal 4, neighbours -1 (no 1/h^2 factor).
  * 3D 7-point Poisson, Dirichlet: diagonal 6, neighbours -1.
  * 3D variable-coefficient diffusion -div(phi grad T) (Sec. 5.2.2 stencil,
    Dirichlet instead of periodic so that the operator is nonsingular):
    per-cell phi = 10^U(lo, hi), face coefficient = harmonic mean of the two
    cells, a Dirichlet boundary face uses the cell's own phi.
  * 2D upwind convection-diffusion (nonsymmetric, 5-point).
  * block-diagonal matrices (no coupling between chosen index groups).

Unknowns are ordered lexicographically with x fastest; coordinates are the
integer grid indices.

Random numbers come from splitmix64 (Steele, Lea & Flood, OOPSLA 2014):
value k of a stream with seed s is mix(s + (k+1) * 0x9E3779B97F4A7C15), with
the published mix function; u = (z >> 11) * 2^-53 in [0, 1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "CSR", "splitmix64", "uniform01", "rhs_uniform", "poisson2d", "poisson3d",
    "varcoef3d", "convdiff2d_upwind", "block_diagonal", "grid_coords",
    "dense_from_csr", "spmv",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class CSR:
    """A square sparse matrix in CSR form plus the coordinates of its unknowns."""

    def __init__(self, rowptr, colind, val, coords, name=""):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.colind = np.ascontiguousarray(colind, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.n = int(self.rowptr.shape[0] - 1)
        self.dim = int(self.coords.shape[1])
        self.name = name

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def with_values(self, val):
        return CSR(self.rowptr, self.colind, val, self.coords, self.name)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Values start..start+count-1 of the splitmix64 stream with this seed."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    z = splitmix64(seed, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def rhs_uniform(n: int, seeds) -> np.ndarray:
    """Column-major n x len(seeds) array; column c is uniform[-1,1] from seeds[c]."""
    seeds = list(seeds)
    b = np.empty((n, len(seeds)), dtype=np.float64, order="F")
    for c, s in enumerate(seeds):
        b[:, c] = 2.0 * uniform01(int(s), n) - 1.0
    return b


def grid_coords(shape) -> np.ndarray:
    """Integer grid coordinates, lexicographic with axis 0 (x) fastest."""
    idx = np.indices(tuple(reversed(shape)), dtype=np.float64)
    # idx[0] is the slowest axis; reverse so column 0 is x.
    cols = [idx[len(shape) - 1 - d].reshape(-1) for d in range(len(shape))]
    return np.stack(cols, axis=1)


def _assemble(n, rows, cols, vals, coords, name):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(rowptr, cols.astype(np.int32), vals, coords, name)


def _stencil(shape, face_coef, diag_extra=None, name="", diag_full=None):
    """Assemble a face-coupled stencil on a grid.

    face_coef(axis, lo_index_array, hi_index_array) -> (c_lo_hi, c_hi_lo): the
    off-diagonal entries A[lo, hi] and A[hi, lo] (negated couplings) for faces
    between a cell and its +1 neighbour along `axis`.  The diagonal is minus
    the row sum of the off-diagonals plus `diag_extra` (boundary terms).
    """
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    lin = np.arange(n, dtype=np.int64).reshape(tuple(reversed(shape)))
    rows, cols, vals = [], [], []
    diag = np.zeros(n, dtype=np.float64)
    for ax in range(len(shape)):
        npax = len(shape) - 1 - ax          # numpy axis of grid axis `ax`
        lo = np.take(lin, np.arange(shape[ax] - 1), axis=npax).reshape(-1)
        hi = np.take(lin, np.arange(1, shape[ax]), axis=npax).reshape(-1)
        a_lohi, a_hilo = face_coef(ax, lo, hi)
        rows += [lo, hi]
        cols += [hi, lo]
        vals += [a_lohi, a_hilo]
        diag_lo = -a_lohi
        diag_hi = -a_hilo
        np.add.at(diag, lo, diag_lo)
        np.add.at(diag, hi, diag_hi)
    if diag_extra is not None:
        diag += diag_extra
    if diag_full is not None:
        diag = np.broadcast_to(np.asarray(diag_full, dtype=np.float64), (n,)).copy()
    rows.append(np.arange(n, dtype=np.int64))
    cols.append(np.arange(n, dtype=np.int64))
    vals.append(diag)
    return _assemble(n, np.concatenate(rows), np.concatenate(cols),
                     np.concatenate(vals), grid_coords(shape), name)


def _boundary_faces(shape):
    """Number of Dirichlet boundary faces of each cell (lexicographic order)."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    coords = grid_coords(shape)
    cnt = np.zeros(n, dtype=np.float64)
    for ax in range(len(shape)):
        cnt += (coords[:, ax] == 0)
        cnt += (coords[:, ax] == shape[ax] - 1)
    return cnt


def poisson2d(nx: int, ny: int) -> CSR:
    """5-point Laplacian on an nx x ny grid, Dirichlet: diag 4, off -1."""
    shape = (nx, ny)
    one = lambda ax, lo, hi: (-np.ones(lo.size), -np.ones(lo.size))
    return _stencil(shape, one, diag_extra=_boundary_faces(shape),
                    name=f"poisson2d_{nx}x{ny}")


def poisson3d(nx: int, ny: int, nz: int) -> CSR:
    """7-point Laplacian on an nx x ny x nz grid, Dirichlet: diag 6, off -1."""
    shape = (nx, ny, nz)
    one = lambda ax, lo, hi: (-np.ones(lo.size), -np.ones(lo.size))
    return _stencil(shape, one, diag_extra=_boundary_faces(shape),
                    name=f"poisson3d_{nx}x{ny}x{nz}")


def varcoef3d(nx: int, ny: int, nz: int, seed: int = 1,
              lo_exp: float = -3.0, hi_exp: float = 3.0) -> CSR:
    """-div(phi grad) with phi = 10^U(lo_exp, hi_exp) per cell, Dirichlet.

    Face coefficient is the harmonic mean of the two cells' phi; a boundary
    face uses the cell's phi.  The matrix is symmetric positive definite.
    """
    shape = (nx, ny, nz)
    n = nx * ny * nz
    phi = 10.0 ** (lo_exp + (hi_exp - lo_exp) * uniform01(seed, n))

    def coef(ax, lo, hi):
        c = 2.0 * phi[lo] * phi[hi] / (phi[lo] + phi[hi])
        return -c, -c

    coords = grid_coords(shape)
    bnd = np.zeros(n)
    for ax in range(3):
        bnd += phi * (coords[:, ax] == 0)
        bnd += phi * (coords[:, ax] == shape[ax] - 1)
    return _stencil(shape, coef, diag_extra=bnd,
                    name=f"varcoef3d_{nx}x{ny}x{nz}_s{seed}")


def vcp_indefinite3d(nx: int, ny: int, nz: int, seed: int = 3) -> CSR:
    """-div(phi grad) with phi ~ U(-1, 1) per cell, Dirichlet: the indefinite
    variable-coefficient case (about half the eigenvalues of each sign).

    The face coefficient is the arithmetic mean of the two cells' phi (a
    harmonic mean is undefined where phi changes sign); a boundary face uses
    the cell's phi.  Symmetric, indefinite.
    """
    shape = (nx, ny, nz)
    n = nx * ny * nz
    phi = 2.0 * uniform01(seed, n) - 1.0

    def coef(ax, lo, hi):
        c = 0.5 * (phi[lo] + phi[hi])
        return -c, -c

    coords = grid_coords(shape)
    bnd = np.zeros(n)
    for ax in range(3):
        bnd += phi * (coords[:, ax] == 0)
        bnd += phi * (coords[:, ax] == shape[ax] - 1)
    return _stencil(shape, coef, diag_extra=bnd,
                    name=f"vcp_indefinite3d_{nx}x{ny}x{nz}_s{seed}")


def convdiff2d_upwind(N: int, angle: float, peclet: float) -> CSR:
    """-Laplace(T) + v . grad_upwind(T) on the unit square, N x N interior grid.

    h = 1/(N+1), |v| = peclet (L = 1, nu = 1), v = peclet (cos a, sin a).  The
    rows are scaled by h^2: diagonal 4 + (|vx| + |vy|) h, the upwind neighbour
    -1 - |v_axis| h, the downwind neighbour -1.  Nonsymmetric values,
    structurally symmetric pattern.
    """
    h = 1.0 / (N + 1)
    v = (peclet * np.cos(angle), peclet * np.sin(angle))

    def coef(ax, lo, hi):
        a_lohi = -1.0 - max(-v[ax], 0.0) * h   # row lo, its +1 neighbour
        a_hilo = -1.0 - max(v[ax], 0.0) * h    # row hi, its -1 neighbour
        return np.full(lo.size, a_lohi), np.full(lo.size, a_hilo)

    full = 4.0 + (abs(v[0]) + abs(v[1])) * h
    return _stencil((N, N), coef, name=f"convdiff2d_{N}", diag_full=full)


def convdiff2d_batch_params(count: int, seed: int = 7):
    """Seeded parameters of a batch of 2D upwind convection-diffusion instances:
    grid side uniform in [64, 512], velocity direction uniform on the circle,
    Peclet number uniform in [1, 100].  Returns (sides, angles, pecletes)."""
    u = uniform01(seed, 3 * count)
    sides = (64 + np.floor(449 * u[:count])).astype(np.int64)
    return sides, 2.0 * np.pi * u[count:2 * count], 1.0 + 99.0 * u[2 * count:]


def convdiff2d_batch(count: int, seed: int = 7, first: int = 0, stop=None):
    """Instances first..stop-1 of the seeded batch of convdiff2d_batch_params."""
    sides, angles, pe = convdiff2d_batch_params(count, seed)
    stop = count if stop is None else stop
    return [convdiff2d_upwind(int(sides[k]), float(angles[k]), float(pe[k])) for k in range(first, stop)]


def knn_graph(n: int, k: int, seed: int) -> CSR:
    """A random geometric graph: n seeded points in the unit square (odd seed)
    or cube (even seed), each coupled to its k nearest neighbours
    (symmetrised); diagonal 2k + 1, off-diagonal -1, and -1.3 above the
    diagonal (nonsymmetric values, symmetric pattern)."""
    dim = 2 if seed % 2 else 3
    pts = uniform01(seed, n * dim).reshape(n, dim)
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    nb = np.argsort(d2, axis=1)[:, :k]
    pairs = {(i, int(j)) for i in range(n) for j in nb[i]}
    pairs |= {(j, i) for i, j in pairs}
    pairs = sorted(pairs)
    rows = np.array([p[0] for p in pairs] + list(range(n)), dtype=np.int64)
    cols = np.array([p[1] for p in pairs] + list(range(n)), dtype=np.int64)
    vals = np.where(rows == cols, 2.0 * k + 1.0, -1.0 - 0.3 * (rows < cols))
    return _assemble(n, rows, cols, vals, pts, f"knn{n}_{k}_s{seed}")


def block_diagonal(csr: CSR, group_of: np.ndarray) -> CSR:
    """Drop every entry that couples two different index groups."""
    rows = np.repeat(np.arange(csr.n), np.diff(csr.rowptr))
    keep = group_of[rows] == group_of[csr.colind]
    return _assemble(csr.n, rows[keep], csr.colind[keep].astype(np.int64),
                     csr.val[keep], csr.coords, csr.name + "_blockdiag")


def dense_from_csr(csr: CSR) -> np.ndarray:
    A = np.zeros((csr.n, csr.n))
    rows = np.repeat(np.arange(csr.n), np.diff(csr.rowptr))
    A[rows, csr.colind] = csr.val
    return A


def spmv(csr: CSR, x: np.ndarray) -> np.ndarray:
    """y = A x for x of shape (n,) or (n, k)."""
    rows = np.repeat(np.arange(csr.n), np.diff(csr.rowptr))
    prod = csr.val[:, None] * np.asarray(x).reshape(csr.n, -1)[csr.colind]
    y = np.zeros((csr.n, prod.shape[1]))
    np.add.at(y, rows, prod)
    return y.reshape(np.shape(x))
