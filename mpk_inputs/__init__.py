"""Seeded synthetic inputs for the matrix power kernel and s-step GMRES workloads.

This module only builds inputs (sparse matrices in CSR form, vectors, shift sets, arrival
streams).  It holds none of the method's arithmetic: no SpMV, no level construction, no
orthogonalisation.  Both the CPU oracle's tests and the GPU path's tests and benchmark draw
their inputs from here, so that the two sides see identical data while sharing no code.

All random numbers come from ``numpy.random.default_rng(seed)`` (PCG64); every seed is an
argument.  Matrices are returned as ``(row_ptr:int32[n+1], col:int32[nnz], val:float64[nnz])``
with columns ascending inside each row.

Workloads (sizes are the ones the benchmarks use; every function also takes smaller sizes):

* ``poisson2d_5pt(64)``            2-D 5-point Dirichlet Laplacian, n=4096, nnz=20,224.
* ``stencil27(160, seed=2)``       3-D 27-point matrix on a 160^3 grid, diagonal 26 and
                                   off-diagonals -1 - U[0,0.1) drawn once per unordered pair
                                   (so the matrix is symmetric), nnz=478^3=109,215,352.
* ``diffusion7_lognormal(256)``    3-D 7-point finite-volume diffusion with log-normal cell
                                   coefficients, harmonic-mean faces, Dirichlet boundary faces,
                                   rows and columns symmetrically permuted, nnz=117,047,296.
* ``stencil27(128, seed=5)``       the block-MPK matrix (used in FP32), nnz=382^3=55,742,968.
* ``anisotropic(N, 7|27, a)``      constant-coefficient anisotropic diffusion for the solve
                                   stream; ``solve_stream`` draws the request sequence.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR", "poisson2d_5pt", "stencil27", "stencil7", "diffusion7_lognormal", "anisotropic",
    "uniform_vectors", "leja_points_interval", "random_sparse", "solve_stream",
    "symmetric_permute", "grid_offsets_3d",
]


@dataclass
class CSR:
    """A square sparse matrix in compressed-row form (int32 indices, float64 values)."""
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def astype(self, dtype) -> "CSR":
        return CSR(self.row_ptr, self.col, self.val.astype(dtype))


def grid_offsets_3d():
    """The 27 offsets (di, dj, dk) in {-1,0,1}^3 in lexicographic order.

    With index = (i*N + j)*N + k, this order makes the column indices of a row ascending."""
    return [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]


def _compress(cols: np.ndarray, vals: np.ndarray, mask: np.ndarray) -> CSR:
    """Turn dense (n, w) per-row slot arrays plus a validity mask into CSR (row-major order)."""
    counts = mask.sum(axis=1, dtype=np.int64)
    row_ptr = np.zeros(mask.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 indices")
    return CSR(row_ptr.astype(np.int32), cols[mask].astype(np.int32), vals[mask].astype(np.float64))


def poisson2d_5pt(N: int) -> CSR:
    """2-D 5-point Laplacian on an N x N grid with Dirichlet truncation: 4 on the diagonal,
    -1 for each in-grid neighbour.  Index = i*N + j."""
    n = N * N
    i, j = np.divmod(np.arange(n, dtype=np.int64), N)
    offs = [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    cols = np.empty((n, 5), dtype=np.int64)
    vals = np.empty((n, 5), dtype=np.float64)
    mask = np.empty((n, 5), dtype=bool)
    for s, (di, dj) in enumerate(offs):
        ii, jj = i + di, j + dj
        mask[:, s] = (ii >= 0) & (ii < N) & (jj >= 0) & (jj < N)
        cols[:, s] = ii * N + jj
        vals[:, s] = 4.0 if (di, dj) == (0, 0) else -1.0
    return _compress(cols, vals, mask)


def _grid3(N: int):
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    i, rem = np.divmod(idx, N * N)
    j, k = np.divmod(rem, N)
    return n, i, j, k


def stencil27(N: int, seed: int, diag: float = 26.0, eps: float = 0.1) -> CSR:
    """3-D 27-point matrix on an N^3 grid (index (i*N+j)*N+k), Dirichlet truncation.

    Diagonal ``diag``; the entry coupling grid points p and p+d (d one of the 26 offsets) is
    -1 - u, with u ~ U[0, eps) drawn once per unordered pair so the matrix is symmetric.
    Draw order: ``u = rng.random((13, N, N, N)) * eps``, one slab per positive offset (the 13
    offsets after (0,0,0) in lexicographic order); the pair {p, p+d} with d positive uses
    ``u[d][p]``."""
    rng = np.random.default_rng(seed)
    offs = grid_offsets_3d()
    pos = [d for d in offs if d > (0, 0, 0)]
    u = rng.random((13, N, N, N)) * eps
    n, i, j, k = _grid3(N)
    cols = np.empty((n, 27), dtype=np.int64)
    vals = np.empty((n, 27), dtype=np.float64)
    mask = np.empty((n, 27), dtype=bool)
    for s, (di, dj, dk) in enumerate(offs):
        ii, jj, kk = i + di, j + dj, k + dk
        m = (ii >= 0) & (ii < N) & (jj >= 0) & (jj < N) & (kk >= 0) & (kk < N)
        mask[:, s] = m
        cols[:, s] = (ii * N + jj) * N + kk
        if (di, dj, dk) == (0, 0, 0):
            vals[:, s] = diag
        elif (di, dj, dk) > (0, 0, 0):
            vals[:, s] = -1.0 - u[pos.index((di, dj, dk))].reshape(-1)
        else:
            # pair {p+d, p} with -d positive: its draw sits at the lower point p+d
            slab = u[pos.index((-di, -dj, -dk))].reshape(-1)
            src = np.where(m, (ii * N + jj) * N + kk, 0)
            vals[:, s] = -1.0 - slab[src]
        del m
    del u
    return _compress(cols, vals, mask)


def stencil7(N: int, wx: float = 1.0, wy: float = 1.0, wz: float = 1.0) -> CSR:
    """Constant-coefficient 7-point operator on N^3 with Dirichlet boundary: off-diagonals
    -w_axis, diagonal 2*(wx+wy+wz).  Axis z is i (slowest), x is k (fastest)."""
    n, i, j, k = _grid3(N)
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    w = {0: wz, 1: wy, 2: wx}
    cols = np.empty((n, 7), dtype=np.int64)
    vals = np.empty((n, 7), dtype=np.float64)
    mask = np.empty((n, 7), dtype=bool)
    for s, d in enumerate(offs):
        ii, jj, kk = i + d[0], j + d[1], k + d[2]
        mask[:, s] = (ii >= 0) & (ii < N) & (jj >= 0) & (jj < N) & (kk >= 0) & (kk < N)
        cols[:, s] = (ii * N + jj) * N + kk
        if d == (0, 0, 0):
            vals[:, s] = 2.0 * (wx + wy + wz)
        else:
            ax = [t for t in range(3) if d[t] != 0][0]
            vals[:, s] = -w[ax]
    return _compress(cols, vals, mask)


def anisotropic(N: int, stencil: int, a: float) -> CSR:
    """Anisotropic diffusion with axis weights (1, 1, a) (a on z).

    7-point: ``stencil7(N, 1, 1, a)``.  27-point: the entry for offset d is minus the weight
    w(d) = (sum over axes of kappa_axis*|d_axis|) / (number of nonzero components of d); the
    diagonal is the sum of w over all 26 offsets (in-grid or not), i.e. Dirichlet."""
    if stencil == 7:
        return stencil7(N, 1.0, 1.0, a)
    if stencil != 27:
        raise ValueError("stencil must be 7 or 27")
    kap = (a, 1.0, 1.0)  # (z, y, x) = (i, j, k) axes
    offs = grid_offsets_3d()

    def wgt(d):
        nzc = sum(1 for t in d if t != 0)
        return sum(kap[t] * abs(d[t]) for t in range(3)) / nzc

    dsum = sum(wgt(d) for d in offs if d != (0, 0, 0))
    n, i, j, k = _grid3(N)
    cols = np.empty((n, 27), dtype=np.int64)
    vals = np.empty((n, 27), dtype=np.float64)
    mask = np.empty((n, 27), dtype=bool)
    for s, d in enumerate(offs):
        ii, jj, kk = i + d[0], j + d[1], k + d[2]
        mask[:, s] = (ii >= 0) & (ii < N) & (jj >= 0) & (jj < N) & (kk >= 0) & (kk < N)
        cols[:, s] = (ii * N + jj) * N + kk
        vals[:, s] = dsum if d == (0, 0, 0) else -wgt(d)
    return _compress(cols, vals, mask)


def symmetric_permute(A: CSR, perm: np.ndarray) -> CSR:
    """Return B = P A P^T with B[r, c] = A[perm[r], perm[c]], columns ascending per row.
    Rows must have at most 32 entries (enough for every stencil here)."""
    n = A.n
    lens = np.diff(A.row_ptr.astype(np.int64))
    w = int(lens.max()) if n else 0
    if w > 32:
        raise ValueError("symmetric_permute handles rows of at most 32 entries")
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n, dtype=np.int64)
    slot = np.arange(A.nnz, dtype=np.int64) - np.repeat(A.row_ptr[:-1].astype(np.int64), lens)
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    cols = np.full((n, w), np.iinfo(np.int64).max, dtype=np.int64)
    vals = np.zeros((n, w), dtype=np.float64)
    cols[rows, slot] = iperm[A.col.astype(np.int64)]
    vals[rows, slot] = A.val
    cols = cols[perm]
    vals = vals[perm]
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    vals = np.take_along_axis(vals, order, axis=1)
    mask = cols != np.iinfo(np.int64).max
    return _compress(cols, vals, mask)


def diffusion7_lognormal(N: int, seed_kappa: int = 3, sigma: float = 1.0, seed_perm: int = 1,
                         permute: bool = True) -> CSR:
    """Cell-centred finite-volume diffusion on N^3 cells.

    kappa_cell = exp(sigma * Z), Z ~ N(0,1) drawn as ``rng(seed_kappa).standard_normal(N^3)``.
    Interior face coefficient = harmonic mean 2*k1*k2/(k1+k2); a boundary face contributes
    kappa_cell to the diagonal (Dirichlet).  Off-diagonal = -face coefficient, diagonal = sum of
    the six face coefficients.  With ``permute`` the matrix is symmetrically permuted by
    ``perm = rng(seed_perm).permutation(n)`` (row r of the result is grid cell perm[r])."""
    rng = np.random.default_rng(seed_kappa)
    n, i, j, k = _grid3(N)
    kap = np.exp(sigma * rng.standard_normal(n))
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    cols = np.empty((n, 7), dtype=np.int64)
    vals = np.empty((n, 7), dtype=np.float64)
    mask = np.empty((n, 7), dtype=bool)
    diag = np.zeros(n, dtype=np.float64)
    for s, d in enumerate(offs):
        if d == (0, 0, 0):
            continue
        ii, jj, kk = i + d[0], j + d[1], k + d[2]
        m = (ii >= 0) & (ii < N) & (jj >= 0) & (jj < N) & (kk >= 0) & (kk < N)
        nb = np.where(m, (ii * N + jj) * N + kk, 0)
        kn = kap[nb]
        face = np.where(m, 2.0 * kap * kn / (kap + kn), kap)
        diag += face
        mask[:, s] = m
        cols[:, s] = nb
        vals[:, s] = -face
    mask[:, 3] = True
    cols[:, 3] = np.arange(n)
    vals[:, 3] = diag
    A = _compress(cols, vals, mask)
    if not permute:
        return A
    perm = np.random.default_rng(seed_perm).permutation(n)
    return symmetric_permute(A, perm)


def uniform_vectors(n: int, seed: int, n_rhs: int = 1, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Column-major block of n_rhs vectors of length n, entries U[lo, hi), shape (n_rhs, n).

    Row c of the result is right-hand side c (so the flat array is column-major n x n_rhs)."""
    rng = np.random.default_rng(seed)
    return lo + (hi - lo) * rng.random((n_rhs, n))


def leja_points_interval(lo: float, hi: float, count: int, n_cand: int = 10001) -> np.ndarray:
    """Leja-ordered points on [lo, hi], used as the fixed Newton shifts of the 27-point MPK
    benchmark.  Candidates are ``n_cand`` equispaced points; the first point is the candidate of
    largest modulus; each next one maximises the product of distances to those already taken
    (computed as a sum of logs); ties go to the smaller value."""
    cand = np.linspace(lo, hi, n_cand)
    taken = []
    mag = np.abs(cand)
    first = int(np.flatnonzero(mag == mag.max())[0])
    taken.append(first)
    score = np.zeros(n_cand)
    for _ in range(1, count):
        last = cand[taken[-1]]
        with np.errstate(divide="ignore"):
            score += np.log(np.abs(cand - last))
        score[taken] = -np.inf
        best = score.max()
        taken.append(int(np.flatnonzero(score == best)[0]))
    return cand[taken].copy()


def random_sparse(n: int, density: float, seed: int, symmetric: bool = True,
                  components: int = 1, diag: bool = True, int_values: bool = False) -> CSR:
    """Small random sparse matrix for brute-force checks.

    The rows are split into ``components`` contiguous blocks with no coupling between blocks.
    Off-diagonal pattern ~ Bernoulli(density) inside each block (mirrored when ``symmetric``).
    Values U[-1,1) (or integers in [-3, 3] with ``int_values``); diagonal entries are present
    when ``diag``."""
    rng = np.random.default_rng(seed)
    M = np.zeros((n, n))
    bounds = np.linspace(0, n, components + 1).astype(int)
    for b in range(components):
        lo, hi = bounds[b], bounds[b + 1]
        m = hi - lo
        pat = rng.random((m, m)) < density
        if symmetric:
            pat = np.triu(pat, 1)
            pat = pat | pat.T
        np.fill_diagonal(pat, False)
        if int_values:
            v = rng.integers(-3, 4, size=(m, m)).astype(np.float64)
            v[v == 0] = 1.0
        else:
            v = rng.random((m, m)) * 2 - 1
        if symmetric:
            v = np.triu(v, 1)
            v = v + v.T
        blk = np.where(pat, v, 0.0)
        if diag:
            d = rng.integers(1, 5, size=m).astype(np.float64) if int_values else 2.0 + rng.random(m)
            blk[np.arange(m), np.arange(m)] = d
        M[lo:hi, lo:hi] = blk
    mask = M != 0
    if not diag:
        mask &= ~np.eye(n, dtype=bool)
    cols = np.broadcast_to(np.arange(n), (n, n))
    return _compress(cols, M, mask)


def solve_stream(n_requests: int, seed: int = 7, rate_hz: float = 200.0, n_min: int = 32,
                 n_max: int = 192, a_min: float = 1.0, a_max: float = 100.0):
    """Request sequence for the solve stream: Poisson arrivals (exponential gaps, mean
    1/rate_hz), grid edge N ~ U{n_min..n_max}, stencil 7 or 27 with probability 1/2 each,
    anisotropy a ~ log-uniform[a_min, a_max], and a right-hand-side seed per request.

    Returns a list of dicts with keys t_arrival, N, stencil, a, b_seed."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    Ns = rng.integers(n_min, n_max + 1, size=n_requests)
    st = np.where(rng.random(n_requests) < 0.5, 7, 27)
    a = np.exp(rng.uniform(math.log(a_min), math.log(a_max), size=n_requests))
    bseed = rng.integers(0, 2**31 - 1, size=n_requests)
    t = np.cumsum(gaps)
    return [dict(t_arrival=float(t[r]), N=int(Ns[r]), stencil=int(st[r]), a=float(a[r]),
                 b_seed=int(bseed[r])) for r in range(n_requests)]
