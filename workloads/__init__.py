"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module builds matrices and vectors only; it holds none of the solver or
SpMV arithmetic.  Matrices are returned as CSR triples
``(rowptr int32[n+1], col int32[nnz], val float64[nnz])`` with sorted, unique
column indices in every row.  Random numbers come from numpy's PCG64
(``np.random.default_rng(seed)``).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "poisson1d", "poisson2d", "stencil27", "powerlaw", "random_csr", "diagonal",
    "convdiff2d", "uniform_vector", "csr_to_dense", "scaled_identity", "varcoef2d", "batch_varcoef2d",
    "varcoef3d", "varcoef3d_from",
]


def _finish(rowptr, col, val):
    return (np.ascontiguousarray(rowptr, dtype=np.int32), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


def _from_offsets(shape, offsets, weights):
    """Structured-grid stencil matrix.  ``offsets`` are tuples over the grid
    axes (slowest first), sorted so that column indices increase within a
    row; unknowns outside the grid are dropped (homogeneous Dirichlet)."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    idx = np.indices(shape).reshape(len(shape), -1)
    strides = np.array([int(np.prod(shape[d + 1:])) for d in range(len(shape))], dtype=np.int64)
    cols = np.empty((n, len(offsets)), dtype=np.int32)
    mask = np.empty((n, len(offsets)), dtype=bool)
    vals = np.empty((n, len(offsets)), dtype=np.float64)
    ar = np.arange(n, dtype=np.int64)
    for j, off in enumerate(offsets):
        ok = np.ones(n, dtype=bool)
        delta = 0
        for d, o in enumerate(off):
            if o:
                ok &= (idx[d] + o >= 0) & (idx[d] + o < shape[d])
                delta += o * int(strides[d])
        mask[:, j] = ok
        cols[:, j] = (ar + delta).astype(np.int32)
        vals[:, j] = weights[j]
    lens = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    return _finish(rowptr, cols[mask], vals[mask])


def poisson1d(n: int, diag: float = 2.0, off: float = -1.0):
    """Tridiagonal 1D Poisson matrix (2 on the diagonal, -1 beside it; Section 4.2)."""
    return _from_offsets((n,), [(-1,), (0,), (1,)], [off, diag, off])


def poisson2d(nx: int, ny: int | None = None):
    """5-point 2D Poisson stencil, 4 on the diagonal and -1 for the four
    neighbours, natural (row-major) ordering, no 1/h^2 scaling.  64x64 gives
    n = 4096 and nnz = 20224."""
    ny = nx if ny is None else ny
    offs = [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    return _from_offsets((ny, nx), offs, [-1.0, -1.0, 4.0, -1.0, -1.0])


def stencil27(N: int):
    """27-point stencil on an N^3 grid: 26 on the diagonal, -1 for each of the
    26 neighbours.  N = 128 gives n = 2,097,152 and nnz = 55,742,968."""
    offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    w = [26.0 if o == (0, 0, 0) else -1.0 for o in offs]
    return _from_offsets((N, N, N), offs, w)


def _coo_to_csr(n_rows, r, c, v, sum_duplicates=True):
    key = r.astype(np.int64) * np.int64(max(n_rows, 1)) + c.astype(np.int64)
    order = np.argsort(key, kind="stable")
    key = key[order]
    v = v[order]
    if sum_duplicates and key.size:
        first = np.ones(key.size, dtype=bool)
        first[1:] = key[1:] != key[:-1]
        starts = np.flatnonzero(first)
        v = np.add.reduceat(v, starts)
        key = key[starts]
    r = key // max(n_rows, 1)
    c = key % max(n_rows, 1)
    rowptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n_rows), out=rowptr[1:])
    return _finish(rowptr, c, v)


def powerlaw(n: int, alpha: float = 1.8, cap: int = 10_000, seed: int = 3):
    """Power-law SPD matrix.

    B: row lengths l ~ P(l = k) proportional to k^-alpha on k = 1..cap, columns
    uniform over [0, n) (repeats within a row dropped, so a row holds distinct
    columns), values N(0, 1).  A = B + B^T on the union pattern (coinciding
    entries summed), then a_ii = sum_{j != i} |a_ij| + 1, making A strictly
    diagonally dominant with a positive diagonal, hence SPD.
    """
    rng = np.random.default_rng(seed)
    k = np.arange(1, cap + 1, dtype=np.float64)
    p = k ** (-alpha)
    p /= p.sum()
    lens = rng.choice(np.arange(1, cap + 1), size=n, p=p)
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    cols = rng.integers(0, n, size=rows.size, dtype=np.int64)
    vals = rng.standard_normal(rows.size)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key, vals = key[first], vals[first]
    r, c = key // n, key % n
    off = r != c
    r, c, vals = r[off], c[off], vals[off]
    R = np.concatenate([r, c])
    C = np.concatenate([c, r])
    V = np.concatenate([vals, vals])
    rowptr, col, val = _coo_to_csr(n, R, C, V)
    rows_of = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    diag = np.bincount(rows_of, weights=np.abs(val), minlength=n) + 1.0
    R2 = np.concatenate([rows_of, np.arange(n)])
    C2 = np.concatenate([col.astype(np.int64), np.arange(n)])
    V2 = np.concatenate([val, diag])
    return _coo_to_csr(n, R2, C2, V2, sum_duplicates=False)


def random_csr(m: int, n: int, seed: int, max_len: int | None = None, empty_frac: float = 0.1,
               long_rows: int = 0, long_len: int | None = None, values: str = "normal"):
    """Random rectangular CSR with uneven rows, some empty rows and optionally
    a few long rows (lengths capped at ``n``)."""
    rng = np.random.default_rng(seed)
    max_len = min(n, max_len if max_len is not None else max(1, min(n, 40)))
    lens = rng.integers(0, max_len + 1, size=m)
    lens[rng.random(m) < empty_frac] = 0
    if long_rows and m:
        ll = min(n, long_len if long_len is not None else n)
        lens[rng.choice(m, size=min(long_rows, m), replace=False)] = ll
    cols = [np.sort(rng.choice(n, size=int(l), replace=False)) for l in lens]
    col = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    if values == "normal":
        val = rng.standard_normal(col.size)
    else:
        val = rng.uniform(-1.0, 1.0, size=col.size)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    return _finish(rowptr, col, val)


def diagonal(d):
    d = np.asarray(d, dtype=np.float64)
    n = d.size
    return _finish(np.arange(n + 1), np.arange(n), d)


def scaled_identity(n: int, c: float):
    return diagonal(np.full(n, c))


def convdiff2d(nx: int, wind: float = 0.5):
    """Nonsymmetric 2D convection-diffusion (first-order upwind, wind along
    +x): 4 + wind on the diagonal, -1 - wind for the upwind x-neighbour, -1
    for the other three neighbours."""
    offs = [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    return _from_offsets((nx, nx), offs, [-1.0, -1.0 - wind, 4.0 + wind, -1.0, -1.0])


def uniform_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def csr_to_dense(A, n_cols: int | None = None):
    rowptr, col, val = A
    m = rowptr.size - 1
    n_cols = m if n_cols is None else n_cols
    D = np.zeros((m, n_cols))
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    D[rows, col] = val
    return D


def varcoef2d(coef):
    """5-point variable-coefficient diffusion on an (ny, nx) grid of cell
    coefficients: face coefficient = harmonic mean of the two cells, faces on
    the boundary take the cell's own coefficient (homogeneous Dirichlet);
    a_ii = sum of the cell's four faces, a_ij = -face.  SPD."""
    coef = np.asarray(coef, dtype=np.float64)
    ny, nx = coef.shape
    n = nx * ny
    hm = lambda a, b: 2.0 * a * b / (a + b)
    west = np.empty_like(coef)
    east = np.empty_like(coef)
    south = np.empty_like(coef)
    north = np.empty_like(coef)
    west[:, 0] = coef[:, 0]
    west[:, 1:] = hm(coef[:, 1:], coef[:, :-1])
    east[:, -1] = coef[:, -1]
    east[:, :-1] = hm(coef[:, :-1], coef[:, 1:])
    south[0, :] = coef[0, :]
    south[1:, :] = hm(coef[1:, :], coef[:-1, :])
    north[-1, :] = coef[-1, :]
    north[:-1, :] = hm(coef[:-1, :], coef[1:, :])
    diag = (west + east + south + north).ravel()
    offs = [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    rowptr, col, _ = _from_offsets((ny, nx), offs, [1.0] * 5)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    delta = col.astype(np.int64) - rows
    val = np.empty(col.size)
    val[delta == 0] = diag[rows[delta == 0]]
    val[delta == -nx] = -south.ravel()[rows[delta == -nx]]
    val[delta == nx] = -north.ravel()[rows[delta == nx]]
    val[delta == -1] = -west.ravel()[rows[delta == -1]]
    val[delta == 1] = -east.ravel()[rows[delta == 1]]
    return _finish(rowptr, col, val)


def batch_varcoef2d(n_sys: int, seed: int = 5, side_lo: int = 6, side_hi: int = 32, sigma: float = 0.5):
    """Batch of independent 2D variable-coefficient systems: side ~ U{lo..hi},
    cell coefficients log-normal(0, sigma).  Returns (sys_ptr int64[n_sys+1],
    block-diagonal CSR triple)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=n_sys)
    rps, cols, vals = [], [], []
    sys_ptr = np.zeros(n_sys + 1, dtype=np.int64)
    nnz_off = 0
    for s, side in enumerate(sides):
        coef = np.exp(sigma * rng.standard_normal((side, side)))
        rp, c, v = varcoef2d(coef)
        r0 = sys_ptr[s]
        sys_ptr[s + 1] = r0 + side * side
        rps.append(rp[:-1].astype(np.int64) + nnz_off)
        cols.append(c.astype(np.int64) + r0)
        vals.append(v)
        nnz_off += c.size
    rowptr = np.concatenate(rps + [np.array([nnz_off])])
    return sys_ptr, _finish(rowptr, np.concatenate(cols), np.concatenate(vals))


def varcoef3d_from(coef):
    """7-point variable-coefficient diffusion on an (nz, ny, nx) grid of cell
    coefficients (slowest axis first): the face between two cells carries the
    harmonic mean of their coefficients, a face on the grid boundary the
    cell's own coefficient (homogeneous Dirichlet); a_ii = the sum of the
    cell's six faces, a_ij = -face.  SPD.  Built one stencil offset at a time
    so that a 256^3 grid needs little more memory than the matrix."""
    c = np.asarray(coef, dtype=np.float64)
    shape = c.shape
    n = c.size
    hm = lambda a, b: 2.0 * a * b / (a + b)
    # faces[(axis, side)]: coefficient of the face towards the neighbour at
    # offset side (-1 or +1) along axis, per cell
    faces = {}
    for ax in range(3):
        lo = np.empty_like(c)
        hi = np.empty_like(c)
        sl = lambda a, b: tuple(slice(a, b) if d == ax else slice(None) for d in range(3))
        inner = hm(c[sl(1, None)], c[sl(None, -1)])
        lo[sl(1, None)] = inner
        lo[sl(0, 1)] = c[sl(0, 1)]
        hi[sl(None, -1)] = inner
        hi[sl(-1, None)] = c[sl(-1, None)]
        faces[(ax, -1)] = lo.ravel()
        faces[(ax, 1)] = hi.ravel()
    diag = sum(faces.values())
    strides = (shape[1] * shape[2], shape[2], 1)
    # offsets in increasing column order
    offs = [(0, -1), (1, -1), (2, -1), None, (2, 1), (1, 1), (0, 1)]
    coords = [np.arange(shape[d]).reshape([-1 if e == d else 1 for e in range(3)]) for d in range(3)]
    masks = []
    for off in offs:
        if off is None:
            masks.append(None)
            continue
        ax, sd = off
        ok = (coords[ax] + sd >= 0) & (coords[ax] + sd < shape[ax])
        masks.append(np.broadcast_to(ok, shape).ravel())
    lens = np.ones(n, dtype=np.int64)
    for m in masks:
        if m is not None:
            lens += m
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    pos = rowptr[:-1].copy()
    rows = np.arange(n, dtype=np.int64)
    for off, m in zip(offs, masks):
        if off is None:
            col[pos] = rows
            val[pos] = diag
            pos += 1
            continue
        ax, sd = off
        idx = np.flatnonzero(m)
        col[pos[idx]] = idx + sd * strides[ax]
        val[pos[idx]] = -faces[off][idx]
        pos[idx] += 1
    return _finish(rowptr, col, val)


def varcoef3d(nx: int, sigma: float = 1.0, seed: int = 4):
    """varcoef3d_from on an nx^3 grid with i.i.d. log-normal(0, sigma) cell
    coefficients (the mixed-precision workload: nx = 256, sigma = 1)."""
    rng = np.random.default_rng(seed)
    coef = np.exp(sigma * rng.standard_normal((nx, nx, nx)))
    return varcoef3d_from(coef)


# ---------------------------------------------------------------------------
# learned warm start: diffusion with a random coefficient field
# ---------------------------------------------------------------------------

def grf_field(side: int, seed, n_modes: int = 16, corr: float = 0.1, sigma: float = 1.0):
    """Gaussian random field on the cell centres ((i + 1) / (side + 1)) of a
    side x side grid: a sum of n_modes cosines with wave vectors drawn from
    N(0, (1 / (2 pi corr))^2 I) and uniform phases, amplitude
    sigma * sqrt(2 / n_modes) -- a random-feature field with variance
    sigma^2 and squared-exponential correlation of length corr.  Each cosine
    is evaluated in separated form, cos(u + v) = cos u cos v - sin u sin v."""
    rng = np.random.default_rng(seed)
    k = rng.normal(0.0, 1.0 / (2.0 * np.pi * corr), size=(n_modes, 2))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    t = (np.arange(side) + 1.0) / (side + 1.0)
    u = 2.0 * np.pi * k[:, 0:1] * t[None, :] + phi[:, None]   # (modes, x)
    v = 2.0 * np.pi * k[:, 1:2] * t[None, :]                  # (modes, y)
    g = np.cos(v).T @ np.cos(u) - np.sin(v).T @ np.sin(u)     # (y, x)
    return sigma * np.sqrt(2.0 / n_modes) * g


def gaussian_bumps(side: int, seed, n_bumps: int = 4):
    """Source term: n_bumps Gaussian bumps with centres U[0.1, 0.9]^2, widths
    U[0.03, 0.08] and amplitudes U[-1, 1] on the cell centres (each bump the
    outer product of its two 1D profiles)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.1, 0.9, size=(n_bumps, 2))
    w = rng.uniform(0.03, 0.08, size=n_bumps)
    a = rng.uniform(-1.0, 1.0, size=n_bumps)
    t = (np.arange(side) + 1.0) / (side + 1.0)
    px = np.exp(-((t[None, :] - c[:, 0:1]) ** 2) / (2.0 * w[:, None] ** 2))  # (bumps, x)
    py = np.exp(-((t[None, :] - c[:, 1:2]) ** 2) / (2.0 * w[:, None] ** 2))  # (bumps, y)
    return (py * a[:, None]).T @ px


def grf_problem(side: int, index: int, base_seed: int = 6):
    """Problem `index` of the learned-warm-start family: g = GRF (16 modes,
    correlation 0.1, sigma 1), cell coefficients exp(g), the 5-point
    variable-coefficient operator of varcoef2d, b = h^2 f with f four
    Gaussian bumps (h = 1 / (side + 1)).  Returns (g, A, b); g and b are
    (side, side) / (side^2,) float64."""
    g = grf_field(side, (base_seed, index, 0))
    f = gaussian_bumps(side, (base_seed, index, 1))
    A = varcoef2d(np.exp(g))
    h = 1.0 / (side + 1.0)
    return g, A, (h * h) * f.ravel()


_PATTERN_CACHE = {}


def _varcoef2d_pattern(side: int):
    """CSR pattern of the 5-point stencil on a side x side grid and, per
    stencil position (south, west, centre, east, north), the entry indices
    and the rows they belong to."""
    if side not in _PATTERN_CACHE:
        offs = [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
        rowptr, col, _ = _from_offsets((side, side), offs, [1.0] * 5)
        rows = np.repeat(np.arange(side * side), np.diff(rowptr))
        delta = col.astype(np.int64) - rows
        pos = {d: (np.flatnonzero(delta == d), rows[delta == d]) for d in (-side, -1, 0, 1, side)}
        _PATTERN_CACHE[side] = (rowptr, col, pos)
    return _PATTERN_CACHE[side]


def varcoef2d_values(coef):
    """Values of varcoef2d(coef) on the fixed pattern of its grid (the same
    numbers as varcoef2d, without rebuilding the pattern)."""
    coef = np.asarray(coef, dtype=np.float64)
    side = coef.shape[0]
    rowptr, col, pos = _varcoef2d_pattern(side)
    hm = lambda a, b: 2.0 * a * b / (a + b)
    west = np.empty_like(coef)
    east = np.empty_like(coef)
    south = np.empty_like(coef)
    north = np.empty_like(coef)
    west[:, 0] = coef[:, 0]
    west[:, 1:] = hm(coef[:, 1:], coef[:, :-1])
    east[:, -1] = coef[:, -1]
    east[:, :-1] = hm(coef[:, :-1], coef[:, 1:])
    south[0, :] = coef[0, :]
    south[1:, :] = hm(coef[1:, :], coef[:-1, :])
    north[-1, :] = coef[-1, :]
    north[:-1, :] = hm(coef[:-1, :], coef[1:, :])
    val = np.empty(col.size)
    for d, face in ((-side, south), (side, north), (-1, west), (1, east)):
        idx, rows = pos[d]
        val[idx] = -face.ravel()[rows]
    idx, rows = pos[0]
    val[idx] = (west + east + south + north).ravel()[rows]
    return val


_STACK_CACHE = {}


def grf_stack(side: int, indices, base_seed: int = 6):
    """Problems `indices` of the learned-warm-start family stacked as one
    block-diagonal system: returns (g (S, side, side), b (S, side^2), CSR of
    the block-diagonal matrix).  Each block equals grf_problem's matrix.  The
    stacked pattern and the output buffers are cached per (side, S) and reused
    by the next call of the same shape (copy what must outlive it)."""
    rowptr, col, _ = _varcoef2d_pattern(side)
    n, nnz = side * side, col.size
    S = len(indices)
    key = (side, S)
    if key not in _STACK_CACHE:
        if S * nnz >= 2 ** 31:
            raise ValueError("stack too large for int32 indices")
        rp = np.empty(S * n + 1, dtype=np.int32)
        rp[:-1].reshape(S, n)[:] = rowptr[None, :-1] + (nnz * np.arange(S, dtype=np.int32))[:, None]
        rp[-1] = S * nnz
        cl = (col[None, :] + (n * np.arange(S, dtype=np.int32))[:, None]).ravel()
        _STACK_CACHE[key] = (rp, cl, np.empty((S, side, side)), np.empty((S, n)), np.empty((S, nnz)))
    rp, cl, gs, bs, vals = _STACK_CACHE[key]
    h = 1.0 / (side + 1.0)
    for k, i in enumerate(indices):
        gs[k] = grf_field(side, (base_seed, int(i), 0))
        bs[k] = (h * h) * gaussian_bumps(side, (base_seed, int(i), 1)).ravel()
        vals[k] = varcoef2d_values(np.exp(gs[k]))
    return gs, bs, (rp, cl, vals.reshape(-1))
