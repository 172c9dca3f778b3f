"""Seeded CSR matrix and vector generators with the shapes of the paper's workloads.

The paper evaluates on SPD matrices and their lower triangles with 0.05-130M
nonzeros (Section V).  Those matrices are not available here, so these
generators build synthetic stand-ins with the same structure classes:

* structured stencils (2-D 5-point, 3-D 7-point and 27-point Laplacians) with
  small-integer values, so that sums are exact in any order;
* an elasticity-like matrix with dense 3x3 blocks on a 27-point node stencil,
  symmetric N(0,1) off-diagonals and a diagonal of 1 + sum(|row|);
* an irregular power-law matrix whose row lengths follow a Zipf-like law with
  30% of the columns placed near the diagonal;
* small random patterns for brute-force tests.

All arrays are host numpy arrays: ``rowptr`` and ``colidx`` are int32, values
are float64, columns are sorted and unique inside each row.  Every generator
is deterministic in its ``seed``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 20211123


@dataclass
class CSR:
    n_rows: int
    n_cols: int
    rowptr: np.ndarray  # int32 [n_rows + 1]
    colidx: np.ndarray  # int32 [nnz]
    values: np.ndarray  # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr.astype(np.int64))


# ----------------------------------------------------------------------------
# structured stencils
# ----------------------------------------------------------------------------

def _stencil_pattern(dims, offsets, slab_rows=1 << 21):
    """CSR pattern of a box stencil on a grid with natural (x fastest) order.

    ``offsets`` is a list of (dx, dy, dz).  Returns rowptr, colidx and the
    index (into ``offsets`` sorted by linear offset) of each stored entry.
    """
    nx, ny, nz = dims
    n = nx * ny * nz
    lin = np.array([dx + nx * (dy + ny * dz) for dx, dy, dz in offsets], dtype=np.int64)
    order = np.argsort(lin, kind="stable")
    offs = [offsets[i] for i in order]
    lin = lin[order]
    k = len(offs)
    counts = np.empty(n, dtype=np.int64)
    cols_parts, which_parts = [], []
    plane = nx * ny
    zstep = max(1, slab_rows // max(plane, 1))
    for z0 in range(0, nz, zstep):
        z1 = min(nz, z0 + zstep)
        idx = np.arange(z0 * plane, z1 * plane, dtype=np.int64)
        ix = idx % nx
        iy = (idx // nx) % ny
        iz = idx // plane
        mask = np.empty((idx.size, k), dtype=bool)
        cols = np.empty((idx.size, k), dtype=np.int64)
        for j, (dx, dy, dz) in enumerate(offs):
            mask[:, j] = ((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
                          & (iz + dz >= 0) & (iz + dz < nz))
            cols[:, j] = idx + lin[j]
        counts[idx] = mask.sum(axis=1)
        cols_parts.append(cols[mask].astype(np.int32))
        which_parts.append(np.broadcast_to(np.arange(k, dtype=np.int8), (idx.size, k))[mask])
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = np.concatenate(cols_parts) if cols_parts else np.zeros(0, np.int32)
    which = np.concatenate(which_parts) if which_parts else np.zeros(0, np.int8)
    return rowptr, colidx, which, lin


def _check_int32(rowptr):
    if rowptr[-1] >= 2 ** 31:
        raise ValueError("matrix has more than 2^31-1 nonzeros")
    return rowptr.astype(np.int32)


def _constant_stencil(dims, offsets, diag, off):
    rowptr, colidx, which, lin = _stencil_pattern(dims, offsets)
    center = np.flatnonzero(lin == 0)[0]
    values = np.where(which == center, float(diag), float(off))
    n = dims[0] * dims[1] * dims[2]
    return CSR(n, n, _check_int32(rowptr), colidx, values.astype(np.float64))


def laplacian_5pt(nx: int, ny: int | None = None) -> CSR:
    """2-D 5-point Laplacian, values 4 on the diagonal and -1 off it."""
    ny = nx if ny is None else ny
    offs = [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    return _constant_stencil((nx, ny, 1), offs, 4.0, -1.0)


def laplacian_7pt(nx: int, ny: int | None = None, nz: int | None = None) -> CSR:
    """3-D 7-point Laplacian, values 6 on the diagonal and -1 off it."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    return _constant_stencil((nx, ny, nz), offs, 6.0, -1.0)


def _box27():
    return [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def stencil_27pt(nx: int, ny: int | None = None, nz: int | None = None) -> CSR:
    """3-D 27-point stencil, values 26 on the diagonal and -1 off it."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _constant_stencil((nx, ny, nz), _box27(), 26.0, -1.0)


# ----------------------------------------------------------------------------
# symmetric pseudo-random values from a counter-based hash
# ----------------------------------------------------------------------------

_M1 = np.uint64(0x9E3779B97F4A7C15)
_M2 = np.uint64(0xBF58476D1CE4E5B9)
_M3 = np.uint64(0x94D049BB133111EB)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    x = x + _M1
    x = (x ^ (x >> np.uint64(30))) * _M2
    x = (x ^ (x >> np.uint64(27))) * _M3
    return x ^ (x >> np.uint64(31))


def _pair_normal(lo: np.ndarray, hi: np.ndarray, n: int, seed: int) -> np.ndarray:
    """N(0,1) value that depends only on the unordered index pair (lo, hi)."""
    smix = _splitmix64(np.array([seed], dtype=np.uint64))[0]
    key = lo.astype(np.uint64) * np.uint64(n) + hi.astype(np.uint64)
    h1 = _splitmix64((key << np.uint64(1)) ^ smix)
    h2 = _splitmix64(((key << np.uint64(1)) | np.uint64(1)) ^ smix)
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _row_ids(rowptr: np.ndarray) -> np.ndarray:
    n = rowptr.size - 1
    return np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr.astype(np.int64)))


def _dominant_diagonal(rowptr, colidx, values):
    """Set each diagonal entry to 1 + sum of |off-diagonal| entries of its row."""
    rows = _row_ids(rowptr)
    isdiag = colidx.astype(np.int64) == rows
    absoff = np.where(isdiag, 0.0, np.abs(values))
    rsum = np.add.reduceat(absoff, rowptr[:-1].astype(np.int64)) if values.size else absoff
    lens = np.diff(rowptr.astype(np.int64))
    rsum = np.where(lens > 0, rsum, 0.0)
    values[isdiag] = 1.0 + rsum[rows[isdiag]]
    return values


def elasticity_blocks(nn: int, seed: int = SEED_BASE + 2, dof: int = 3) -> CSR:
    """Elasticity-like matrix: dense dof x dof blocks on a 27-point node stencil.

    Nodes lie on an nn^3 grid; each node carries ``dof`` unknowns numbered
    consecutively.  Off-diagonal values are symmetric N(0,1); the diagonal is
    1 + sum(|off-diagonal|) of its row.
    """
    nrp, ncol, _, _ = _stencil_pattern((nn, nn, nn), _box27())
    nnodes = nn ** 3
    deg = np.diff(nrp)
    # expanded node pattern: each node column q becomes dof columns dof*q + b
    exp_cols = ((dof * ncol.astype(np.int64))[:, None] + np.arange(dof)).reshape(-1)
    seg_len = dof * deg                      # row length of every dof row of node p
    lens = np.repeat(seg_len, dof)           # dof rows per node
    n = dof * nnodes
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    seg_start = np.repeat(dof * nrp[:-1], dof)
    total = int(rowptr[-1])
    within = np.arange(total, dtype=np.int64) - np.repeat(rowptr[:-1], lens)
    colidx64 = exp_cols[np.repeat(seg_start, lens) + within]
    del within
    rows = _row_ids(rowptr)
    lo = np.minimum(rows, colidx64)
    hi = np.maximum(rows, colidx64)
    values = _pair_normal(lo, hi, n, seed)
    del lo, hi, rows
    colidx = colidx64.astype(np.int32)
    del colidx64
    values = _dominant_diagonal(rowptr, colidx, values)
    return CSR(n, n, _check_int32(rowptr), colidx, values)


# ----------------------------------------------------------------------------
# irregular power-law matrix
# ----------------------------------------------------------------------------

def powerlaw(n: int, seed: int = SEED_BASE + 3, scale: float = 2.5241, tail: float = 1.1,
             max_len: int = 20000, p_near: float = 0.3, band: int = 64) -> CSR:
    """Irregular matrix with Zipf-like row lengths (mean about 16).

    Row length k = floor(scale * U^(-1/tail)), redrawn while k > max_len.  Each
    drawn column lies with probability ``p_near`` within +-``band`` of the
    diagonal (clamped to the matrix), otherwise uniformly in [0, n).  Columns
    are de-duplicated and the diagonal is always present.  Values are N(0,1).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    u = 1.0 - rng.random(n)
    k = np.floor(scale * u ** (-1.0 / tail)).astype(np.int64)
    bad = np.flatnonzero(k > max_len)
    while bad.size:
        u = 1.0 - rng.random(bad.size)
        k[bad] = np.floor(scale * u ** (-1.0 / tail)).astype(np.int64)
        bad = bad[k[bad] > max_len]
    total = int(k.sum())
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    near = rng.random(total) < p_near
    shift = rng.integers(-band, band + 1, size=total)
    far = rng.integers(0, n, size=total)
    cols = np.where(near, np.clip(rows + shift, 0, n - 1), far)
    del near, shift, far
    keys = np.concatenate([rows * n + cols, np.arange(n, dtype=np.int64) * (n + 1)])
    del rows, cols
    # sorted distinct keys (a sort and a neighbour compare: np.unique on tens
    # of millions of int64 keys is far slower and gives the same array)
    keys.sort()
    if keys.size:
        keys = keys[np.concatenate([[True], keys[1:] != keys[:-1]])]
    r = keys // n
    c = (keys - r * n).astype(np.int32)
    del keys
    counts = np.bincount(r, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    values = rng.standard_normal(c.size)
    return CSR(n, n, _check_int32(rowptr), c, values)


# ----------------------------------------------------------------------------
# lower triangles, small random patterns, vectors
# ----------------------------------------------------------------------------

def lower_triangle(a: CSR, diag: str = "keep") -> CSR:
    """Lower triangle of ``a`` including the diagonal.

    ``diag='keep'`` keeps the stored diagonal; ``diag='unit_dominant'`` sets
    L_ii = 1 + sum_{j<i} |L_ij|.  Every row of ``a`` must hold its diagonal.
    """
    rows = _row_ids(a.rowptr)
    keep = a.colidx.astype(np.int64) <= rows
    counts = np.bincount(rows[keep], minlength=a.n_rows)
    rowptr = np.zeros(a.n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = a.colidx[keep]
    values = a.values[keep].copy()
    if diag == "unit_dominant":
        values = _dominant_diagonal(rowptr, colidx, values)
    elif diag != "keep":
        raise ValueError(diag)
    return CSR(a.n_rows, a.n_cols, _check_int32(rowptr), colidx, values)


def random_pattern(n_rows: int, n_cols: int, density: float, seed: int, *, diag: bool = False,
                   lower: bool = False, values: str = "normal", empty_rows: float = 0.0) -> CSR:
    """Small random CSR matrix for brute-force tests.

    ``values`` is 'normal' (N(0,1)) or 'int' (integers in [-3, 3] without 0).
    With ``lower=True`` only columns <= row are kept; with ``diag=True`` the
    diagonal is present (diagonally dominant when ``values='normal'``, equal
    to 1 when ``values='int'`` so that forward substitution stays exact).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dense = rng.random((n_rows, n_cols)) < density
    if empty_rows > 0:
        dense[rng.random(n_rows) < empty_rows] = False
    if lower:
        dense &= np.tri(n_rows, n_cols, dtype=bool)
    if diag:
        m = min(n_rows, n_cols)
        dense[np.arange(m), np.arange(m)] = True
    r, c = np.nonzero(dense)
    counts = np.bincount(r, minlength=n_rows)
    rowptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if values == "int":
        v = rng.integers(1, 4, size=r.size) * rng.choice([-1, 1], size=r.size)
        v = v.astype(np.float64)
        if diag:
            v[r == c] = 1.0
    else:
        v = rng.standard_normal(r.size)
        if diag:
            v = _dominant_diagonal(rowptr, c.astype(np.int32), v)
    return CSR(n_rows, n_cols, rowptr.astype(np.int32), c.astype(np.int32), v)


def banded(n: int, half_bw: int, seed: int = SEED_BASE + 6) -> CSR:
    """Band matrix: row i holds columns max(0, i - half_bw) .. min(n - 1, i +
    half_bw), all of them, with symmetric N(0,1) off-diagonals and a diagonal
    of 1 + sum(|row|).  Every interior row is a run of contiguous columns one
    further right than the row before, the pattern of a BLAS codelet."""
    lo = np.maximum(np.arange(n, dtype=np.int64) - half_bw, 0)
    hi = np.minimum(np.arange(n, dtype=np.int64) + half_bw, n - 1)
    lens = hi - lo + 1
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    total = int(rowptr[-1])
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    cols = np.repeat(lo, lens) + (np.arange(total, dtype=np.int64) - np.repeat(rowptr[:-1], lens))
    values = _pair_normal(np.minimum(rows, cols), np.maximum(rows, cols), n, seed)
    colidx = cols.astype(np.int32)
    del rows, cols
    values = _dominant_diagonal(rowptr, colidx, values)
    return CSR(n, n, _check_int32(rowptr), colidx, values)


def chain(n: int) -> CSR:
    """Lower bidiagonal matrix (1 on the diagonal, -1/2 below): every row reads
    the one before it, so its dependency graph is one path of n levels."""
    rp = np.zeros(n + 1, np.int32)
    if n > 0:
        rp[1:] = 2 * np.arange(1, n + 1, dtype=np.int32) - 1
    ci = np.empty(max(2 * n - 1, 0), np.int32)
    v = np.empty(max(2 * n - 1, 0), np.float64)
    if n > 0:
        ci[0] = 0
        v[0] = 1.0
        r = np.arange(1, n, dtype=np.int32)
        ci[1::2] = r - 1
        ci[2::2] = r
        v[1::2] = -0.5
        v[2::2] = 1.0
    return CSR(n, n, rp, ci, v)


def uniform_vector(n: int, seed: int) -> np.ndarray:
    """x ~ U[-1, 1]^n."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, n)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def _w_5pt(scale):
    k = max(4, int(64 * scale))
    return laplacian_5pt(k)


def _w_7pt(scale):
    k = max(4, int(round(128 * scale)))
    return laplacian_7pt(k)


def _w_elast(scale):
    k = max(3, int(round(64 * scale)))
    return elasticity_blocks(k)


def _w_powerlaw(scale):
    return powerlaw(max(1024, int((1 << 22) * scale)))


def _w_27pt(scale):
    k = max(4, int(round(168 * scale)))
    return stencil_27pt(k)


def _w_27pt_normal(scale):
    # the 27-point pattern (one unknown per node) with symmetric N(0,1)
    # off-diagonals and a diagonal of 1 + sum(|row|): the value variant of the
    # precision form whose entries round in FP32 / BF16
    k = max(4, int(round(168 * scale)))
    return elasticity_blocks(k, seed=SEED_BASE + 5, dof=1)


#: name -> (builder(scale), diag rule for the SpTRSV lower triangle, seed)
WORKLOADS = {
    "lap5_64": (_w_5pt, "keep", SEED_BASE + 1),
    "lap7_128": (_w_7pt, "keep", SEED_BASE + 2),
    "elast3x3_64": (_w_elast, "keep", SEED_BASE + 2),
    "powerlaw_4m": (_w_powerlaw, "unit_dominant", SEED_BASE + 3),
    "st27_168": (_w_27pt, "keep", SEED_BASE + 4),
    "st27r_168": (_w_27pt_normal, "keep", SEED_BASE + 5),
}


def workload(name: str, scale: float = 1.0):
    """Return (A, L, x, b) for a named workload.

    A is the SpMV matrix, L its lower triangle (with the workload's diagonal
    rule), and x, b ~ U[-1,1] are the SpMV input and the SpTRSV right-hand
    side.  A manufactured right-hand side b = L x_true is a sparse product and
    therefore left to the caller.
    """
    build, diag_rule, seed = WORKLOADS[name]
    a = build(scale)
    lo = lower_triangle(a, diag_rule)
    x = uniform_vector(a.n_cols, seed)
    b = uniform_vector(a.n_rows, seed + 1000)
    return a, lo, x, b


# ----------------------------------------------------------------------------
# batch of uneven matrices (many small systems with many right-hand sides)
# ----------------------------------------------------------------------------

def _star(dims, radius):
    """Offsets of a star stencil: the centre and +-1..radius along each axis."""
    offs = [(0, 0, 0)]
    for ax in range(len(dims)):
        for r in range(1, radius + 1):
            for sgn in (-1, 1):
                o = [0, 0, 0]
                o[ax] = sgn * r
                offs.append(tuple(o))
    return offs


def _f32_dominant(rowptr, colidx, rng):
    """N(0,1) off-diagonals and a diagonal of 1 + sum(|row|), all exactly
    representable in FP32."""
    nnz = colidx.size
    v = rng.standard_normal(nnz).astype(np.float32).astype(np.float64)
    v = _dominant_diagonal(rowptr, colidx, v)
    return v.astype(np.float32).astype(np.float64)


def batch_member(n_target: int, kind: str, seed: int) -> CSR:
    """One matrix of the batch: a 2-D star stencil of radius 3 (13 points), a
    3-D star stencil of radius 2 (13 points) or a power-law pattern with mean
    row length 12; FP32-exact N(0,1) values made diagonally dominant."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "2d":
        k = max(4, int(round(n_target ** 0.5)))
        dims = (k, max(4, n_target // k), 1)
        rowptr, colidx, _, _ = _stencil_pattern(dims, _star(dims[:2], 3))
        n = dims[0] * dims[1]
    elif kind == "3d":
        k = max(4, int(round(n_target ** (1.0 / 3.0))))
        dims = (k, k, max(4, n_target // (k * k)))
        rowptr, colidx, _, _ = _stencil_pattern(dims, _star(dims, 2))
        n = dims[0] * dims[1] * dims[2]
    else:
        a = powerlaw(n_target, seed=seed, scale=1.9, max_len=2000)
        v = _f32_dominant(a.rowptr.astype(np.int64), a.colidx, rng)
        return CSR(a.n_rows, a.n_cols, a.rowptr, a.colidx, v)
    rowptr = rowptr.astype(np.int64)
    v = _f32_dominant(rowptr, colidx, rng)
    return CSR(n, n, _check_int32(rowptr), colidx, v)


def batch(count: int = 256, n_min: int = 1000, n_max: int = 200000, nrhs: int = 32,
          seed: int = SEED_BASE + 5):
    """(matrices, right-hand sides): ``count`` matrices with n log-uniform in
    [n_min, n_max], each a random 2-D / 3-D star stencil or power-law pattern,
    and for each an (n x nrhs) row-major float32 block of U[-1, 1] right-hand sides."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(np.log(n_min), np.log(n_max), count)).astype(np.int64)
    kinds = rng.choice(["2d", "3d", "powerlaw"], size=count)
    mats, rhs = [], []
    for i in range(count):
        m = batch_member(int(sizes[i]), str(kinds[i]), seed * 1000 + i)
        mats.append(m)
        rhs.append(np.random.Generator(np.random.PCG64(seed + 7 + i))
                   .uniform(-1.0, 1.0, (m.n_rows, nrhs)).astype(np.float32))
    return mats, rhs
