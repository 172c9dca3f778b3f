"""Trace-level definitions of Section III (oracle, test infrastructure only).

These functions take the access functions of one codelet as explicit tables
over its iteration space I = [i0, i1] (numpy arrays of shape (m, n)) and apply
the paper's definitions literally:

* first order partial differences (Sec. III-D):
  Delta_{i0} f = f(i0+1, i1) - f(i0, i1),  Delta_{i1} f = f(i0, i1+1) - f(i0, i1);
* a function is strided when all its Delta_{i0} are equal and all its
  Delta_{i1} are equal (Sec. III-D), i.e. it is a linear combination of the
  induction variables plus a constant (Sec. III-A);
* the codelet class is the number of strided functions (Sec. III-B): all
  three -> BLAS, two -> PSC I, one -> PSC II;
* memory accesses of a function (Sec. III-C): 1 when strided, |s| + 1 when it
  is expressed through an offset array s;
* Eq. 1 is in ``oracle.codelet_cost``.
"""
from __future__ import annotations

import numpy as np

CLASS_NAMES = {3: "BLAS", 2: "PSC I", 1: "PSC II", 0: "none strided"}


def fopd_i0(t: np.ndarray) -> np.ndarray:
    """Delta_{i0} t over the table (shape (m-1, n))."""
    t = np.asarray(t, dtype=np.int64)
    return t[1:, :] - t[:-1, :]


def fopd_i1(t: np.ndarray) -> np.ndarray:
    """Delta_{i1} t over the table (shape (m, n-1))."""
    t = np.asarray(t, dtype=np.int64)
    return t[:, 1:] - t[:, :-1]


def _all_equal(d: np.ndarray) -> bool:
    return d.size == 0 or bool(np.all(d == d.flat[0]))


def is_strided(t: np.ndarray) -> bool:
    """Strided <=> every Delta_{i0} equal and every Delta_{i1} equal."""
    return _all_equal(fopd_i0(t)) and _all_equal(fopd_i1(t))


def classify(f: np.ndarray, g: np.ndarray, h: np.ndarray):
    """(strided flags (f, g, h), class name) of a codelet given its tables."""
    flags = tuple(is_strided(t) for t in (f, g, h))
    return flags, CLASS_NAMES[sum(flags)]


def shared_offsets(h: np.ndarray):
    """If h(i0, i1) = h0 + delta*i0 + s[i1] for one offset array s, return
    (h0, delta, s); otherwise None."""
    h = np.asarray(h, dtype=np.int64)
    if h.shape[1] == 0:
        return 0, 0, np.zeros(0, np.int64)
    d0 = fopd_i0(h)
    if d0.size and not np.all(d0 == d0.flat[0]):
        return None
    delta = int(d0.flat[0]) if d0.size else 0
    h0 = int(h[0, 0])
    return h0, delta, h[0, :] - h0


def loads(t: np.ndarray) -> int:
    """Memory accesses needed for one access function of a codelet: 1 when it
    is strided, else |s| + 1 with s the smallest offset array that expresses
    it (shared across rows when possible, else one entry per point)."""
    if is_strided(t):
        return 1
    so = shared_offsets(t)
    if so is not None:
        return so[2].size + 1
    return int(np.asarray(t).size) + 1


def spmv_tables(rowptr, colidx, rows):
    """(f, g, h) tables of SpMV ``y[i] += Ax[k] * x[Ai[k]]`` over the given rows,
    which must all have the same length (Sec. III-A, Fig. 2)."""
    rows = np.asarray(rows, dtype=np.int64)
    lens = rowptr[rows + 1].astype(np.int64) - rowptr[rows]
    if lens.size and not np.all(lens == lens[0]):
        raise ValueError("rows of unequal length do not form a rectangular iteration space")
    n = int(lens[0]) if lens.size else 0
    i1 = np.arange(n, dtype=np.int64)
    f = np.repeat(rows[:, None], n, axis=1)
    g = rowptr[rows].astype(np.int64)[:, None] + i1[None, :]
    h = colidx[g] if n else np.zeros((rows.size, 0), np.int64)
    return f, g, np.asarray(h, dtype=np.int64)


def sequence_tables(rowptr, colidx, seq, gs, q0, m, offdiag: bool):
    """(f, g, h) tables over positions q0..q0+m-1 of a partition sequence:
    f = seq[q], g = gs[q] + i1, h = colidx[rowptr[seq[q]] + i1]; with
    ``offdiag`` the last entry of each row (the diagonal) is left out."""
    qs = np.arange(q0, q0 + m)
    rows = np.asarray(seq, dtype=np.int64)[qs]
    lens = rowptr[rows + 1].astype(np.int64) - rowptr[rows] - (1 if offdiag else 0)
    if not np.all(lens == lens[0]):
        raise ValueError("unequal lengths")
    n = int(lens[0])
    i1 = np.arange(n, dtype=np.int64)
    f = np.repeat(rows[:, None], n, axis=1)
    g = np.asarray(gs, dtype=np.int64)[qs][:, None] + i1[None, :]
    h = colidx[rowptr[rows].astype(np.int64)[:, None] + i1[None, :]] if n else np.zeros((m, 0))
    return f, g, np.asarray(h, dtype=np.int64)


def is_strided_1d(v) -> bool:
    """A function of i0 alone (the row function f): strided when all its
    Delta_{i0} are equal.  Used for f, which is defined even on empty rows."""
    v = np.asarray(v, dtype=np.int64)
    d = v[1:] - v[:-1]
    return _all_equal(d)
