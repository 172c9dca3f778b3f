"""Pins for the synthetic inputs (no GPU): the benchmark and parity matrices
have the sizes their closed forms give, so the workloads the GPU is measured
on are the ones described, independently of the generator's code.

A k-point stencil on an m^d grid has one entry per (row, neighbour) pair
inside the grid: per dimension, the pairs of offsets -1, 0, +1 number
3m - 2, so a box stencil has (3m - 2)^d entries (times b^2 for b x b
blocks) and the 2d+1-point star has (2d + 1) m^d - 2 d m^(d-1).  Every
pattern here is symmetric with its diagonal stored, so the lower triangle
holds (nnz + n) / 2 entries.
"""
import numpy as np
import pytest

import synth


def star(m, d):
    n = m ** d
    return n, (2 * d + 1) * n - 2 * d * m ** (d - 1)


def box(m, d, b=1):
    return b * m ** d, b * b * (3 * m - 2) ** d


@pytest.mark.parametrize("name,sizes", [
    ("lap5_64", star(64, 2)),
    ("lap7_128", star(128, 3)),
    ("elast3x3_64", box(64, 3, 3)),
    ("st27_168", box(168, 3)),
])
def test_workload_sizes_match_closed_forms(name, sizes):
    n, nnz = sizes
    a, lo, x, b = synth.workload(name)
    assert (a.n_rows, a.n_cols, a.nnz) == (n, n, nnz)
    assert lo.nnz == (nnz + n) // 2
    assert len(x) == n and len(b) == n
    assert np.all(np.abs(x) <= 1) and np.all(np.abs(b) <= 1)
    # the lower triangle ends every row with its diagonal
    assert np.all(lo.colidx[lo.rowptr[1:] - 1] == np.arange(n))
    if nnz < 100_000_000:
        # strictly increasing columns inside every row
        rows = np.repeat(np.arange(n, dtype=np.int32), np.diff(a.rowptr))
        same = rows[1:] == rows[:-1]
        assert np.all(a.colidx[1:][same] > a.colidx[:-1][same])


def test_elasticity_rows_are_diagonally_dominant():
    a = synth.workload("elast3x3_64", scale=0.25)[0]
    rows = np.repeat(np.arange(a.n_rows), np.diff(a.rowptr))
    diag = rows == a.colidx
    off = np.bincount(rows[~diag], weights=np.abs(a.values[~diag]), minlength=a.n_rows)
    d = np.zeros(a.n_rows)
    d[rows[diag]] = a.values[diag]
    assert np.all(d > off)


def test_generators_are_seeded():
    a1 = synth.workload("lap7_128", scale=0.25)
    a2 = synth.workload("lap7_128", scale=0.25)
    assert np.array_equal(a1[2], a2[2]) and np.array_equal(a1[3], a2[3])
    p1 = synth.powerlaw(3000, 11)
    p2 = synth.powerlaw(3000, 11)
    assert np.array_equal(p1.colidx, p2.colidx) and np.array_equal(p1.values, p2.values)
