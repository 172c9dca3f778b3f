"""The CPU baseline's byte count (bench.oracle_exec_bytes) on plans whose
executor traffic has a closed form.

The algorithmic bytes of one execution are, per plan:
  SpMV:   8 per point (value) + 8 per column (x) + 8 per row (y)
          + 4 per PSC II point + 4 per (PSC II row + codelet) + 4 per PSC I
          offset-array entry + 64 per codelet descriptor;
  SpTRSV: 8 per off-diagonal point + 32 per row (1/L_ii, b, x written, x
          filled) + the same index terms + 4 per row whose f is not strided.
"""
import numpy as np
import pytest

import oracle
import synth

bench = pytest.importorskip("bench")


def _diag(n):
    return synth.CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                     np.arange(1, n + 1, dtype=np.float64))


def _bidiagonal(n):
    rows = [[0]] + [[r - 1, r] for r in range(1, n)]
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in r], np.int32)
    return synth.CSR(n, n, rp, ci, np.ones(ci.size))


@pytest.mark.parametrize("n", [8, 40])
def test_closed_forms(n):
    oracle.build()
    a, lo = _diag(n), _bidiagonal(n)
    # a diagonal matrix is one BLAS codelet (f, g, h all strided): no index
    # bytes, one descriptor
    pa = oracle.inspect(a, oracle.SPMV)
    assert pa.records.shape[0] == 1 and pa.records[0, 1] == oracle.BLAS
    spmv = 8 * n + 8 * n + 8 * n + 64
    # a chain is n levels of one row each: n single-row strided codelets, n - 1
    # off-diagonal points, no index bytes
    pl = oracle.inspect(lo, oracle.SPTRSV)
    assert pl.records.shape[0] == n and set(pl.records[:, 1]) == {oracle.BLAS}
    sptrsv = 8 * (n - 1) + 32 * n + 64 * n
    assert bench.oracle_exec_bytes([("d", a, lo, None, None)]) == spmv + sptrsv
