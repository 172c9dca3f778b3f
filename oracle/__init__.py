"""CPU oracle for the DDF hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this package.  It never imports the CUDA path
and the CUDA path never imports it.

The heavy definitions live in plain C (``ddf_oracle.c``: CSR SpMV, forward
substitution, levels, Algorithm 1, the plan-expansion check), compiled with
``-O2 -ffp-contract=off`` and loaded through ctypes.  ``oracle.fopd`` holds the
trace-level definitions of Section III-D written out in numpy.

Arrays are taken from any object with ``n_rows``, ``rowptr`` (int32),
``colidx`` (int32) and ``values`` (float64) attributes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libddf_oracle.so")

SPMV, SPTRSV = 1, 2
BLAS, PSC1, PSC2 = 0, 1, 2
ALLOW_BLAS, ALLOW_PSC1, ALLOW_PSC2 = 1, 2, 4
ALLOW_ALL = 7
#: Eq. 1 exactly as printed: |p| + m + sum |s_d| with m = 3 access functions
PAPER_WEIGHTS = (1, 3, 1)
#: rows per block of coarsened SpTRSV partitions; the CUDA library's default
#: option value, so that default plans on both sides are comparable
DEFAULT_COARSEN = 0
#: record layout of one codelet (12 x int64)
FIELDS = ("part", "type", "q0", "m", "n", "f_str", "rho", "g_str", "gamma", "h0", "delta", "sigma")

ERR = {0: "ok", 1: "bad argument", 5: "entry above the diagonal", 6: "missing diagonal",
       7: "zero diagonal", 9: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (in-tree, ignored by git)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        lib.ora_spmv_csr.argtypes = [i32, P, P, P, P, P]
        lib.ora_spmv_csr_par.argtypes = [i32, P, P, P, P, P, i32]
        lib.ora_sptrsv_csr.argtypes = [i32, P, P, P, P, P]
        lib.ora_levels.argtypes = [i32, P, P, P]
        lib.ora_levels.restype = i32
        lib.ora_level_order.argtypes = [i32, P, i32, P, P]
        lib.ora_coarse_order.argtypes = [i32, P, i32, i32, P, P, P]
        lib.ora_check_schedule.argtypes = [i32, P, P, P, P, i32, P]
        lib.ora_codelet_cost.argtypes = [i64] * 7
        lib.ora_codelet_cost.restype = i64
        lib.ora_inspect.argtypes = [ctypes.c_int, i32, P, P, i32, ctypes.c_int, P, i32, P, P, P, P,
                                    ctypes.POINTER(ctypes.POINTER(i64)), ctypes.POINTER(i64)]
        lib.ora_check_plan.argtypes = [ctypes.c_int, i32, P, P, P, P, i32, P, P, i64,
                                       ctypes.POINTER(i64)]
        lib.ora_free.argtypes = [P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(a):
    rp = np.ascontiguousarray(a.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(a.colidx, dtype=np.int32)
    return int(a.n_rows), rp, ci


class OracleError(RuntimeError):
    pass


def spmv(a, x: np.ndarray) -> np.ndarray:
    """y = A x, FP64, row by row in CSR order (Fig. 1a)."""
    n, rp, ci = _csr(a)
    v = np.ascontiguousarray(a.values, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n, dtype=np.float64)
    _L().ora_spmv_csr(n, _p(rp), _p(ci), _p(v), _p(x), _p(y))
    return y


def spmv_par(a, x: np.ndarray, threads: int | None = None) -> np.ndarray:
    """y = A x with the rows split over ``threads`` host threads (default: all
    cores); every row is summed in CSR order, so y equals ``spmv`` exactly."""
    n, rp, ci = _csr(a)
    v = np.ascontiguousarray(a.values, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n, dtype=np.float64)
    t = threads or os.cpu_count() or 1
    rc = _L().ora_spmv_csr_par(n, _p(rp), _p(ci), _p(v), _p(x), _p(y), int(t))
    if rc:
        raise OracleError(ERR.get(rc, str(rc)))
    return y


def sptrsv(lo, b: np.ndarray) -> np.ndarray:
    """Forward substitution L x = b with true division by the diagonal."""
    n, rp, ci = _csr(lo)
    v = np.ascontiguousarray(lo.values, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(n, dtype=np.float64)
    rc = _L().ora_sptrsv_csr(n, _p(rp), _p(ci), _p(v), _p(b), _p(x))
    if rc:
        raise OracleError(ERR.get(rc, str(rc)))
    return x


def levels(lo):
    """Longest-path level of every row of G(L) and the depth."""
    n, rp, ci = _csr(lo)
    lev = np.empty(max(n, 1), dtype=np.int32)
    depth = _L().ora_levels(n, _p(rp), _p(ci), _p(lev))
    if depth < 0:
        raise OracleError("entry above the diagonal")
    return lev[:n], int(depth)


def level_order(lev: np.ndarray, depth: int):
    """(level_ptr, perm): rows sorted by (level, row)."""
    n = lev.size
    lev = np.ascontiguousarray(lev, dtype=np.int32)
    lp = np.empty(depth + 1, dtype=np.int32)
    perm = np.empty(max(n, 1), dtype=np.int32)
    _L().ora_level_order(n, _p(lev), depth, _p(lp), _p(perm))
    return lp, perm[:n]


def coarse_order(lev: np.ndarray, depth: int, rows_per_block: int):
    """(part_ptr, perm): rows sorted by (row // R, level, row); one partition per
    non-empty (block, level) pair (LBC-style coarsening, Sec. IV-A)."""
    n = lev.size
    lev = np.ascontiguousarray(lev, dtype=np.int32)
    pp = np.empty(n + 1, dtype=np.int32)
    perm = np.empty(max(n, 1), dtype=np.int32)
    npart = ctypes.c_int32(0)
    rc = _L().ora_coarse_order(n, _p(lev), depth, int(rows_per_block), _p(pp), _p(perm), ctypes.byref(npart))
    if rc:
        raise OracleError(ERR.get(rc, str(rc)))
    return pp[:npart.value + 1].copy(), perm[:n].copy()


def check_schedule(lo, perm, part_ptr):
    """(code, row): code 0 when every dependency of every row lies in a strictly
    earlier partition; 1 (with the row) when one does not; 2 when malformed."""
    n, rp, ci = _csr(lo)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    pp = np.ascontiguousarray(part_ptr, dtype=np.int32)
    bad = ctypes.c_int32(-1)
    rc = _L().ora_check_schedule(n, _p(rp), _p(ci), _p(perm), _p(pp), pp.size - 1, ctypes.byref(bad))
    return int(rc), int(bad.value)


def codelet_cost(p, s_f, s_g, s_h, weights=PAPER_WEIGHTS) -> int:
    """Eq. 1: c = w_op |p| + w_cl + w_idx (|s_f| + |s_g| + |s_h|)."""
    return int(_L().ora_codelet_cost(p, s_f, s_g, s_h, *weights))


@dataclass
class Plan:
    kind: int
    records: np.ndarray    # (ncodelets, 12) int64, FIELDS order
    perm: np.ndarray       # int32 [n]   partition sequence
    level_ptr: np.ndarray  # int32 [nparts + 1]
    gs: np.ndarray         # int64 [n]   value offset of each position

    @property
    def nparts(self) -> int:
        return self.level_ptr.size - 1


def inspect(a, kind: int, t: int = 256, allowed: int = ALLOW_ALL,
            weights=(8, 32, 4), coarsen: int = DEFAULT_COARSEN) -> Plan:
    """Algorithm 1 on the pattern of ``a`` for kind SPMV or SPTRSV.

    ``coarsen`` = R > 0 partitions a SpTRSV by (block of R rows, level)
    (LBC-style coarsening, Sec. IV-A); 0 gives the plain level sets."""
    n, rp, ci = _csr(a)
    perm = np.empty(max(n, 1), dtype=np.int32)
    lp = np.empty(n + 2, dtype=np.int32)
    nparts = ctypes.c_int32(0)
    gs = np.empty(max(n, 1), dtype=np.int64)
    w = np.asarray(weights, dtype=np.int64)
    out = ctypes.POINTER(ctypes.c_int64)()
    ncod = ctypes.c_int64(0)
    rc = _L().ora_inspect(kind, n, _p(rp), _p(ci), int(t), int(allowed), _p(w), int(coarsen), _p(perm), _p(lp),
                          ctypes.byref(nparts), _p(gs), ctypes.byref(out), ctypes.byref(ncod))
    if rc:
        raise OracleError(ERR.get(rc, str(rc)))
    k = int(ncod.value)
    if k:
        recs = np.ctypeslib.as_array(out, shape=(k, len(FIELDS))).copy()
    else:
        recs = np.zeros((0, len(FIELDS)), dtype=np.int64)
    _L().ora_free(ctypes.cast(out, ctypes.c_void_p))
    npart = int(nparts.value)
    return Plan(kind, recs, perm[:n].copy(), lp[:npart + 1].copy(), gs[:n].copy())


def check_plan(a, kind: int, perm, level_ptr, gs, records):
    """Plan-expansion check.  Returns (code, index); code 0 means valid."""
    n, rp, ci = _csr(a)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    lp = np.ascontiguousarray(level_ptr, dtype=np.int32)
    gs = np.ascontiguousarray(gs, dtype=np.int64)
    rec = np.ascontiguousarray(records, dtype=np.int64)
    bad = ctypes.c_int64(-1)
    rc = _L().ora_check_plan(kind, n, _p(rp), _p(ci), _p(perm), _p(lp), lp.size - 1, _p(gs),
                             _p(rec), rec.shape[0], ctypes.byref(bad))
    return int(rc), int(bad.value)


def plan_cost(a, plan: Plan, weights) -> int:
    """Sum of Eq. 1 over every codelet of a plan (used to compare strategies)."""
    n, rp, ci = _csr(a)
    lens = np.diff(rp.astype(np.int64))[plan.perm]
    if plan.kind == SPTRSV:
        lens = lens - 1
    total = 0
    for r in plan.records:
        q0, m, typ = int(r[2]), int(r[3]), int(r[1])
        p = int(lens[q0:q0 + m].sum())
        if typ == BLAS:
            s = (0, 0, 0)
        elif typ == PSC1:
            s = (0, 0, int(lens[q0]))
        else:
            s = (0 if r[5] else m, 0 if r[7] else m, p)
        total += codelet_cost(p, *s, weights=weights)
    return total
