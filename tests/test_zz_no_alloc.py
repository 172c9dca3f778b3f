"""The allocation-free solve, checked against the CPU oracle and the plan-based solve.

ddf_sptrsv_csr_noalloc serves callers that must not allocate device memory
(for example code running inside an allocator hook, or under a fixed memory
budget): it keeps its scratch in a static device array instead of calling
cudaMalloc.  It is called here through the C ABI: twice in a row on the same
inputs (the second call reuses the scratch the first one left behind), each
result within 1e-12 of the oracle's forward substitution and of ddf_sptrsv on
a plan; an empty call as the warm-up; malformed rows, which must return their
statuses without reading out of bounds; a dependency wait that runs out (a
tiny limit on a long chain), which must return DDF_ERR_TIMEOUT and leave the
context usable; and the largest size the scratch holds.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2111_12243_gb300 as ddf
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12
CAP = 2_000_000_000


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_12243_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def relerr(y, ref):
    return float(np.linalg.norm(y - ref) / np.linalg.norm(ref))


def dev(v):
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()


def noalloc(lo, b, cap=CAP):
    """One call through the C ABI; returns (status, x on the host)."""
    rp, ci, va, bd = dev(lo.rowptr), dev(lo.colidx), dev(lo.values), dev(b)
    x = torch.full((lo.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = ddf.lib().ddf_sptrsv_csr_noalloc(lo.n_rows, lo.nnz, ctypes.c_void_p(rp.data_ptr()),
                                          ctypes.c_void_p(ci.data_ptr()), ctypes.c_void_p(va.data_ptr()),
                                          ctypes.c_void_p(bd.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                          int(cap), stream)
    return st, x.cpu().numpy()


def test_empty_call_is_the_warm_up():
    L = ddf.lib()
    assert L.ddf_sptrsv_csr_noalloc(0, 0, None, None, None, None, None, CAP, None) == 0


@pytest.mark.parametrize("name", ["lap7_24", "powerlaw_20000", "elast_6"])
def test_noalloc_matches_oracle_and_plan_solve_twice(name):
    if name == "lap7_24":
        lo = synth.lower_triangle(synth.laplacian_7pt(24))
    elif name == "elast_6":
        lo = synth.lower_triangle(synth.elasticity_blocks(6))
    else:
        lo = synth.lower_triangle(synth.powerlaw(20000), "unit_dominant")
    b = synth.uniform_vector(lo.n_rows, 3)
    ref = oracle.sptrsv(lo, b)
    plan = ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), dev(lo.values), lo.n_cols, ddf.DDF_SPTRSV)
    xp = torch.empty(lo.n_rows, dtype=torch.float64, device="cuda")
    ddf.ddf_sptrsv(plan, dev(b), xp)
    assert ddf.ddf_get_status(plan) == 0
    for _ in range(2):
        st, x = noalloc(lo, b)
        assert st == 0, ddf.ddf_status_string(st)
        assert relerr(x, ref) <= TOL
        assert relerr(x, xp.cpu().numpy()) <= TOL
        # the oracle's residual of the returned solution
        assert np.linalg.norm(b - oracle.spmv(lo, x)) / np.linalg.norm(b) <= TOL


def malformed(kind):
    """A 6-row lower triangle with one bad row."""
    rows = [[0], [0, 1], [1, 2], [0, 2, 3], [3, 4], [2, 4, 5]]
    vals = [[2.0], [1.0, 2.0], [1.0, 2.0], [1.0, 1.0, 2.0], [1.0, 2.0], [1.0, 1.0, 2.0]]
    if kind == "not_lower":       # row 3 names column 4, above the diagonal, before its diagonal
        rows[3] = [0, 4, 3]
        vals[3] = [1.0, 1.0, 2.0]
    elif kind == "missing_diag":  # row 4 ends before its diagonal
        rows[4] = [3]
        vals[4] = [1.0]
    elif kind == "zero_diag":     # row 2's diagonal is 0
        vals[2] = [1.0, 0.0]
    rp = np.zeros(7, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    return synth.CSR(6, 6, rp, np.array([c for r in rows for c in r], np.int32),
                     np.array([v for r in vals for v in r], np.float64))


@pytest.mark.parametrize("kind,code", [("not_lower", 5), ("missing_diag", 6), ("zero_diag", 7)])
def test_malformed_rows_return_their_status(kind, code):
    lo = malformed(kind)
    st, _ = noalloc(lo, np.ones(6))
    assert st == code, ddf.ddf_status_string(st)
    # the oracle refuses the same matrix
    with pytest.raises(oracle.OracleError):
        oracle.sptrsv(lo, np.ones(6))
    # the next call starts clean
    good = malformed("none")
    st, x = noalloc(good, np.ones(6))
    assert st == 0 and relerr(x, oracle.sptrsv(good, np.ones(6))) <= TOL


def test_wait_that_runs_out_returns_timeout_and_leaves_the_context_usable():
    # a chain of 2^18 rows: every CTA but the first waits on the rows of the
    # one before it, far longer than a 1 ns limit
    lo = synth.chain(1 << 18)
    b = synth.uniform_vector(lo.n_rows, 5)
    st, _ = noalloc(lo, b, cap=1)
    assert st == 11, ddf.ddf_status_string(st)
    torch.cuda.synchronize()
    st, x = noalloc(lo, b)
    assert st == 0 and relerr(x, oracle.sptrsv(lo, b)) <= TOL


def test_largest_size_and_beyond():
    n = ddf.DDF_NOALLOC_MAX_ROWS
    lo = synth.lower_triangle(synth.banded(n, 2))
    b = synth.uniform_vector(n, 6)
    st, x = noalloc(lo, b)
    assert st == 0, ddf.ddf_status_string(st)
    assert relerr(x, oracle.sptrsv(lo, b)) <= TOL
    L = ddf.lib()
    st = L.ddf_sptrsv_csr_noalloc(n + 1, 0, None, None, None, None, None, 1_000_000, None)
    assert st == 13 and "maximum" in ddf.ddf_status_string(st)
