"""The allocation-free solve, checked against the plan-based solve.

ddf_sptrsv_csr_noalloc serves callers that must not allocate device memory
(for example code running inside an allocator hook, or under a fixed memory
budget): it keeps its scratch in a static device array instead of calling
cudaMalloc.  It is called here through the C ABI, twice in a row on the same
inputs (the second call reuses the scratch the first one left behind), and
each result must match ddf_sptrsv on a plan within the tolerance the other
GPU tests use.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_12243_gb300 as ddf
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_12243_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def relerr(y, ref):
    return float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref))


@pytest.mark.parametrize("name", ["lap7_24", "powerlaw_20000"])
def test_noalloc_matches_plan_solve_twice(name):
    a = synth.laplacian_7pt(24) if name == "lap7_24" else synth.powerlaw(20000)
    lo = synth.lower_triangle(a, "keep" if name == "lap7_24" else "unit_dominant")
    dev = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()  # noqa: E731
    rp, ci, va = dev(lo.rowptr), dev(lo.colidx), dev(lo.values)
    b = dev(synth.uniform_vector(lo.n_rows, 3))
    plan = ddf.ddf_inspect(rp, ci, va, lo.n_cols, ddf.DDF_SPTRSV)
    ref = torch.empty(lo.n_rows, dtype=torch.float64, device="cuda")
    ddf.ddf_sptrsv(plan, b, ref)
    assert ddf.ddf_get_status(plan) == 0
    L = ddf.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        x = torch.full((lo.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        st = L.ddf_sptrsv_csr_noalloc(lo.n_rows, lo.nnz, ctypes.c_void_p(rp.data_ptr()),
                                      ctypes.c_void_p(ci.data_ptr()), ctypes.c_void_p(va.data_ptr()),
                                      ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                      2_000_000_000, stream)
        assert st == 0, ddf.ddf_status_string(st)
        assert relerr(x, ref) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = ddf.lib()
    n = ddf.DDF_NOALLOC_MAX_ROWS + 1
    st = L.ddf_sptrsv_csr_noalloc(n, 0, None, None, None, None, None, 1_000_000, None)
    assert st == 13 and "maximum" in ddf.ddf_status_string(st)
