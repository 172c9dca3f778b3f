"""Host-side checks of the C ABI library (no GPU compute).

The library is built for sm_103a with nvcc (cross-compiles without a GPU),
loaded through ctypes, and must export every function include/ddf.h declares.
"""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2111_12243_gb300 as ddf
from paper_2111_12243_gb300 import build as ddf_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ddf.h")


@pytest.fixture(scope="module")
def libpath():
    return ddf_build.build()


def header_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^DDF_API\s+[\w\s\*]*?\b(ddf_\w+)\s*\(", text, re.M)))


def test_header_declares_the_exports():
    assert header_functions() == sorted(ddf.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (ddf_\w+)$", out, re.M))
    assert set(header_functions()) <= exported
    # nothing else leaks out of the library under the ddf_ prefix
    assert exported == set(header_functions())


def test_library_loads_and_host_calls(libpath):
    L = ddf.lib()
    for name in ddf.EXPORTS:
        assert hasattr(L, name)
    o = ddf.ddf_opts_default()
    assert (o.window_t, o.allowed_types, o.w_op, o.w_codelet, o.w_index, o.unit_nnz, o.coarsen_rows) == (
        256, 7, 8, 32, 4, 256, ddf.DDF_COARSEN_DEFAULT_ROWS)
    import oracle
    assert oracle.DEFAULT_COARSEN == ddf.DDF_COARSEN_DEFAULT_ROWS
    assert ddf.ddf_status_string(0) == "ok"
    assert "timed out" in ddf.ddf_status_string(11)
    assert ddf.ddf_status_string(999) == "unknown status"


def test_header_constants_match_binding():
    import re
    text = open(HEADER).read()
    for name in ("DDF_COARSEN_MAX_ROWS", "DDF_COARSEN_DEFAULT_ROWS"):
        m = re.search(r"#define %s (\d+)" % name, text)
        assert m and int(m.group(1)) == getattr(ddf, name)


def test_ctypes_layouts_match_header():
    # ddf_csr: 2 x int32, int64, 3 pointers, 2 x int32
    assert ctypes.sizeof(ddf.ddf_csr) == 4 + 4 + 8 + 3 * 8 + 4 + 4
    assert ctypes.sizeof(ddf.ddf_opts) == 2 * 4 + 4 * 8 + 4 + 9 * 4
    assert ctypes.sizeof(ddf.ddf_plan_stats_t) == 4 * 4 + 8 * (2 + 9 + 3 + 6)


def test_host_argument_errors_without_gpu(libpath):
    # NULL output handle and bad kinds fail before any CUDA call
    L = ddf.lib()
    A = ddf.ddf_csr()
    assert L.ddf_inspect(ctypes.byref(A), 1, None, None, None) == 1
    h = ctypes.c_void_p()
    assert L.ddf_inspect(ctypes.byref(A), 3, None, None, ctypes.byref(h)) == 1
    A.n_rows, A.n_cols = 3, 4
    A.rowptr = ctypes.c_void_p(1)
    assert L.ddf_inspect(ctypes.byref(A), 2, None, None, ctypes.byref(h)) == 2   # not square
    o = ddf.ddf_opts_default(window_t=0)
    assert L.ddf_inspect(ctypes.byref(A), 1, ctypes.byref(o), None, ctypes.byref(h)) == 1
    o = ddf.ddf_opts_default(allowed_types=ddf.DDF_ALLOW_BLAS)
    assert L.ddf_inspect(ctypes.byref(A), 1, ctypes.byref(o), None, ctypes.byref(h)) == 1
    for bad in (-1, ddf.DDF_COARSEN_MAX_ROWS + 1):
        o = ddf.ddf_opts_default(coarsen_rows=bad)
        assert L.ddf_inspect(ctypes.byref(A), 1, ctypes.byref(o), None, ctypes.byref(h)) == 1
    assert L.ddf_spmv(None, None, None, None) == 1
    assert L.ddf_sptrsv(None, None, None, None) == 1
    assert L.ddf_last_launches(None) == 0


def test_every_entry_point_rejects_missing_handles_without_gpu(libpath):
    # Argument checks come before any CUDA call, so they run here without a GPU
    L = ddf.lib()
    ARG, TOO_LARGE = 1, 13
    sz = ctypes.c_size_t(0)
    i32 = ctypes.c_int32(0)
    i64 = ctypes.c_int64(0)
    h = ctypes.c_void_p()
    assert L.ddf_update_values(None, None, 1, None) == ARG
    assert L.ddf_get_status(None, None) == ARG
    assert L.ddf_plan_stats(None, None) == ARG
    assert L.ddf_plan_export(None, None, ctypes.byref(i64), None, None, ctypes.byref(i32), None) == ARG
    assert L.ddf_debug_set_dependency(None, 0, 0) == ARG
    assert L.ddf_spmv_lowp(None, None, None, 1, None) == ARG
    assert L.ddf_sptrsv_refine(None, None, None, 1e-12, 10, None, None, None) == ARG
    assert L.ddf_plan_validate(None) == ARG
    assert L.ddf_plan_save(None, None, ctypes.byref(sz)) == ARG
    # loading: no buffer, a buffer too short for the header, a wrong magic, no output handle
    assert L.ddf_plan_load(None, 0, None, ctypes.byref(h)) == ARG
    junk = ctypes.create_string_buffer(b"x" * 4096)
    assert L.ddf_plan_load(junk, 8, None, ctypes.byref(h)) == ARG
    assert L.ddf_plan_load(junk, 4096, None, ctypes.byref(h)) == ARG
    assert L.ddf_plan_load(junk, 4096, None, None) == ARG
    # batches and several right-hand sides
    A = ddf.ddf_csr()
    assert L.ddf_inspect_batch(None, 2, 1, None, None, ctypes.byref(h)) == ARG
    assert L.ddf_inspect_batch(ctypes.byref(A), 0, 1, None, None, ctypes.byref(h)) == ARG
    assert L.ddf_inspect_batch(ctypes.byref(A), 1, 3, None, None, ctypes.byref(h)) == ARG
    assert L.ddf_inspect_batch(ctypes.byref(A), 1, 1, None, None, None) == ARG
    assert L.ddf_spmm(None, None, None, 32, 1, None) == ARG
    assert L.ddf_sptrsm(None, None, None, 32, 1, None) == ARG
    assert L.ddf_batch_run(None, None, None, None, None, None, 32, 1, None) == ARG
    assert L.ddf_tune(None, None, None, 32, 1, None, ctypes.byref(i32)) == ARG
    o = ddf.ddf_opts_default()
    assert L.ddf_tune_cost(None, 1, ctypes.byref(o), None, ctypes.byref(i32)) == ARG
    assert L.ddf_tune_cost(ctypes.byref(A), 1, ctypes.byref(o), None, ctypes.byref(i32)) == ARG   # no values
    assert L.ddf_tune_cost(ctypes.byref(A), 3, ctypes.byref(o), None, ctypes.byref(i32)) == ARG
    # the allocation-free solve: bad sizes and limits, then a size beyond its scratch
    assert L.ddf_sptrsv_csr_noalloc(-1, 0, None, None, None, None, None, 1000, None) == ARG
    assert L.ddf_sptrsv_csr_noalloc(4, 4, None, None, None, None, None, 0, None) == ARG
    assert L.ddf_sptrsv_csr_noalloc((1 << 20) + 1, 0, None, None, None, None, None, 1000, None) == TOO_LARGE
