"""Python binding of libddf.so, the GB300 DDF library (include/ddf.h).

Argument marshalling only: every step of inspection and execution runs in the
library's CUDA kernels.  There is no CPU fallback; when the library has not
been built, the first call raises ``DDFLibraryMissing``.  Build it with
``paper_2111_12243_gb300.build.build()``.

PyTorch provides device memory and streams: vectors passed to ``ddf_spmv``
and ``ddf_sptrsv`` are contiguous float64 CUDA tensors, and the default stream
argument is ``torch.cuda.current_stream()``.  CSR arrays given to
``ddf_inspect`` may be CUDA tensors, CPU tensors or numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libddf.so")

DDF_SPMV, DDF_SPTRSV = 1, 2
DDF_F64, DDF_F32, DDF_BF16 = 0, 1, 2
DDF_BLAS, DDF_PSC1, DDF_PSC2 = 0, 1, 2
DDF_ALLOW_BLAS, DDF_ALLOW_PSC1, DDF_ALLOW_PSC2, DDF_ALLOW_ALL = 1, 2, 4, 7
STATUS = {0: "DDF_OK", 1: "DDF_ERR_ARG", 2: "DDF_ERR_NOT_SQUARE", 3: "DDF_ERR_UNSORTED",
          4: "DDF_ERR_OUT_OF_RANGE", 5: "DDF_ERR_NOT_LOWER", 6: "DDF_ERR_MISSING_DIAG",
          7: "DDF_ERR_ZERO_DIAG", 8: "DDF_ERR_WRONG_KIND", 9: "DDF_ERR_OOM", 10: "DDF_ERR_CUDA",
          11: "DDF_ERR_TIMEOUT", 12: "DDF_ERR_NOT_CONVERGED", 13: "DDF_ERR_TOO_LARGE"}
RECORD_FIELDS = ("part", "type", "q0", "m", "n", "f_str", "rho", "g_str", "gamma", "h0", "delta",
                 "sigma")
#: every symbol include/ddf.h declares
EXPORTS = ("ddf_opts_default", "ddf_inspect", "ddf_update_values", "ddf_spmv", "ddf_sptrsv",
           "ddf_get_status", "ddf_plan_stats", "ddf_plan_export", "ddf_plan_destroy",
           "ddf_status_string", "ddf_last_launches", "ddf_kernel_launches",
           "ddf_debug_set_dependency", "ddf_sptrsv_csr_noalloc", "ddf_spmv_lowp", "ddf_sptrsv_refine",
           "ddf_inspect_batch", "ddf_spmm", "ddf_sptrsm", "ddf_batch_run", "ddf_tune", "ddf_tune_cost", "ddf_plan_save",
           "ddf_plan_load", "ddf_plan_validate", "ddf_debug_fail_alloc")
#: rows accepted by ddf_sptrsv_csr_noalloc (the size of its static scratch)
DDF_NOALLOC_MAX_ROWS = 1 << 20
DDF_COARSEN_MAX_ROWS = 16384
DDF_COARSEN_DEFAULT_ROWS = 0


class DDFLibraryMissing(ImportError):
    pass


class DDFError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS.get(self.status, self.status)} ({ddf_status_string(status)})")


class ddf_csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("on_device", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ddf_opts(ctypes.Structure):
    _fields_ = [("window_t", ctypes.c_int32), ("allowed_types", ctypes.c_int32),
                ("w_op", ctypes.c_int64), ("w_codelet", ctypes.c_int64), ("w_index", ctypes.c_int64),
                ("spin_cap_ns", ctypes.c_int64), ("unit_nnz", ctypes.c_int32),
                ("store_dtype", ctypes.c_int32), ("coarsen_rows", ctypes.c_int32),
                ("lower_of_input", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


class ddf_plan_stats_t(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("nnz", ctypes.c_int64), ("points", ctypes.c_int64),
                ("ncodelets", ctypes.c_int64 * 3), ("ops", ctypes.c_int64 * 3),
                ("rows", ctypes.c_int64 * 3), ("nunits", ctypes.c_int64),
                ("bytes_exec", ctypes.c_int64), ("max_row_len", ctypes.c_int64),
                ("levels", ctypes.c_int64), ("blocks", ctypes.c_int64), ("reserved", ctypes.c_int64 * 4)]


_lib = None


def lib():
    """The loaded libddf.so (raises DDFLibraryMissing when it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise DDFLibraryMissing(f"{LIB_PATH} is missing: build it with "
                                    "paper_2111_12243_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.ddf_opts_default.argtypes = [ctypes.POINTER(ddf_opts)]
        L.ddf_opts_default.restype = None
        L.ddf_inspect.argtypes = [ctypes.POINTER(ddf_csr), ctypes.c_int, ctypes.POINTER(ddf_opts), P,
                                  ctypes.POINTER(P)]
        L.ddf_update_values.argtypes = [P, P, I32, P]
        L.ddf_spmv.argtypes = [P, P, P, P]
        L.ddf_sptrsv.argtypes = [P, P, P, P]
        L.ddf_get_status.argtypes = [P, P]
        L.ddf_plan_stats.argtypes = [P, ctypes.POINTER(ddf_plan_stats_t)]
        L.ddf_plan_export.argtypes = [P, P, ctypes.POINTER(I64), P, P, ctypes.POINTER(I32), P]
        L.ddf_plan_destroy.argtypes = [P]
        L.ddf_plan_destroy.restype = None
        L.ddf_status_string.argtypes = [ctypes.c_int]
        L.ddf_status_string.restype = ctypes.c_char_p
        L.ddf_last_launches.argtypes = [P]
        L.ddf_last_launches.restype = I32
        L.ddf_kernel_launches.argtypes = []
        L.ddf_kernel_launches.restype = I64
        L.ddf_debug_set_dependency.argtypes = [P, I64, I32]
        L.ddf_spmv_lowp.argtypes = [P, P, P, ctypes.c_int, P]
        L.ddf_spmv_lowp.restype = ctypes.c_int
        L.ddf_sptrsv_refine.argtypes = [P, P, P, ctypes.c_double, I32, P, ctypes.POINTER(I32),
                                        ctypes.POINTER(ctypes.c_double)]
        L.ddf_sptrsv_refine.restype = ctypes.c_int
        L.ddf_inspect_batch.argtypes = [ctypes.POINTER(ddf_csr), I32, ctypes.c_int, ctypes.POINTER(ddf_opts), P,
                                        ctypes.POINTER(P)]
        L.ddf_inspect_batch.restype = ctypes.c_int
        L.ddf_spmm.argtypes = [P, P, P, I32, ctypes.c_int, P]
        L.ddf_spmm.restype = ctypes.c_int
        L.ddf_sptrsm.argtypes = [P, P, P, I32, ctypes.c_int, P]
        L.ddf_sptrsm.restype = ctypes.c_int
        L.ddf_batch_run.argtypes = [P, P, P, P, P, P, I32, ctypes.c_int, P]
        L.ddf_batch_run.restype = ctypes.c_int
        L.ddf_tune_cost.argtypes = [P, ctypes.c_int, P, P, ctypes.POINTER(I32)]
        L.ddf_tune_cost.restype = ctypes.c_int
        L.ddf_tune.argtypes = [P, P, P, I32, ctypes.c_int, P, ctypes.POINTER(I32)]
        L.ddf_tune.restype = ctypes.c_int
        L.ddf_plan_save.argtypes = [P, P, ctypes.POINTER(ctypes.c_size_t)]
        L.ddf_plan_save.restype = ctypes.c_int
        L.ddf_plan_load.argtypes = [P, ctypes.c_size_t, P, ctypes.POINTER(P)]
        L.ddf_plan_load.restype = ctypes.c_int
        L.ddf_sptrsv_csr_noalloc.argtypes = [I32, I64, P, P, P, P, P, I64, P]
        L.ddf_sptrsv_csr_noalloc.restype = ctypes.c_int
        for name in ("ddf_inspect", "ddf_update_values", "ddf_spmv", "ddf_sptrsv", "ddf_get_status",
                     "ddf_plan_stats", "ddf_plan_export", "ddf_debug_set_dependency"):
            getattr(L, name).restype = ctypes.c_int
        L.ddf_plan_validate.argtypes = [P]
        L.ddf_plan_validate.restype = ctypes.c_int
        L.ddf_debug_fail_alloc.argtypes = [I64]
        L.ddf_debug_fail_alloc.restype = ctypes.c_int
        _lib = L
    return _lib


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    import torch
    return ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))


def _check(st: int, where: str):
    if st != 0:
        raise DDFError(st, where)


def _ptr(a, dtype):
    """(pointer, on_device, keep-alive) of a tensor / ndarray with the given numpy dtype."""
    if a is None:
        return None, 0, None
    if hasattr(a, "is_cuda"):   # torch tensor
        import torch
        tdt = {np.int32: torch.int32, np.float64: torch.float64}[dtype]
        if a.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


def ddf_status_string(st: int) -> str:
    return lib().ddf_status_string(int(st)).decode()


def ddf_opts_default(**overrides) -> ddf_opts:
    o = ddf_opts()
    lib().ddf_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class Plan:
    """A device-resident DDF plan (owns its device memory)."""

    def __init__(self, handle, kind: int, n_rows: int, n_cols: int):
        self._h = handle
        self.kind = kind
        self.n_rows = n_rows
        self.n_cols = n_cols

    @property
    def handle(self):
        if not self._h:
            raise ValueError("plan has been destroyed")
        return self._h

    def destroy(self):
        if self._h:
            lib().ddf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def ddf_inspect(rowptr, colidx, values, n_cols: int, kind: int, opts: ddf_opts | None = None,
                stream=None) -> Plan:
    """Inspector (Alg. 1) on a CSR matrix; ``values`` may be None (pattern only)."""
    rp, dev_r, k1 = _ptr(rowptr, np.int32)
    ci, dev_c, k2 = _ptr(colidx, np.int32)
    va, dev_v, k3 = _ptr(values, np.float64)
    if len({dev_r, dev_c} | ({dev_v} if values is not None else set())) != 1:
        raise ValueError("rowptr, colidx and values must all be on the device or all on the host")
    n_rows = int(len(rowptr)) - 1
    nnz = int(len(colidx))
    A = ddf_csr(n_rows, int(n_cols), nnz, rp, ci, va, dev_r, 0)
    h = ctypes.c_void_p()
    st = lib().ddf_inspect(ctypes.byref(A), int(kind), ctypes.byref(opts) if opts is not None else None,
                           _stream(stream), ctypes.byref(h))
    _check(st, "ddf_inspect")
    return Plan(h, int(kind), n_rows, int(n_cols))


def ddf_update_values(plan: Plan, values, stream=None):
    va, dev, keep = _ptr(values, np.float64)
    _check(lib().ddf_update_values(plan.handle, va, dev, _stream(stream)), "ddf_update_values")
    del keep


def _dev_vec(t, n, name):
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    import torch
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be a contiguous float64 tensor with {n} entries")
    return ctypes.c_void_p(t.data_ptr())


def ddf_spmv(plan: Plan, x, y, stream=None):
    """y = A x on the device (asynchronous on the stream)."""
    _check(lib().ddf_spmv(plan.handle, _dev_vec(x, plan.n_cols, "x"), _dev_vec(y, plan.n_rows, "y"),
                          _stream(stream)), "ddf_spmv")


def ddf_sptrsv(plan: Plan, b, x, stream=None):
    """Solve L x = b on the device (asynchronous on the stream)."""
    _check(lib().ddf_sptrsv(plan.handle, _dev_vec(b, plan.n_rows, "b"), _dev_vec(x, plan.n_rows, "x"),
                            _stream(stream)), "ddf_sptrsv")


def _lp_vec(t, n, name):
    import torch
    if not (hasattr(t, "is_cuda") and t.is_cuda) or t.dtype not in (torch.float32, torch.bfloat16) \
            or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be a contiguous float32 or bfloat16 CUDA tensor with {n} entries")
    return ctypes.c_void_p(t.data_ptr()), (DDF_F32 if t.dtype == torch.float32 else DDF_BF16)


def ddf_spmv_lowp(plan: Plan, x, y, stream=None):
    """y = A x with FP32 / BF16 values and vectors, FP32 sums (plan store_dtype F32 or BF16)."""
    px, dx = _lp_vec(x, plan.n_cols, "x")
    py, dy = _lp_vec(y, plan.n_rows, "y")
    if dx != dy:
        raise ValueError("x and y must have the same dtype")
    _check(lib().ddf_spmv_lowp(plan.handle, px, py, dx, _stream(stream)), "ddf_spmv_lowp")


def ddf_sptrsv_refine(plan: Plan, b, x, tol: float = 1e-12, max_iter: int = 20, stream=None):
    """Solve L x = b by low-precision solves and FP64 refinement; returns (status, iters, relres)."""
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    st = lib().ddf_sptrsv_refine(plan.handle, _dev_vec(b, plan.n_rows, "b"), _dev_vec(x, plan.n_rows, "x"),
                                 float(tol), int(max_iter), _stream(stream), ctypes.byref(it), ctypes.byref(rr))
    return int(st), int(it.value), float(rr.value)


def ddf_inspect_batch(mats, kind: int, opts: ddf_opts | None = None, stream=None) -> Plan:
    """Inspect a list of (rowptr, colidx, values, n_cols) CSR tuples as one
    block-diagonal matrix (tensors on the device or host arrays)."""
    arr = (ddf_csr * len(mats))()
    keep = []
    n_rows = n_cols = 0
    for i, (rp, ci, va, nc) in enumerate(mats):
        prp, dr, k1 = _ptr(rp, np.int32)
        pci, dc, k2 = _ptr(ci, np.int32)
        pva, dv, k3 = _ptr(va, np.float64)
        keep += [k1, k2, k3]
        arr[i] = ddf_csr(int(len(rp)) - 1, int(nc), int(len(ci)), prp, pci, pva, dr, 0)
        n_rows += int(len(rp)) - 1
        n_cols += int(nc)
    h = ctypes.c_void_p()
    st = lib().ddf_inspect_batch(arr, len(mats), int(kind), ctypes.byref(opts) if opts is not None else None,
                                 _stream(stream), ctypes.byref(h))
    del keep
    _check(st, "ddf_inspect_batch")
    return Plan(h, int(kind), n_rows, n_cols)


def _mat(t, rows, nrhs, name):
    import torch
    if not (hasattr(t, "is_cuda") and t.is_cuda) or t.dtype not in (torch.float64, torch.float32) \
            or not t.is_contiguous() or t.numel() != rows * nrhs:
        raise ValueError(f"{name} must be a contiguous float64/float32 CUDA tensor of {rows} x {nrhs}")
    return ctypes.c_void_p(t.data_ptr()), (DDF_F64 if t.dtype == torch.float64 else DDF_F32)


def ddf_spmm(plan: Plan, X, Y, nrhs: int, stream=None):
    """Y = A X for nrhs right-hand sides (row-major [n][nrhs] CUDA tensors)."""
    px, dx = _mat(X, plan.n_cols, nrhs, "X")
    py, dy = _mat(Y, plan.n_rows, nrhs, "Y")
    if dx != dy:
        raise ValueError("X and Y must have the same dtype")
    _check(lib().ddf_spmm(plan.handle, px, py, int(nrhs), dx, _stream(stream)), "ddf_spmm")


def ddf_sptrsm(plan: Plan, B, X, nrhs: int, stream=None):
    """Solve L X = B for nrhs right-hand sides (row-major [n][nrhs] CUDA tensors)."""
    pb, db = _mat(B, plan.n_rows, nrhs, "B")
    px, dx = _mat(X, plan.n_rows, nrhs, "X")
    if db != dx:
        raise ValueError("B and X must have the same dtype")
    _check(lib().ddf_sptrsm(plan.handle, pb, px, int(nrhs), db, _stream(stream)), "ddf_sptrsm")


def ddf_batch_run(pa: Plan, X, Y, pl: Plan, B, Xs, nrhs: int, stream=None):
    """Y = A X on the SpMV plan pa and L Xs = B on the SpTRSV plan pl in one launch
    (row-major [n][nrhs] CUDA tensors of one dtype)."""
    px, dx = _mat(X, pa.n_cols, nrhs, "X")
    py, dy = _mat(Y, pa.n_rows, nrhs, "Y")
    pb, db = _mat(B, pl.n_rows, nrhs, "B")
    ps, ds = _mat(Xs, pl.n_rows, nrhs, "Xs")
    if len({dx, dy, db, ds}) != 1:
        raise ValueError("X, Y, B and Xs must have the same dtype")
    _check(lib().ddf_batch_run(pa.handle, px, py, pl.handle, pb, ps, int(nrhs), dx, _stream(stream)),
           "ddf_batch_run")


def ddf_tune(plan: Plan, inp, out, nrhs: int, stream=None) -> int:
    """Pick the multi-RHS tile size of a plan by timing candidates; returns it."""
    rows_in = plan.n_cols if plan.kind == DDF_SPMV else plan.n_rows
    pi, di = _mat(inp, rows_in, nrhs, "in")
    po, do = _mat(out, plan.n_rows, nrhs, "out")
    best = ctypes.c_int32(0)
    _check(lib().ddf_tune(plan.handle, pi, po, int(nrhs), di, _stream(stream), ctypes.byref(best)), "ddf_tune")
    return int(best.value)


def ddf_tune_cost(rowptr, colidx, values, n_cols: int, kind: int, opts: ddf_opts | None = None,
                  stream=None):
    """Pick Eq. 1's weights on the GPU by timing the executor of plans mined with
    candidate weight sets; returns (options with the chosen weights, its index)."""
    rp, dev_r, k1 = _ptr(rowptr, np.int32)
    ci, dev_c, k2 = _ptr(colidx, np.int32)
    va, dev_v, k3 = _ptr(values, np.float64)
    if values is None or len({dev_r, dev_c, dev_v}) != 1:
        raise ValueError("rowptr, colidx and values must be given, all on the device or all on the host")
    A = ddf_csr(int(len(rowptr)) - 1, int(n_cols), int(len(colidx)), rp, ci, va, dev_r, 0)
    o = ddf_opts()
    if opts is not None:
        ctypes.memmove(ctypes.byref(o), ctypes.byref(opts), ctypes.sizeof(o))
    else:
        lib().ddf_opts_default(ctypes.byref(o))
    pick = ctypes.c_int32(-1)
    _check(lib().ddf_tune_cost(ctypes.byref(A), int(kind), ctypes.byref(o), _stream(stream), ctypes.byref(pick)),
           "ddf_tune_cost")
    return o, int(pick.value)


def ddf_plan_save(plan: Plan) -> bytes:
    """Serialise a plan into bytes (reload it with ddf_plan_load)."""
    L = lib()
    n = ctypes.c_size_t(0)
    _check(L.ddf_plan_save(plan.handle, None, ctypes.byref(n)), "ddf_plan_save")
    buf = ctypes.create_string_buffer(n.value)
    _check(L.ddf_plan_save(plan.handle, buf, ctypes.byref(n)), "ddf_plan_save")
    return buf.raw[:n.value]


def ddf_plan_load(data: bytes, n_rows: int, n_cols: int, kind: int, stream=None) -> Plan:
    """Rebuild a device plan from ddf_plan_save's bytes, without re-inspection."""
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(lib().ddf_plan_load(buf, len(data), _stream(stream), ctypes.byref(h)), "ddf_plan_load")
    return Plan(h, int(kind), int(n_rows), int(n_cols))


def ddf_plan_validate(plan: Plan) -> int:
    """Bounds and dependency checks of a plan on the device; returns the status (0 = valid)."""
    return int(lib().ddf_plan_validate(plan.handle))


def ddf_get_status(plan: Plan, stream=None) -> int:
    """Synchronise, return and clear the plan's device status word."""
    return int(lib().ddf_get_status(plan.handle, _stream(stream)))


def ddf_plan_stats(plan: Plan) -> dict:
    s = ddf_plan_stats_t()
    _check(lib().ddf_plan_stats(plan.handle, ctypes.byref(s)), "ddf_plan_stats")
    return {"kind": s.kind, "n_rows": s.n_rows, "n_cols": s.n_cols, "depth": s.depth, "nnz": s.nnz,
            "points": s.points, "ncodelets": list(s.ncodelets), "ops": list(s.ops),
            "rows": list(s.rows), "nunits": s.nunits, "bytes_exec": s.bytes_exec,
            "max_row_len": s.max_row_len, "levels": s.levels, "blocks": s.blocks}


def ddf_plan_export(plan: Plan) -> dict:
    """Canonical plan: records (k, 12) int64, seq, part_ptr and gs (see ddf.h)."""
    L = lib()
    k = ctypes.c_int64(0)
    d = ctypes.c_int32(0)
    _check(L.ddf_plan_export(plan.handle, None, ctypes.byref(k), None, None, ctypes.byref(d), None),
           "ddf_plan_export")
    rec = np.zeros((k.value, 12), dtype=np.int64)
    seq = np.zeros(max(plan.n_rows, 1), dtype=np.int32)
    pp = np.zeros(d.value + 1, dtype=np.int32)
    gs = np.zeros(max(plan.n_rows, 1), dtype=np.int64)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(L.ddf_plan_export(plan.handle, P(rec), ctypes.byref(k), P(seq), P(pp), ctypes.byref(d), P(gs)),
           "ddf_plan_export")
    return {"records": rec, "seq": seq[:plan.n_rows], "part_ptr": pp, "gs": gs[:plan.n_rows]}


def ddf_plan_destroy(plan: Plan):
    plan.destroy()


def ddf_last_launches(plan: Plan) -> int:
    return int(lib().ddf_last_launches(plan.handle))


def ddf_kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().ddf_kernel_launches())


def ddf_debug_set_dependency(plan: Plan, k: int, col: int):
    _check(lib().ddf_debug_set_dependency(plan.handle, int(k), int(col)), "ddf_debug_set_dependency")


def ddf_debug_fail_alloc(k: int):
    """Make the library's device allocation after the next k fail with DDF_ERR_OOM (k < 0: off)."""
    lib().ddf_debug_fail_alloc(int(k))


def ddf_sptrsv_csr_noalloc(rowptr, colidx, values, b, x, spin_cap_ns: int = 2_000_000_000,
                           stream=None) -> int:
    """Solve L x = b on CUDA tensors without any device allocation (no plan).

    Returns the status code (0 on success); synchronises the stream.
    """
    import torch
    for t, name, dt in ((rowptr, "rowptr", torch.int32), (colidx, "colidx", torch.int32),
                        (values, "values", torch.float64), (b, "b", torch.float64),
                        (x, "x", torch.float64)):
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous CUDA {dt} tensor")
    n = int(rowptr.numel()) - 1
    return int(lib().ddf_sptrsv_csr_noalloc(n, int(colidx.numel()), ctypes.c_void_p(rowptr.data_ptr()),
                                            ctypes.c_void_p(colidx.data_ptr()),
                                            ctypes.c_void_p(values.data_ptr()),
                                            ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                            int(spin_cap_ns), _stream(stream)))
