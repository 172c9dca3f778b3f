"""Plan serialisation round trips on the GPU: a reloaded plan exports the same
canonical plan and gives bit-identical results; corrupted or truncated
buffers are rejected."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_12243_gb300 as ddf
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_12243_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def same_export(p, q):
    a, b = ddf.ddf_plan_export(p), ddf.ddf_plan_export(q)
    return all(np.array_equal(a[k], b[k]) for k in ("records", "seq", "part_ptr", "gs"))


@pytest.mark.parametrize("store", [ddf.DDF_F64, ddf.DDF_F32])
def test_round_trip(store):
    a = synth.elasticity_blocks(5)
    lo = synth.lower_triangle(a)
    o = ddf.ddf_opts_default(store_dtype=store)
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV, o)
    q = ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), dev(lo.values), lo.n_cols, ddf.DDF_SPTRSV, o)
    p2 = ddf.ddf_plan_load(ddf.ddf_plan_save(p), a.n_rows, a.n_cols, ddf.DDF_SPMV)
    q2 = ddf.ddf_plan_load(ddf.ddf_plan_save(q), lo.n_rows, lo.n_cols, ddf.DDF_SPTRSV)
    assert same_export(p, p2) and same_export(q, q2)
    assert ddf.ddf_plan_stats(p)["bytes_exec"] == ddf.ddf_plan_stats(p2)["bytes_exec"]
    x = dev(synth.uniform_vector(a.n_cols, 1))
    y1 = torch.empty(a.n_rows, dtype=torch.float64, device="cuda")
    y2 = torch.empty_like(y1)
    ddf.ddf_spmv(p, x, y1)
    ddf.ddf_spmv(p2, x, y2)
    assert torch.equal(y1, y2)
    b = dev(synth.uniform_vector(lo.n_rows, 2))
    x1 = torch.empty(lo.n_rows, dtype=torch.float64, device="cuda")
    x2 = torch.empty_like(x1)
    ddf.ddf_sptrsv(q, b, x1)
    ddf.ddf_sptrsv(q2, b, x2)
    assert ddf.ddf_get_status(q2) == 0 and torch.equal(x1, x2)
    if store == ddf.DDF_F32:
        st1 = ddf.ddf_sptrsv_refine(q, b, x1)
        st2 = ddf.ddf_sptrsv_refine(q2, b, x2)
        assert st1[0] == 0 and st2[0] == 0 and torch.equal(x1, x2)


def test_rejects_damaged_buffers():
    a = synth.laplacian_7pt(8)
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV)
    data = bytearray(ddf.ddf_plan_save(p))
    for pos in (len(data) // 2, len(data) - 20):
        bad = bytearray(data)
        bad[pos] ^= 0x55
        with pytest.raises(ddf.DDFError) as e:
            ddf.ddf_plan_load(bytes(bad), a.n_rows, a.n_cols, ddf.DDF_SPMV)
        assert e.value.status == 1
    with pytest.raises(ddf.DDFError):
        ddf.ddf_plan_load(bytes(data[:len(data) // 3]), a.n_rows, a.n_cols, ddf.DDF_SPMV)
    bad = bytearray(data)
    bad[0:8] = b"NOTAPLAN"
    with pytest.raises(ddf.DDFError):
        ddf.ddf_plan_load(bytes(bad), a.n_rows, a.n_cols, ddf.DDF_SPMV)


def test_round_trip_coarsened_and_batched():
    # a coarsened plan carries its block and chunk tables in the buffer
    lo = synth.lower_triangle(synth.laplacian_7pt(12))
    o = ddf.ddf_opts_default(coarsen_rows=200)
    q = ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), dev(lo.values), lo.n_cols, ddf.DDF_SPTRSV, o)
    q2 = ddf.ddf_plan_load(ddf.ddf_plan_save(q), lo.n_rows, lo.n_cols, ddf.DDF_SPTRSV)
    assert same_export(q, q2)
    st, st2 = ddf.ddf_plan_stats(q), ddf.ddf_plan_stats(q2)
    assert (st2["blocks"], st2["levels"], st2["depth"]) == (st["blocks"], st["levels"], st["depth"])
    b = dev(synth.uniform_vector(lo.n_rows, 3))
    x1 = torch.empty(lo.n_rows, dtype=torch.float64, device="cuda")
    x2 = torch.empty_like(x1)
    ddf.ddf_sptrsv(q, b, x1)
    ddf.ddf_sptrsv(q2, b, x2)
    assert ddf.ddf_get_status(q2) == 0 and torch.equal(x1, x2)
    # a batched plan solves several right-hand sides after reloading
    mats = [synth.batch_member(n, k, 7 + i) for i, (n, k) in enumerate([(900, "2d"), (1300, "3d"), (1100, "powerlaw")])]
    lows = [synth.lower_triangle(m) for m in mats]
    o32 = ddf.ddf_opts_default(store_dtype=ddf.DDF_F32)
    p = ddf.ddf_inspect_batch([(dev(m.rowptr), dev(m.colidx), dev(m.values), m.n_cols) for m in lows],
                              ddf.DDF_SPTRSV, o32)
    n = sum(m.n_rows for m in lows)
    p2 = ddf.ddf_plan_load(ddf.ddf_plan_save(p), n, n, ddf.DDF_SPTRSV)
    assert same_export(p, p2)
    B = torch.rand((n, 4), dtype=torch.float32, device="cuda")
    X1 = torch.empty_like(B)
    X2 = torch.empty_like(B)
    ddf.ddf_sptrsm(p, B, X1, 4)
    ddf.ddf_sptrsm(p2, B, X2, 4)
    assert ddf.ddf_get_status(p2) == 0 and torch.equal(X1, X2)


def test_size_query_and_short_buffer():
    a = synth.laplacian_5pt(10)
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV)
    import ctypes
    L = ddf.lib()
    need = ctypes.c_size_t(0)
    assert L.ddf_plan_save(p.handle, None, ctypes.byref(need)) == 0 and need.value > 0
    short = ctypes.c_size_t(need.value - 1)
    buf = ctypes.create_string_buffer(need.value)
    assert L.ddf_plan_save(p.handle, buf, ctypes.byref(short)) == 1     # too small
    assert short.value == need.value                                      # reports the size
