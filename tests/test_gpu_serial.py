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
