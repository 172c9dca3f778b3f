"""Allocation failures injected on the host (ddf_debug_fail_alloc): every
device allocation an entry point makes is failed in turn, and each attempt
must return DDF_ERR_OOM after releasing what it had allocated, with no GPU
fault.  The attempt that finally succeeds must give the same result as a
call made without the hook, bit for bit (the executors are deterministic),
so the earlier failures left nothing behind that changes a later call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_12243_gb300 as ddf
import synth

pytestmark = pytest.mark.gpu

OOM = 9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_12243_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    ddf.ddf_debug_fail_alloc(-1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


A = synth.laplacian_7pt(10)
LO = synth.lower_triangle(A)
X = synth.uniform_vector(A.n_cols, 1)
B = synth.uniform_vector(A.n_rows, 2)


def spmv():
    p = ddf.ddf_inspect(dev(A.rowptr), dev(A.colidx), dev(A.values), A.n_cols, ddf.DDF_SPMV)
    try:
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        ddf.ddf_spmv(p, dev(X), y)
        return y.cpu()
    finally:
        p.destroy()


def sptrsv(**opts):
    q = ddf.ddf_inspect(dev(LO.rowptr), dev(LO.colidx), dev(LO.values), LO.n_cols, ddf.DDF_SPTRSV,
                        ddf.ddf_opts_default(**opts))
    try:
        x = torch.empty(LO.n_rows, dtype=torch.float64, device="cuda")
        ddf.ddf_sptrsv(q, dev(B), x)
        assert ddf.ddf_get_status(q) == 0
        return x.cpu()
    finally:
        q.destroy()


def refine():
    q = ddf.ddf_inspect(LO.rowptr, LO.colidx, LO.values, LO.n_cols, ddf.DDF_SPTRSV,
                        ddf.ddf_opts_default(store_dtype=ddf.DDF_F32))
    try:
        x = torch.empty(LO.n_rows, dtype=torch.float64, device="cuda")
        st = ddf.ddf_sptrsv_refine(q, dev(B), x)
        assert st[0] == 0
        return x.cpu()
    finally:
        q.destroy()


def batch():
    mats = [synth.lower_triangle(synth.batch_member(n, k, 60 + i))
            for i, (n, k) in enumerate([(500, "2d"), (800, "3d"), (600, "powerlaw")])]
    p = ddf.ddf_inspect_batch([(dev(m.rowptr), dev(m.colidx), dev(m.values), m.n_cols) for m in mats],
                              ddf.DDF_SPTRSV)
    try:
        n = sum(m.n_rows for m in mats)
        Bm = dev(np.linspace(-1, 1, 4 * n).reshape(n, 4))
        Xm = torch.empty_like(Bm)
        ddf.ddf_sptrsm(p, Bm, Xm, 4)
        assert ddf.ddf_get_status(p) == 0
        return Xm.cpu()
    finally:
        p.destroy()


_SAVED = {}


def load():
    if "buf" not in _SAVED:
        q = ddf.ddf_inspect(dev(LO.rowptr), dev(LO.colidx), dev(LO.values), LO.n_cols, ddf.DDF_SPTRSV,
                            ddf.ddf_opts_default(coarsen_rows=128))
        _SAVED["buf"] = ddf.ddf_plan_save(q)
        q.destroy()
    q = ddf.ddf_plan_load(_SAVED["buf"], LO.n_rows, LO.n_cols, ddf.DDF_SPTRSV)
    try:
        x = torch.empty(LO.n_rows, dtype=torch.float64, device="cuda")
        ddf.ddf_sptrsv(q, dev(B), x)
        assert ddf.ddf_get_status(q) == 0
        return x.cpu()
    finally:
        q.destroy()


CASES = {
    "spmv": spmv,
    "sptrsv": sptrsv,
    "sptrsv_coarsened": lambda: sptrsv(coarsen_rows=128),
    "refine_f32": refine,
    "batch_sptrsm": batch,
    "plan_load": load,
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_each_allocation_failure_is_reported_and_released(name):
    call = CASES[name]
    ddf.ddf_debug_fail_alloc(-1)
    ref = call()
    failures = 0
    for k in range(400):
        ddf.ddf_debug_fail_alloc(k)
        try:
            got = call()
        except ddf.DDFError as e:
            assert e.status == OOM, (k, e.status)
            failures += 1
            continue
        ddf.ddf_debug_fail_alloc(-1)
        break
    else:
        pytest.fail("the call never succeeded")
    assert failures >= 2          # the call allocates, and every failure was reported
    assert torch.equal(got, ref)
