"""SpMV executor layouts on the GPU against the CPU oracle.

Runs of BLAS / PSC I codelets with short rows are executed one lane per row,
their values stored point-major in tiles of 8 rows.  These tests cover the
shapes that exercise that layout: runs whose length is not a multiple of the
tile (ragged last tiles), tiles that span several small codelets (3-row
elasticity codelets), rows longer than the tile limit (which stay on the
work-unit path), empty rows, PSC II rows from one point to thousands (staged
products, one warp per row, one CTA per row), values supplied after inspection, low-precision
copies, the multi-RHS executor, plan save / load and validation.  Results must
match the oracle's CSR-order definitions within 1e-12 (FP64), exactly where
every partial sum is an integer.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(y, ref):
    nr = np.linalg.norm(ref)
    d = np.linalg.norm(np.asarray(y, dtype=np.float64) - ref)
    return d / nr if nr > 0 else d


def spmv(plan, x, n_rows):
    y = torch.full((n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    ddf.ddf_spmv(plan, dev(x), y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def with_long_rows(n=600, long_len=300, seed=4):
    """A band matrix whose every 50th row is replaced by a dense row of
    long_len columns (longer than a tile row may be), some of them adjacent,
    and a few empty rows: tiled runs broken by untiled BLAS rows."""
    b = synth.banded(n, 3, seed)
    rows = [list(b.colidx[b.rowptr[i]:b.rowptr[i + 1]]) for i in range(n)]
    for i in range(0, n, 50):
        rows[i] = list(range(long_len))
        if i + 1 < n:
            rows[i + 1] = list(range(long_len))
    for i in (7, 8, 9, 333):
        rows[i] = []
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in r], np.int32)
    v = np.random.default_rng(seed).standard_normal(ci.size)
    return synth.CSR(n, n, rp.astype(np.int32), ci, v)


def long_psc2_rows(n=6000, seed=8):
    """Irregular rows (PSC II) of lengths 1 .. 5000: a few longer than 1024
    points (one CTA per row), some between 256 and 1024 (one warp), the rest
    short (staged products), and empty rows."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, 12, n)
    lens[rng.choice(n, 12, replace=False)] = rng.integers(1025, 5000, 12)
    lens[rng.choice(n, 20, replace=False)] = rng.integers(257, 1024, 20)
    lens[rng.choice(n, 30, replace=False)] = 0
    rows = [np.sort(rng.choice(n, int(k), replace=False)) for k in lens]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    ci = np.concatenate(rows).astype(np.int32)
    return synth.CSR(n, n, rp.astype(np.int32), ci, rng.standard_normal(ci.size))


CASES = {
    "band_1000": lambda: synth.banded(1000, 4),
    "band_29": lambda: synth.banded(29, 2),
    "lap7_11": lambda: synth.laplacian_7pt(11),
    "st27_10": lambda: synth.stencil_27pt(10),
    "st27_13": lambda: synth.stencil_27pt(13),
    "elast_6": lambda: synth.elasticity_blocks(6),
    "st27r_9": lambda: synth.workload("st27r_168", 9 / 168)[0],
    "long_rows": with_long_rows,
    "random_500": lambda: synth.random_pattern(500, 450, 0.02, 3, empty_rows=0.2),
    "powerlaw_3000": lambda: synth.powerlaw(3000),
    "long_psc2": long_psc2_rows,
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("on_device", [True, False])
def test_tiled_spmv_matches_oracle(name, on_device):
    a = CASES[name]()
    x = synth.uniform_vector(a.n_cols, 31)
    if on_device:
        p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV)
    else:
        p = ddf.ddf_inspect(a.rowptr, a.colidx, a.values, a.n_cols, ddf.DDF_SPMV)
    assert ddf.ddf_plan_validate(p) == 0
    y = spmv(p, x, a.n_rows)
    assert relerr(y, oracle.spmv(a, x)) <= TOL
    # twice in a row: the executor keeps no state between calls
    assert np.array_equal(spmv(p, x, a.n_rows), y)


@pytest.mark.parametrize("name", ["st27_13", "lap7_11", "band_1000"])
def test_integer_values_are_exact(name):
    a = CASES[name]()
    if name == "band_1000":
        a.values = np.round(a.values * 4)
    xi = np.random.default_rng(5).integers(-20, 20, a.n_cols).astype(np.float64)
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV)
    assert np.array_equal(spmv(p, xi, a.n_rows), oracle.spmv(a, xi))


def test_values_after_inspection_and_updates():
    a = CASES["elast_6"]()
    x = synth.uniform_vector(a.n_cols, 8)
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), None, a.n_cols, ddf.DDF_SPMV)
    for k, on_dev in ((0, True), (1, False), (2, True)):
        v = np.random.default_rng(k).standard_normal(a.nnz)
        ddf.ddf_update_values(p, dev(v) if on_dev else v)
        b = synth.CSR(a.n_rows, a.n_cols, a.rowptr, a.colidx, v)
        assert relerr(spmv(p, x, a.n_rows), oracle.spmv(b, x)) <= TOL


@pytest.mark.parametrize("dtype,tol", [(ddf.DDF_F32, 2e-6), (ddf.DDF_BF16, 2e-2)])
@pytest.mark.parametrize("name", ["st27_13", "long_rows", "elast_6", "long_psc2"])
def test_low_precision_tiles(dtype, tol, name):
    a = CASES[name]()
    x = synth.uniform_vector(a.n_cols, 9)
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV,
                        ddf.ddf_opts_default(store_dtype=dtype))
    tdt = torch.float32 if dtype == ddf.DDF_F32 else torch.bfloat16
    xl = dev(x).to(tdt)
    yl = torch.empty(a.n_rows, dtype=tdt, device="cuda")
    ddf.ddf_spmv_lowp(p, xl, yl)
    torch.cuda.synchronize()
    # the reference rounds values and x to the storage type, then sums in FP64
    vr = torch.from_numpy(a.values).to(tdt).double().numpy()
    xr = xl.double().cpu().numpy()
    ref = oracle.spmv(synth.CSR(a.n_rows, a.n_cols, a.rowptr, a.colidx, vr), xr)
    assert relerr(yl.double().cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("nrhs", [5, 8])
@pytest.mark.parametrize("name", ["st27_10", "long_rows", "elast_6", "long_psc2"])
def test_multi_rhs_on_tiled_plan(name, nrhs):
    a = CASES[name]()
    X = np.stack([synth.uniform_vector(a.n_cols, 40 + k) for k in range(nrhs)], axis=1)
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV)
    Y = torch.empty((a.n_rows, nrhs), dtype=torch.float64, device="cuda")
    ddf.ddf_spmm(p, dev(X), Y, nrhs)
    Yh = Y.cpu().numpy()
    for k in range(nrhs):
        assert relerr(Yh[:, k], oracle.spmv(a, X[:, k].copy())) <= TOL


def test_save_load_keeps_tiles():
    a = CASES["st27_13"]()
    x = synth.uniform_vector(a.n_cols, 12)
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV)
    y0 = spmv(p, x, a.n_rows)
    buf = ddf.ddf_plan_save(p)
    q = ddf.ddf_plan_load(buf, a.n_rows, a.n_cols, ddf.DDF_SPMV)
    assert np.array_equal(spmv(q, x, a.n_rows), y0)
    assert ddf.ddf_plan_stats(q)["nunits"] == ddf.ddf_plan_stats(p)["nunits"]


def test_tiles_do_not_change_the_canonical_plan():
    # the tiles are an executor layout: the exported plan (Alg. 1's codelets,
    # CSR value offsets) is the oracle's, bit for bit
    for name in ("st27_10", "elast_6", "long_rows"):
        a = CASES[name]()
        p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV)
        got = ddf.ddf_plan_export(p)
        ref = oracle.inspect(a, oracle.SPMV, weights=(8, 32, 4))
        assert np.array_equal(got["records"], ref.records)
        assert np.array_equal(got["gs"], ref.gs)


def test_long_psc2_rows_are_deterministic():
    a = long_psc2_rows(5500, 9)
    x = synth.uniform_vector(a.n_cols, 13)
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV)
    st = ddf.ddf_plan_stats(p)
    assert st["max_row_len"] > 1024
    y0 = spmv(p, x, a.n_rows)
    for _ in range(3):
        assert np.array_equal(spmv(p, x, a.n_rows).view(np.uint64), y0.view(np.uint64))
    assert relerr(y0, oracle.spmv(a, x)) <= TOL
    q = ddf.ddf_plan_load(ddf.ddf_plan_save(p), a.n_rows, a.n_cols, ddf.DDF_SPMV)
    assert np.array_equal(spmv(q, x, a.n_rows).view(np.uint64), y0.view(np.uint64))
