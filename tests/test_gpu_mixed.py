"""GPU checks of the mixed-precision forms against the FP64 oracle.

* ddf_spmv_lowp: values and vectors stored in FP32 or BF16, FP32 sums.  The
  result is compared with the oracle run on the same rounded inputs, so the
  only difference left is FP32 accumulation: |y - y_ref| <= 2 k u32 |A||x| per
  row (k = row length).  Integer stencils with small integer x are exact.
* ddf_sptrsv_refine: FP32 / BF16 solves with FP64 residual and update must
  reach a relative residual <= 1e-12, computed by the oracle in FP64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2111_12243_gb300 as ddf
import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_12243_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def round_bf16(a):
    """Round float64 values to bfloat16 (nearest, ties to even) and back."""
    f = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bias = ((f >> 16) & 1) + 0x7FFF
    r = ((f + bias) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def rounded(a, dt):
    return round_bf16(a) if dt == ddf.DDF_BF16 else np.asarray(a, np.float32).astype(np.float64)


MATS = {
    "lap7_16": lambda: synth.laplacian_7pt(16),
    "elast_6": lambda: synth.elasticity_blocks(6),
    "st27_10": lambda: synth.stencil_27pt(10),
    "powerlaw_20000": lambda: synth.powerlaw(20000),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("vdt", [ddf.DDF_F32, ddf.DDF_BF16])
@pytest.mark.parametrize("xdt", [ddf.DDF_F32, ddf.DDF_BF16])
def test_spmv_lowp_accumulation_bound(name, vdt, xdt):
    a = MATS[name]()
    x = synth.uniform_vector(a.n_cols, 5)
    av = rounded(a.values, vdt)
    xv = rounded(x, xdt)
    ar = synth.CSR(a.n_rows, a.n_cols, a.rowptr, a.colidx, av)
    ref = oracle.spmv(ar, xv)
    absref = oracle.spmv(synth.CSR(a.n_rows, a.n_cols, a.rowptr, a.colidx, np.abs(av)), np.abs(xv))
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV,
                        ddf.ddf_opts_default(store_dtype=vdt))
    tdt = torch.float32 if xdt == ddf.DDF_F32 else torch.bfloat16
    xt = dev(xv).to(tdt)
    y = torch.empty(a.n_rows, dtype=tdt, device="cuda")
    ddf.ddf_spmv_lowp(p, xt, y)
    got = y.double().cpu().numpy()
    k = np.maximum(np.diff(a.rowptr), 1)
    bound = 2 * k * U32 * absref + 1e-30
    if xdt == ddf.DDF_BF16:
        # the result itself is stored in BF16: one more rounding of |y|
        bound = bound + 2.0 ** -8 * np.abs(ref)
    assert np.all(np.abs(got - ref) <= bound)


def test_spmv_lowp_integer_exact():
    a = synth.laplacian_7pt(20)
    xi = np.random.default_rng(4).integers(-40, 40, a.n_cols).astype(float)
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV,
                        ddf.ddf_opts_default(store_dtype=ddf.DDF_BF16))
    y = torch.empty(a.n_rows, dtype=torch.float32, device="cuda")
    ddf.ddf_spmv_lowp(p, dev(xi).float(), y)
    assert np.array_equal(y.double().cpu().numpy(), oracle.spmv(a, xi))


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("vdt", [ddf.DDF_F32, ddf.DDF_BF16])
def test_refinement_reaches_1e12(name, vdt):
    a = MATS[name]()
    lo = synth.lower_triangle(a, "unit_dominant" if name.startswith("power") else "keep")
    b = synth.uniform_vector(lo.n_rows, 6)
    q = ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), dev(lo.values), lo.n_cols, ddf.DDF_SPTRSV,
                        ddf.ddf_opts_default(store_dtype=vdt))
    x = torch.zeros(lo.n_rows, dtype=torch.float64, device="cuda")
    st, iters, rel = ddf.ddf_sptrsv_refine(q, dev(b), x, tol=1e-12, max_iter=30)
    assert st == 0, (ddf.ddf_status_string(st), iters, rel)
    xs = x.cpu().numpy()
    r = b - oracle.spmv(lo, xs)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)
    assert rel <= 1e-12 and iters <= (6 if vdt == ddf.DDF_F32 else 20)
    ref = oracle.sptrsv(lo, b)
    assert np.linalg.norm(xs - ref) <= 1e-10 * np.linalg.norm(ref)
    # the FP64 solve of the same plan still works
    x2 = torch.empty(lo.n_rows, dtype=torch.float64, device="cuda")
    ddf.ddf_sptrsv(q, dev(b), x2)
    assert ddf.ddf_get_status(q) == 0
    assert np.linalg.norm(x2.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)


def test_refinement_not_converged_and_kind_checks():
    lo = synth.lower_triangle(synth.laplacian_7pt(10))
    b = dev(synth.uniform_vector(lo.n_rows, 1))
    q = ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), dev(lo.values), lo.n_cols, ddf.DDF_SPTRSV,
                        ddf.ddf_opts_default(store_dtype=ddf.DDF_BF16))
    x = torch.zeros(lo.n_rows, dtype=torch.float64, device="cuda")
    st, iters, rel = ddf.ddf_sptrsv_refine(q, b, x, tol=1e-14, max_iter=0)
    assert st == 12 and iters == 0 and rel > 1e-14
    p64 = ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), dev(lo.values), lo.n_cols, ddf.DDF_SPTRSV)
    st, _, _ = ddf.ddf_sptrsv_refine(p64, b, x)
    assert st == 1                                            # FP64-only plan
    a = synth.laplacian_7pt(10)
    pa = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV)
    y = torch.empty(a.n_rows, dtype=torch.float32, device="cuda")
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_spmv_lowp(pa, dev(np.ones(a.n_cols)).float(), y)
    assert e.value.status == 1
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV,
                        ddf.ddf_opts_default(store_dtype=7))
    assert e.value.status == 1


def test_update_values_refreshes_low_precision_copies():
    a = synth.elasticity_blocks(4)
    lo = synth.lower_triangle(a)
    q = ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), None, lo.n_cols, ddf.DDF_SPTRSV,
                        ddf.ddf_opts_default(store_dtype=ddf.DDF_F32))
    ddf.ddf_update_values(q, dev(lo.values * 3.0))
    b = synth.uniform_vector(lo.n_rows, 2)
    x = torch.zeros(lo.n_rows, dtype=torch.float64, device="cuda")
    st, iters, rel = ddf.ddf_sptrsv_refine(q, dev(b), x)
    assert st == 0
    lo3 = synth.CSR(lo.n_rows, lo.n_cols, lo.rowptr, lo.colidx, lo.values * 3.0)
    ref = oracle.sptrsv(lo3, b)
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["st27_168", "st27r_168"])
def test_precision_form_full_size(name):
    """The precision form at its full size: the 27-point stencil on 168^3
    (126.5M nonzeros) with integer values 26 / -1 (exact in FP32 and BF16)
    and with N(0,1) diagonally dominant values (rounded by FP32 / BF16).
    SpMV: every row within the FP32 accumulation bound of the oracle run on
    the same rounded inputs, and the normwise error against the FP64 oracle
    stated.  SpTRSV: refined to an oracle-computed relative residual <= 1e-12."""
    a, lo, x, b = synth.workload(name)
    y64 = oracle.spmv(a, x)
    k = np.maximum(np.diff(a.rowptr), 1)
    A = (dev(a.rowptr), dev(a.colidx), dev(a.values))
    for vdt, tdt, loose in ((ddf.DDF_F32, torch.float32, 1e-6), (ddf.DDF_BF16, torch.bfloat16, 1e-2)):
        av = rounded(a.values, vdt)
        xv = rounded(x, vdt)
        ar = synth.CSR(a.n_rows, a.n_cols, a.rowptr, a.colidx, av)
        ref = oracle.spmv(ar, xv)
        absref = oracle.spmv(synth.CSR(a.n_rows, a.n_cols, a.rowptr, a.colidx, np.abs(av)), np.abs(xv))
        p = ddf.ddf_inspect(*A, a.n_cols, ddf.DDF_SPMV, ddf.ddf_opts_default(store_dtype=vdt))
        y = torch.empty(a.n_rows, dtype=tdt, device="cuda")
        ddf.ddf_spmv_lowp(p, dev(xv).to(tdt), y)
        got = y.double().cpu().numpy()
        bound = 2 * k * U32 * absref + 1e-30
        if vdt == ddf.DDF_BF16:
            bound = bound + 2.0 ** -8 * np.abs(ref)
        assert np.all(np.abs(got - ref) <= bound)
        assert np.linalg.norm(got - y64) <= loose * np.linalg.norm(y64)
        del p
    del A
    torch.cuda.empty_cache()
    ref_x = oracle.sptrsv(lo, b)
    L = (dev(lo.rowptr), dev(lo.colidx), dev(lo.values))
    for vdt in (ddf.DDF_F32, ddf.DDF_BF16):
        q = ddf.ddf_inspect(*L, lo.n_cols, ddf.DDF_SPTRSV, ddf.ddf_opts_default(store_dtype=vdt))
        xr = torch.zeros(lo.n_rows, dtype=torch.float64, device="cuda")
        st, iters, rel = ddf.ddf_sptrsv_refine(q, dev(b), xr, tol=1e-12, max_iter=30)
        assert st == 0, (ddf.ddf_status_string(st), iters, rel)
        xs = xr.cpu().numpy()
        assert np.linalg.norm(b - oracle.spmv(lo, xs)) <= 1e-12 * np.linalg.norm(b)
        assert np.linalg.norm(xs - ref_x) <= 1e-10 * np.linalg.norm(ref_x)
        del q
    torch.cuda.empty_cache()
