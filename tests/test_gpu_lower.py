"""SpTRSV plans built from a square matrix A with lower_of_input = 1: the
inspector reads each row's lower part (the prefix of the sorted row that ends
with the diagonal) in place.  Such a plan must equal, bit for bit, the plan
inspected from the lower triangle L = tril(A) (and the oracle's plan of L),
and solve identically; ddf_update_values takes A's values; faults of A are
reported with the same codes as for L."""
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


def inspect(m, on_device=True, values=True, **opts):
    arrs = (m.rowptr, m.colidx, m.values if values else None)
    if on_device:
        arrs = tuple(dev(a) if a is not None else None for a in arrs)
    return ddf.ddf_inspect(*arrs, m.n_cols, ddf.DDF_SPTRSV, ddf.ddf_opts_default(**opts))


def solve(q, b):
    x = torch.empty(len(b), dtype=torch.float64, device="cuda")
    ddf.ddf_sptrsv(q, dev(b), x)
    assert ddf.ddf_get_status(q) == 0
    return x


def same_plan(p, q):
    a, b = ddf.ddf_plan_export(p), ddf.ddf_plan_export(q)
    return all(np.array_equal(a[k], b[k]) for k in ("records", "seq", "part_ptr", "gs"))


MATS = {
    "lap7_12": lambda: synth.laplacian_7pt(12),
    "elast_5": lambda: synth.elasticity_blocks(5),
    "st27_8": lambda: synth.stencil_27pt(8),
    "random_3000": lambda: synth.random_pattern(3000, 3000, 0.003, 21, diag=True),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("coarsen", [0, 128])
def test_plan_from_lower_part_equals_plan_of_l(name, coarsen):
    a = MATS[name]()
    lo = synth.lower_triangle(a)
    p = inspect(a, lower_of_input=1, coarsen_rows=coarsen)
    q = inspect(lo, coarsen_rows=coarsen)
    assert same_plan(p, q)
    exp = ddf.ddf_plan_export(p)
    okind = oracle.SPTRSV
    ref = oracle.inspect(lo, okind, coarsen=coarsen)
    assert np.array_equal(exp["records"], ref.records)
    assert oracle.check_plan(lo, okind, exp["seq"], exp["part_ptr"], exp["gs"], exp["records"]) == (0, -1)
    st_p, st_q = ddf.ddf_plan_stats(p), ddf.ddf_plan_stats(q)
    for k in ("nnz", "points", "depth", "levels", "bytes_exec", "ncodelets"):
        assert st_p[k] == st_q[k], k
    b = synth.uniform_vector(lo.n_rows, 3)
    xp, xq = solve(p, b), solve(q, b)
    assert torch.equal(xp, xq)
    xr = oracle.sptrsv(lo, b)
    assert np.linalg.norm(xp.cpu().numpy() - xr) <= TOL * np.linalg.norm(xr)
    assert ddf.ddf_plan_validate(p) == 0


def test_host_input_pattern_only_and_new_values():
    a = synth.elasticity_blocks(4)
    lo = synth.lower_triangle(a)
    b = synth.uniform_vector(lo.n_rows, 5)
    p = inspect(a, on_device=False, values=False, lower_of_input=1)
    ddf.ddf_update_values(p, a.values)                      # A's values, host
    q = inspect(lo)
    assert torch.equal(solve(p, b), solve(q, b))
    # new values of A, same pattern: the plan takes them from A's layout
    a2 = synth.CSR(a.n_rows, a.n_cols, a.rowptr, a.colidx, a.values * 1.5 + 0.25)
    ddf.ddf_update_values(p, dev(a2.values))
    lo2 = synth.lower_triangle(a2)
    ddf.ddf_update_values(q, lo2.values)
    assert torch.equal(solve(p, b), solve(q, b))
    bad = a2.values.copy()
    r = 7
    diag_k = a.rowptr[r] + int(np.searchsorted(a.colidx[a.rowptr[r]:a.rowptr[r + 1]], r))
    bad[diag_k] = 0.0
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_update_values(p, bad)
    assert e.value.status == 7


def test_refined_low_precision_and_save_load():
    a = synth.laplacian_7pt(10)
    lo = synth.lower_triangle(a)
    b = synth.uniform_vector(lo.n_rows, 6)
    p = inspect(a, lower_of_input=1, store_dtype=ddf.DDF_F32)
    x = torch.empty(lo.n_rows, dtype=torch.float64, device="cuda")
    st = ddf.ddf_sptrsv_refine(p, dev(b), x)
    assert st[0] == 0
    xr = oracle.sptrsv(lo, b)
    assert np.linalg.norm(x.cpu().numpy() - xr) <= TOL * np.linalg.norm(xr)
    p2 = ddf.ddf_plan_load(ddf.ddf_plan_save(p), a.n_rows, a.n_cols, ddf.DDF_SPTRSV)
    assert same_plan(p, p2)
    a3 = synth.CSR(a.n_rows, a.n_cols, a.rowptr, a.colidx, a.values * 3.0)
    ddf.ddf_update_values(p2, a3.values)                    # reloaded plan still maps A's layout
    q3 = inspect(synth.lower_triangle(a3))
    x2 = torch.empty_like(x)
    ddf.ddf_sptrsv(p2, dev(b), x2)
    assert ddf.ddf_get_status(p2) == 0
    assert torch.equal(x2, solve(q3, b))


def csr(rows, n_cols, vals=None):
    rp = np.zeros(len(rows) + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in r], np.int32)
    v = np.ones(len(ci)) if vals is None else np.asarray(vals, float)
    return synth.CSR(len(rows), n_cols, rp, ci, v)


@pytest.mark.parametrize("rows,n_cols,vals,code", [
    ([[0, 1], [1, 0]], 2, None, 3),                 # unsorted row
    ([[0, 5], [1]], 2, None, 4),                    # column out of range
    ([[0, 1], [0, 2], [2]], 3, None, 6),            # row 1 holds no diagonal
    ([[1], [1]], 2, None, 6),                       # row 0: nothing at or below the diagonal
    ([[0, 1], [0, 1]], 2, [1.0, 2.0, 3.0, 0.0], 7),  # zero diagonal
    ([[0]], 2, None, 2),                            # not square
])
def test_faults_of_a(rows, n_cols, vals, code):
    a = csr(rows, n_cols, vals)
    for on_device in (True, False):
        with pytest.raises(ddf.DDFError) as e:
            inspect(a, on_device=on_device, lower_of_input=1)
        assert e.value.status == code


def test_option_is_sptrsv_only():
    a = synth.laplacian_5pt(6)
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, ddf.DDF_SPMV,
                        ddf.ddf_opts_default(lower_of_input=1))
    assert e.value.status == 1
    with pytest.raises(ddf.DDFError) as e:
        inspect(a, lower_of_input=2)
    assert e.value.status == 1
