"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

* plans: the exported GPU plan equals the oracle's Algorithm 1 output bit for
  bit (records, partition sequence, partition pointers, value offsets), and
  the oracle's plan-expansion check accepts it;
* SpMV / SpTRSV values: normwise relative error <= 1e-12 against the FP64
  oracle (the GPU sums in another order and uses fused multiply-adds and a
  reciprocal of the diagonal); integer cases must be exact;
* edge cases, validation errors and the bounded dependency wait.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2111_12243_gb300 as ddf
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12
KIND = {1: oracle.SPMV, 2: oracle.SPTRSV}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_12243_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def inspect(a, kind, on_device=True, values=True, **opts):
    o = ddf.ddf_opts_default(**opts)
    if on_device:
        return ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values) if values else None,
                               a.n_cols, kind, o)
    return ddf.ddf_inspect(a.rowptr, a.colidx, a.values if values else None, a.n_cols, kind, o)


def relerr(y, ref):
    nr = np.linalg.norm(ref)
    d = np.linalg.norm(y - ref)
    return d / nr if nr > 0 else d


def check_plan(a, kind, plan, t=256, allowed=7, weights=(8, 32, 4)):
    got = ddf.ddf_plan_export(plan)
    ref = oracle.inspect(a, KIND[kind], t=t, allowed=allowed, weights=weights)
    assert np.array_equal(got["seq"], ref.perm)
    assert np.array_equal(got["part_ptr"], ref.level_ptr)
    assert np.array_equal(got["gs"], ref.gs)
    assert got["records"].shape == ref.records.shape
    diff = np.flatnonzero(np.any(got["records"] != ref.records, axis=1))
    assert diff.size == 0, (diff[:5], got["records"][diff[:3]], ref.records[diff[:3]])
    rc = oracle.check_plan(a, KIND[kind], got["seq"], got["part_ptr"], got["gs"], got["records"])
    assert rc == (0, -1)
    return got


def run_spmv(plan, x, n_rows):
    y = torch.full((n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    ddf.ddf_spmv(plan, dev(x), y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def run_sptrsv(plan, b, n):
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    ddf.ddf_sptrsv(plan, dev(b), x)
    st = ddf.ddf_get_status(plan)
    assert st == 0, ddf.ddf_status_string(st)
    return x.cpu().numpy()


SMALL = {
    "lap5_16": lambda: synth.laplacian_5pt(16),
    "lap7_12": lambda: synth.laplacian_7pt(12),
    "elast_5": lambda: synth.elasticity_blocks(5),
    "st27_9": lambda: synth.stencil_27pt(9),
    "powerlaw_5000": lambda: synth.powerlaw(5000),
    "random_300": lambda: synth.random_pattern(300, 300, 0.03, 5, diag=True, empty_rows=0.1),
}


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("t", [256, 7])
def test_small_plans_and_values(name, t):
    a = SMALL[name]()
    lo = synth.lower_triangle(a, "unit_dominant" if name.startswith("power") else "keep")
    x = synth.uniform_vector(a.n_cols, 1)
    b = synth.uniform_vector(a.n_rows, 2)
    p = inspect(a, ddf.DDF_SPMV, window_t=t)
    check_plan(a, 1, p, t=t)
    assert relerr(run_spmv(p, x, a.n_rows), oracle.spmv(a, x)) <= TOL
    q = inspect(lo, ddf.DDF_SPTRSV, window_t=t)
    check_plan(lo, 2, q, t=t)
    assert relerr(run_sptrsv(q, b, a.n_rows), oracle.sptrsv(lo, b)) <= TOL
    st = ddf.ddf_plan_stats(q)
    assert st["depth"] == oracle.levels(lo)[1]


@pytest.mark.parametrize("allowed", [7, 5, 6, 4])
@pytest.mark.parametrize("weights", [(8, 32, 4), (1, 3, 1), (8, 0, 4), (1, 1000, 1)])
def test_plan_options(allowed, weights):
    a = synth.random_pattern(400, 400, 0.02, 9, diag=True, empty_rows=0.05)
    for m, kind in ((a, 1), (synth.lower_triangle(a), 2)):
        p = inspect(m, kind, allowed_types=allowed, w_op=weights[0], w_codelet=weights[1],
                    w_index=weights[2], window_t=64)
        check_plan(m, kind, p, t=64, allowed=allowed, weights=weights)


def test_integer_exact():
    a = synth.laplacian_7pt(20)
    xi = np.random.default_rng(1).integers(-40, 40, a.n_cols).astype(float)
    p = inspect(a, ddf.DDF_SPMV)
    assert np.array_equal(run_spmv(p, xi, a.n_rows), oracle.spmv(a, xi))
    lo = synth.random_pattern(500, 500, 0.02, 3, diag=True, lower=True, values="int")
    xt = np.random.default_rng(2).integers(-5, 6, 500).astype(float)
    b = oracle.spmv(lo, xt)
    q = inspect(lo, ddf.DDF_SPTRSV)
    assert np.array_equal(run_sptrsv(q, b, 500), xt)


def test_host_inputs_and_pattern_only():
    a = synth.elasticity_blocks(4)
    x = synth.uniform_vector(a.n_cols, 3)
    p = inspect(a, ddf.DDF_SPMV, on_device=False)
    assert relerr(run_spmv(p, x, a.n_rows), oracle.spmv(a, x)) <= TOL
    p2 = inspect(a, ddf.DDF_SPMV, values=False)
    with pytest.raises(ddf.DDFError):
        run_spmv(p2, x, a.n_rows)
    ddf.ddf_update_values(p2, a.values)                 # host values
    assert relerr(run_spmv(p2, x, a.n_rows), oracle.spmv(a, x)) <= TOL
    lo = synth.lower_triangle(a)
    q = inspect(lo, ddf.DDF_SPTRSV, values=False)
    ddf.ddf_update_values(q, dev(lo.values))            # device values
    b = synth.uniform_vector(a.n_rows, 4)
    assert relerr(run_sptrsv(q, b, a.n_rows), oracle.sptrsv(lo, b)) <= TOL
    # new values, same pattern: no re-inspection
    lo2 = synth.CSR(lo.n_rows, lo.n_cols, lo.rowptr, lo.colidx, lo.values * 2.0)
    ddf.ddf_update_values(q, lo2.values)
    assert relerr(run_sptrsv(q, b, a.n_rows), oracle.sptrsv(lo2, b)) <= TOL
    bad = lo.values.copy()
    bad[lo.rowptr[5] - 1] = 0.0
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_update_values(q, bad)
    assert e.value.status == 7


def csr(rows, n_cols, vals=None):
    rp = np.zeros(len(rows) + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in r], np.int32)
    v = np.arange(1, ci.size + 1, dtype=float) if vals is None else np.asarray(vals, float)
    return synth.CSR(len(rows), n_cols, rp, ci, v)


def test_edge_cases():
    # empty matrix
    z = synth.CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    p = ddf.ddf_inspect(z.rowptr, z.colidx, z.values, 0, ddf.DDF_SPMV)
    assert ddf.ddf_plan_export(p)["records"].shape == (0, 12)
    q = ddf.ddf_inspect(z.rowptr, z.colidx, z.values, 0, ddf.DDF_SPTRSV)
    assert ddf.ddf_plan_stats(q)["depth"] == 0
    # 1 x 1
    one = csr([[0]], 1, [4.0])
    assert run_spmv(inspect(one, 1), np.array([0.5]), 1).tolist() == [2.0]
    assert run_sptrsv(inspect(one, 2), np.array([2.0]), 1).tolist() == [0.5]
    # rectangular with empty rows and one long row (several warp passes)
    rng = np.random.default_rng(0)
    rows = [[], sorted(rng.choice(5000, 4000, replace=False).tolist()), [], [1, 2, 3], [4999]]
    a = csr(rows, 5000, rng.standard_normal(4004))
    x = synth.uniform_vector(5000, 1)
    p = inspect(a, 1, window_t=2)
    check_plan(a, 1, p, t=2)
    y = run_spmv(p, x, 5)
    assert y[0] == 0.0 and y[2] == 0.0
    assert relerr(y, oracle.spmv(a, x)) <= TOL
    # lower triangle with a dense last row and a diagonal-only first half
    n = 2000
    rows = [[i] for i in range(n // 2)] + [[i - 1, i] for i in range(n // 2, n - 1)] + [list(range(n))]
    lo = csr(rows, n, None)
    lo.values = np.where(np.isin(np.arange(lo.colidx.size), lo.rowptr[1:] - 1), 2.0, 0.001)
    b = synth.uniform_vector(n, 7)
    q = inspect(lo, 2, window_t=5)
    check_plan(lo, 2, q, t=5)
    assert relerr(run_sptrsv(q, b, n), oracle.sptrsv(lo, b)) <= TOL


@pytest.mark.parametrize("rows,n_cols,kind,code", [
    ([[0, 0]], 2, 1, 3),            # duplicate column
    ([[1, 0]], 2, 1, 3),            # unsorted
    ([[0, 5]], 2, 1, 4),            # out of range
    ([[0], [0, 1, 2], [2]], 3, 2, 5),  # above the diagonal
    ([[0], [0]], 2, 2, 6),          # missing diagonal
    ([[0, 1], [1]], 2, 2, 5),
    ([[0]], 2, 2, 2),               # not square
])
def test_validation_errors(rows, n_cols, kind, code):
    a = csr(rows, n_cols)
    with pytest.raises(ddf.DDFError) as e:
        inspect(a, kind)
    assert e.value.status == code
    with pytest.raises(ddf.DDFError) as e:
        inspect(a, kind, on_device=False)
    assert e.value.status == code


def _ragged(n, seed, lower):
    """Random CSR with rows of 0 to 100 sorted distinct columns (a few empty
    rows), so that rows and their pairs fall across 32-entry steps; lower:
    columns below the row, then the diagonal (values 1 off it, 4 on it)."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        m = int(rng.integers(0, 101)) if rng.random() > 0.05 else 0
        if lower:
            cols = np.unique(rng.integers(0, i, m)) if i > 0 else np.zeros(0, np.int64)
            rows.append(list(cols) + [i])
        else:
            rows.append(list(np.unique(rng.integers(0, n, m))))
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in r], np.int32)
    v = np.ones(ci.size)
    if lower:
        v[rp[1:] - 1] = 4.0
    return synth.CSR(n, n, rp, ci, v)


def _plant(a, k, col):
    b = synth.CSR(a.n_rows, a.n_cols, a.rowptr.copy(), a.colidx.copy(), a.values.copy())
    b.colidx[k] = col
    return b


def _straddling_pair(a):
    """An entry k with k % 32 == 31 whose successor is in the same row."""
    rp = a.rowptr
    for k in range(31, a.colidx.size - 1, 32):
        r = int(np.searchsorted(rp, k, side="right")) - 1
        if k + 1 < rp[r + 1]:
            return k
    raise AssertionError("no straddling pair")


@pytest.mark.parametrize("case", ["clean", "swap_straddling", "dup_straddling", "last_out_of_range",
                                  "negative_mid", "both"])
def test_validation_of_ragged_rows(case):
    # The CSR check streams each block of 32 rows in 32-entry steps: faults at
    # a step boundary, in the last entry and in the middle must all be found,
    # and descending columns across a row boundary must not be flagged.
    a = _ragged(3001, 11, lower=False)
    n, nnz = a.n_rows, a.colidx.size
    k = _straddling_pair(a)
    if case == "clean":
        b, code = a, 0
    elif case == "swap_straddling":
        b, code = _plant(a, k, a.colidx[k + 1]), 3
        b.colidx[k + 1] = a.colidx[k]
    elif case == "dup_straddling":
        b, code = _plant(a, k + 1, a.colidx[k]), 3
    elif case == "last_out_of_range":
        b, code = _plant(a, nnz - 1, n), 4
    elif case == "negative_mid":   # the first entry of a middle row: the row stays sorted
        r = int(np.nonzero(np.diff(a.rowptr)[n // 2:] > 0)[0][0]) + n // 2
        b, code = _plant(a, int(a.rowptr[r]), -1), 4
    else:
        b, code = _plant(a, nnz - 1, n), 3
        b.colidx[k + 1] = a.colidx[k]
    if code == 0:
        inspect(b, 1).destroy()
        return
    with pytest.raises(ddf.DDFError) as e:
        inspect(b, 1)
    assert e.value.status == code


@pytest.mark.parametrize("case,code", [("clean", 0), ("missing_diag_last_row", 6), ("above_diag", 5),
                                       ("zero_diag", 7), ("empty_row", 6)])
def test_validation_of_ragged_lower(case, code):
    a = _ragged(1001, 12, lower=True)   # 1001 rows: the last warp of rows is partial
    n, rp = a.n_rows, a.rowptr
    b = synth.CSR(n, n, rp.copy(), a.colidx.copy(), a.values.copy())
    if case == "missing_diag_last_row":   # drop the last row's diagonal
        m = b.colidx.size - 1
        nrp = rp.copy()
        nrp[n] = m
        b = synth.CSR(n, n, nrp, b.colidx[:m].copy(), b.values[:m].copy())
    elif case == "above_diag":
        r = 500
        b.colidx[rp[r + 1] - 1] = r + 1
    elif case == "zero_diag":
        b.values[rp[700] - 1] = 0.0
    elif case == "empty_row":
        r = 999
        keep = np.ones(b.colidx.size, bool)
        keep[rp[r]:rp[r + 1]] = False
        cnt = np.diff(rp)
        cnt[r] = 0
        nrp = np.zeros(n + 1, np.int32)
        nrp[1:] = np.cumsum(cnt)
        b = synth.CSR(n, n, nrp, b.colidx[keep], b.values[keep])
    if code == 0:
        inspect(b, 2).destroy()
        return
    with pytest.raises(ddf.DDFError) as e:
        inspect(b, 2)
    assert e.value.status == code


def test_zero_diagonal_rejected():
    a = csr([[0], [0, 1]], 2, [1.0, 1.0, 0.0])
    with pytest.raises(ddf.DDFError) as e:
        inspect(a, 2)
    assert e.value.status == 7


def test_wrong_kind_and_overlap():
    a = synth.laplacian_5pt(8)
    p = inspect(a, 1)
    x = torch.zeros(a.n_rows, dtype=torch.float64, device="cuda")
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_sptrsv(p, x, x)
    assert e.value.status == 8
    q = inspect(synth.lower_triangle(a), 2)
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_sptrsv(q, x, x)
    assert e.value.status == 1


@pytest.mark.parametrize("coarsen", [0, 256])
def test_dependency_wait_times_out_and_recovers(coarsen):
    # Point one off-diagonal entry of a PSC II row r (executed through its
    # column indices) at a row d that itself reads r: r waits for d and d for
    # r, so the wait must run out, latch DDF_ERR_TIMEOUT, and leave the
    # context usable.  In a coarsened plan only entries that name a column
    # before the row's block go through the flag protocol (the rest are
    # ordered by the block's own schedule), so the planted entry is the first
    # entry of a row whose first column lies in an earlier block.
    lo = synth.random_pattern(3000, 3000, 0.003, 17, diag=True, lower=True)
    q = inspect(lo, 2, spin_cap_ns=50_000_000, coarsen_rows=coarsen)
    exp = ddf.ddf_plan_export(q)
    rec, seq, gs = exp["records"], exp["seq"], exp["gs"]
    offl = np.diff(lo.rowptr) - 1
    rows_of = np.repeat(np.arange(lo.n_rows), np.diff(lo.rowptr))
    target = None
    for r in rec[(rec[:, 1] == 2) & (rec[:, 0] >= 1)]:
        for pos in range(r[2], r[2] + r[3]):
            row = int(seq[pos])
            if offl[row] < 1:
                continue
            if coarsen and lo.colidx[lo.rowptr[row]] >= (row // coarsen) * coarsen:
                continue
            deps = rows_of[(lo.colidx == row) & (rows_of != row)]
            if deps.size:
                target = (int(gs[pos]), int(deps[0]))
                break
        if target:
            break
    assert target is not None
    ddf.ddf_debug_set_dependency(q, *target)
    b = synth.uniform_vector(lo.n_rows, 1)
    x = torch.zeros(lo.n_rows, dtype=torch.float64, device="cuda")
    ddf.ddf_sptrsv(q, dev(b), x)
    assert ddf.ddf_get_status(q) == 11
    assert ddf.ddf_get_status(q) == 0     # cleared
    assert torch.isnan(x).any()
    with pytest.raises(ddf.DDFError):
        ddf.ddf_debug_set_dependency(q, -1, 0)
    # the device is still usable
    q2 = inspect(lo, 2)
    assert relerr(run_sptrsv(q2, b, lo.n_rows), oracle.sptrsv(lo, b)) <= TOL


def test_launch_counts():
    a = synth.laplacian_7pt(10)
    p = inspect(a, 1)
    run_spmv(p, np.ones(a.n_cols), a.n_rows)
    st = ddf.ddf_plan_stats(p)
    assert ddf.ddf_last_launches(p) == sum(1 for c in st["ncodelets"] if c > 0)
    q = inspect(synth.lower_triangle(a), 2)
    run_sptrsv(q, np.ones(a.n_rows), a.n_rows)
    assert ddf.ddf_last_launches(q) == 2


FULL = {
    "lap5_64": lambda: synth.workload("lap5_64"),
    "lap7_128": lambda: synth.workload("lap7_128"),
    "elast3x3_64": lambda: synth.workload("elast3x3_64"),
    "powerlaw_4m": lambda: synth.workload("powerlaw_4m"),
    "st27_168": lambda: synth.workload("st27_168"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", list(FULL))
def test_full_size_parity(name):
    """Full workload sizes, default options (the benchmark's configuration):
    complete plans and complete result vectors against the oracle."""
    a, lo, x, b = FULL[name]()
    p = inspect(a, ddf.DDF_SPMV)
    check_plan(a, 1, p)
    assert relerr(run_spmv(p, x, a.n_rows), oracle.spmv(a, x)) <= TOL
    del p
    q = inspect(lo, ddf.DDF_SPTRSV)
    check_plan(lo, 2, q)
    xs = run_sptrsv(q, b, lo.n_rows)
    assert relerr(xs, oracle.sptrsv(lo, b)) <= TOL
    # relative residual of the GPU solution, computed by the oracle in FP64
    r = b - oracle.spmv(lo, xs)
    assert np.linalg.norm(r) <= TOL * np.linalg.norm(b)
    del q
    torch.cuda.empty_cache()


@pytest.mark.parametrize("name", ["elast_5", "powerlaw_5000", "random_300"])
@pytest.mark.parametrize("coarsen", [0, 64])
def test_deterministic_plans_and_results(name, coarsen):
    """Two inspections of one matrix give identical plans (every exported
    array), and two executions identical bits: every reduction has a fixed
    order."""
    a = SMALL[name]()
    lo = synth.lower_triangle(a, "unit_dominant" if name.startswith("power") else "keep")
    x = synth.uniform_vector(a.n_cols, 2)
    b = synth.uniform_vector(lo.n_rows, 3)
    exports, ys, xs = [], [], []
    for _ in range(2):
        p = inspect(a, 1)
        q = inspect(lo, 2, coarsen_rows=coarsen)
        exports.append((ddf.ddf_plan_export(p), ddf.ddf_plan_export(q)))
        ys.append(run_spmv(p, x, a.n_rows))
        xs.append(run_sptrsv(q, b, lo.n_rows))
    for k in ("records", "seq", "part_ptr", "gs"):
        assert np.array_equal(exports[0][0][k], exports[1][0][k])
        assert np.array_equal(exports[0][1][k], exports[1][1][k])
    assert np.array_equal(ys[0].view(np.uint64), ys[1].view(np.uint64))
    assert np.array_equal(xs[0].view(np.uint64), xs[1].view(np.uint64))
