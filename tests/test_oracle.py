"""Pins for the CPU oracle (no GPU).

Every check here ties the oracle to something other than itself: dense brute
force, LAPACK, closed forms, exact integer arithmetic, known level depths,
the paper's worked example (tests/golden/worked_example.json) and planted
mistakes that the plan checker must catch.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import fopd
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")


def dense(a):
    d = np.zeros((a.n_rows, a.n_cols))
    for i in range(a.n_rows):
        for k in range(a.rowptr[i], a.rowptr[i + 1]):
            d[i, a.colidx[k]] += a.values[k]
    return d


def csr_from_rows(rows, n_cols=None, values=None):
    """CSR from a list of column lists (values 1..nnz unless given)."""
    rp = [0]
    ci = []
    for r in rows:
        ci.extend(r)
        rp.append(len(ci))
    n_cols = n_cols if n_cols is not None else (max(ci) + 1 if ci else len(rows))
    v = np.arange(1, len(ci) + 1, dtype=np.float64) if values is None else np.asarray(values, float)
    return synth.CSR(len(rows), n_cols, np.array(rp, np.int32), np.array(ci, np.int32), v)


# ---------------------------------------------------------------------------
# SpMV and SpTRSV values
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("shape", [(1, 1), (5, 7), (33, 33), (64, 40)])
def test_spmv_matches_dense_brute_force(seed, shape):
    a = synth.random_pattern(shape[0], shape[1], 0.3, seed, empty_rows=0.1)
    x = synth.uniform_vector(shape[1], seed + 7)
    y = oracle.spmv(a, x)
    d = dense(a)
    ref = d @ x
    # forward error bound of a dot product of length k: gamma_k |A| |x|
    k = max(1, int(np.diff(a.rowptr).max(initial=1)))
    u = np.finfo(float).eps / 2
    bound = (k * u / (1 - k * u)) * (np.abs(d) @ np.abs(x)) * 2 + 1e-300
    assert np.all(np.abs(y - ref) <= bound)


def test_spmv_empty_and_integer_exact():
    a = csr_from_rows([[], [0], [], [0, 1, 2]], n_cols=3, values=[2.0, 1.0, -3.0, 4.0])
    y = oracle.spmv(a, np.array([1.0, 2.0, 3.0]))
    assert y.tolist() == [0.0, 2.0, 0.0, 1.0 - 6.0 + 12.0]
    z = synth.CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert oracle.spmv(z, np.zeros(0)).size == 0


@pytest.mark.parametrize("threads", [1, 2, 3, 8, 64])
def test_spmv_parallel_equals_sequential_and_brute_force(threads):
    # the row split must cover every row once (a skipped or doubled boundary
    # row would differ), and each row is summed in CSR order, so the result is
    # the sequential one bit for bit; it is also within the dot-product bound
    # of the dense product
    a = synth.random_pattern(97, 50, 0.2, 5, empty_rows=0.2)
    x = synth.uniform_vector(50, 12)
    y = oracle.spmv_par(a, x, threads)
    assert np.array_equal(y, oracle.spmv(a, x))
    d = dense(a)
    assert np.allclose(y, d @ x, rtol=0, atol=1e-12)
    z = synth.CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert oracle.spmv_par(z, np.zeros(0), threads).size == 0
    p = synth.powerlaw(5000, 3)
    xp = synth.uniform_vector(5000, 4)
    assert np.array_equal(oracle.spmv_par(p, xp, threads), oracle.spmv(p, xp))


def test_spmv_stencil_closed_forms():
    # A * 1 = row sums: zero on interior Laplacian rows, 6 - #neighbours on the boundary
    a = synth.laplacian_7pt(9)
    y = oracle.spmv(a, np.ones(a.n_cols))
    n = 9
    idx = np.arange(a.n_rows)
    ix, iy, iz = idx % n, (idx // n) % n, idx // (n * n)
    nb = ((ix > 0).astype(int) + (ix < n - 1) + (iy > 0) + (iy < n - 1) + (iz > 0) + (iz < n - 1))
    assert np.array_equal(y, 6.0 - nb)
    # integer x: every partial sum is an exact integer, so the result is exact
    rng = np.random.default_rng(3)
    xi = rng.integers(-50, 50, a.n_cols).astype(float)
    yi = oracle.spmv(a, xi)
    assert np.array_equal(yi, dense(a).astype(np.int64) @ xi.astype(np.int64))


@pytest.mark.parametrize("seed", range(6))
def test_sptrsv_matches_lapack(seed):
    lo = synth.random_pattern(48, 48, 0.2, seed, diag=True, lower=True)
    b = synth.uniform_vector(48, seed + 1)
    x = oracle.sptrsv(lo, b)
    ref = scipy.linalg.solve_triangular(dense(lo), b, lower=True)
    assert np.linalg.norm(x - ref) <= 1e-13 * np.linalg.norm(ref)


def test_sptrsv_manufactured_integer_exact():
    # unit diagonal and integer entries: forward substitution is exact
    lo = synth.random_pattern(200, 200, 0.05, 11, diag=True, lower=True, values="int")
    xt = np.random.default_rng(0).integers(-5, 6, 200).astype(float)
    b = dense(lo).astype(np.int64) @ xt.astype(np.int64)
    assert np.array_equal(oracle.sptrsv(lo, b.astype(float)), xt)
    # power-of-two diagonal keeps the division exact as well
    lo2 = synth.lower_triangle(synth.laplacian_5pt(8))
    lo2.values = np.where(lo2.values == 4.0, 4.0, -1.0)
    xt2 = np.arange(64, dtype=float) * 4.0
    b2 = dense(lo2) @ xt2
    assert np.array_equal(oracle.sptrsv(lo2, b2), xt2)


def test_sptrsv_errors():
    with pytest.raises(oracle.OracleError):
        oracle.sptrsv(csr_from_rows([[0], [0]], n_cols=2), np.ones(2))     # missing diagonal
    with pytest.raises(oracle.OracleError):
        oracle.sptrsv(csr_from_rows([[0], [0, 1]], values=[1.0, 1.0, 0.0]), np.ones(2))  # zero diagonal
    with pytest.raises(oracle.OracleError):
        oracle.sptrsv(csr_from_rows([[0, 1], [1]], n_cols=2), np.ones(2))  # above the diagonal


# ---------------------------------------------------------------------------
# levels
# ---------------------------------------------------------------------------

def longest_path_levels(lo):
    """Levels by memoised DFS on the reversed DAG (independent of row order)."""
    import sys
    sys.setrecursionlimit(10000)
    preds = [[int(j) for j in lo.colidx[lo.rowptr[i]:lo.rowptr[i + 1]] if j != i]
             for i in range(lo.n_rows)]
    memo = {}

    def lev(i):
        if i not in memo:
            memo[i] = 0 if not preds[i] else 1 + max(lev(j) for j in preds[i])
        return memo[i]

    return np.array([lev(i) for i in reversed(range(lo.n_rows))][::-1])


@pytest.mark.parametrize("seed", range(5))
def test_levels_brute_force(seed):
    lo = synth.random_pattern(120, 120, 0.04, seed, diag=True, lower=True)
    lev, depth = oracle.levels(lo)
    ref = longest_path_levels(lo)
    assert np.array_equal(lev, ref)
    assert depth == ref.max() + 1
    lp, perm = oracle.level_order(lev, depth)
    assert np.array_equal(perm, np.lexsort((np.arange(120), lev)))
    assert np.array_equal(np.diff(lp), np.bincount(lev, minlength=depth))


@pytest.mark.parametrize("k", [4, 7, 12])
def test_level_depth_closed_forms(k):
    # 5-pt: level = ix + iy; 7-pt: ix + iy + iz; 27-pt: ix + 2 iy + 4 iz
    lev, depth = oracle.levels(synth.lower_triangle(synth.laplacian_5pt(k)))
    assert depth == 2 * (k - 1) + 1
    lev, depth = oracle.levels(synth.lower_triangle(synth.laplacian_7pt(k)))
    idx = np.arange(k ** 3)
    assert np.array_equal(lev, idx % k + (idx // k) % k + idx // (k * k))
    lev, depth = oracle.levels(synth.lower_triangle(synth.stencil_27pt(k)))
    assert np.array_equal(lev, idx % k + 2 * ((idx // k) % k) + 4 * (idx // (k * k)))
    assert depth == 7 * (k - 1) + 1


def test_level_depth_paper_sizes():
    # the 64x64 5-point grid has 127 levels
    assert oracle.levels(synth.lower_triangle(synth.laplacian_5pt(64)))[1] == 127


# ---------------------------------------------------------------------------
# Section III definitions and the worked example
# ---------------------------------------------------------------------------

def example_tables():
    g = json.load(open(GOLDEN))
    m, n = g["region"]["rows"], g["region"]["row_length"]
    s = np.array(g["region"]["column_offsets_s"])
    i0 = np.arange(m)[:, None]
    i1 = np.arange(n)[None, :]
    f = np.broadcast_to(i0, (m, n))
    gg = g["region"]["gamma"] * i0 + i1
    h = g["region"]["delta"] * i0 + s[None, :]
    return g, f, gg, h


def test_worked_example_fopd_and_class():
    g, f, gg, h = example_tables()
    assert fopd.fopd_i1(h)[1, 1] == g["fopd"]["dh_di1_at_1_1"]
    assert fopd.fopd_i1(gg)[0, 0] == g["fopd"]["dg_di1_at_0_0"]
    assert fopd.fopd_i1(gg)[0, 1] == g["fopd"]["dg_di1_at_0_1"]
    assert fopd.fopd_i0(gg)[0, 0] == g["fopd"]["dg_di0_at_0_0"]
    assert fopd.fopd_i0(gg)[1, 0] == g["fopd"]["dg_di0_at_1_0"]
    flags, name = fopd.classify(f, gg, h)
    c = g["classification"]
    assert flags == (c["f_strided"], c["g_strided"], c["h_strided"])
    assert name == c["class"]


def test_worked_example_loads_and_eq1():
    g, f, gg, h = example_tables()
    assert fopd.loads(h) == g["loads"]["psc1_h"]
    # one BLAS codelet per column i1: every function strided along i0
    cols = [(f[:, [j]], gg[:, [j]], h[:, [j]]) for j in range(h.shape[1])]
    assert all(fopd.classify(*c)[1] == "BLAS" for c in cols)
    assert len(cols) == g["loads"]["blas_codelets_min"]
    assert sum(fopd.loads(t) for c in cols for t in c) == g["loads"]["blas_loads"]
    # the whole region is not BLAS (h has Delta_i1 = 2 then 3); by the strided
    # definition alone a pair of columns is (constant Delta_i1), so the text's
    # count of 3 BLAS codelets is the one-codelet-per-column cover
    assert fopd.classify(f, gg, h)[1] != "BLAS"
    assert fopd.classify(f[:, :2], gg[:, :2], h[:, :2])[1] == "BLAS"
    assert fopd.classify(f[:2, :], gg[:2, :], h[:2, :])[1] != "BLAS"
    w = oracle.PAPER_WEIGHTS
    psc1 = oracle.codelet_cost(9, 0, 0, 3, w)
    blas = sum(oracle.codelet_cost(3, 0, 0, 0, w) for _ in range(3))
    assert psc1 == g["eq1_costs_paper_weights"]["psc1"]
    assert blas == g["eq1_costs_paper_weights"]["blas_three_columns"]


def test_worked_example_inspector():
    g = json.load(open(GOLDEN))
    s = g["region"]["column_offsets_s"]
    a = csr_from_rows([[i + o for o in s] for i in range(3)])
    p = oracle.inspect(a, oracle.SPMV, t=8, weights=oracle.PAPER_WEIGHTS)
    assert p.records.shape[0] == 1
    r = dict(zip(oracle.FIELDS, p.records[0].tolist()))
    assert r["type"] == oracle.PSC1 and r["m"] == 3 and r["n"] == 3
    assert (r["f_str"], r["rho"], r["g_str"], r["gamma"]) == (1, 1, 1, 3)
    assert (r["h0"], r["delta"]) == (0, 1)
    assert oracle.plan_cost(a, p, oracle.PAPER_WEIGHTS) == 15


def test_seven_point_interior_is_psc1():
    k = 10
    a = synth.laplacian_7pt(k)
    p = oracle.inspect(a, oracle.SPMV, t=k, weights=(8, 32, 4))
    # an x-line of interior rows (y, z interior) is one PSC I codelet with
    # s = {-N^2, -N, -1, 0, 1, N, N^2} relative to the row, delta = 1
    row0 = 1 + k * (3 + k * 4)
    recs = [dict(zip(oracle.FIELDS, r)) for r in p.records.tolist()]
    c = [r for r in recs if r["q0"] == row0]
    assert len(c) == 1
    c = c[0]
    assert c["type"] == oracle.PSC1 and c["m"] == k - 2 and c["n"] == 7 and c["delta"] == 1
    s = a.colidx[a.rowptr[row0]:a.rowptr[row0 + 1]] - row0
    assert s.tolist() == [-k * k, -k, -1, 0, 1, k, k * k]
    assert c["h0"] == row0 - k * k


def test_special_cases_blas():
    # diagonal matrix: one BLAS run per region, sigma irrelevant, delta = 1
    a = csr_from_rows([[i] for i in range(40)])
    p = oracle.inspect(a, oracle.SPMV, t=16)
    assert [tuple(r[[1, 2, 3, 4, 10]]) for r in p.records] == [
        (0, 0, 16, 1, 1), (0, 16, 16, 1, 1), (0, 32, 8, 1, 1)]
    # dense 4x6 block: one BLAS codelet, delta 0, sigma 1
    a = csr_from_rows([list(range(6))] * 4)
    p = oracle.inspect(a, oracle.SPMV, t=16)
    assert p.records.shape[0] == 1
    assert tuple(p.records[0][[1, 3, 4, 8, 9, 10, 11]]) == (0, 4, 6, 6, 0, 0, 1)
    # tridiagonal interior rows: BLAS with delta 1, sigma 1
    n = 20
    a = csr_from_rows([[j for j in (i - 1, i, i + 1) if 0 <= j < n] for i in range(n)])
    p = oracle.inspect(a, oracle.SPMV, t=64)
    recs = [dict(zip(oracle.FIELDS, r)) for r in p.records.tolist()]
    mid = [r for r in recs if r["q0"] == 1][0]
    assert (mid["type"], mid["m"], mid["n"], mid["delta"], mid["sigma"]) == (0, n - 2, 3, 1, 1)


def test_min_cost_prefers_psc2_on_irregular_rows():
    # short rows of different lengths: only PSC II pieces are possible except
    # for 1-2 nnz rows, whose BLAS singletons cost more than staying in one run
    rows = [[0, 3, 9], [1, 2], [0, 4, 5, 11], [2, 7, 8], [3], [1, 6, 10, 12, 13]]
    a = csr_from_rows(rows, n_cols=14)
    p = oracle.inspect(a, oracle.SPMV, t=8, weights=oracle.PAPER_WEIGHTS)
    assert p.records.shape[0] == 1 and p.records[0][1] == oracle.PSC2
    # paper weights, by hand: |p| = 18; f strided (|s_f| = 0); unequal lengths so
    # |s_g| = m = 6; |s_h| = |p|: 18 + 3 + 6 + 18 = 45.  BLAS_first would make
    # BLAS singletons of rows 1 and 4 (5 + 4) and PSC II pieces [0] (9),
    # [2,3] (7+3+2+7 = 19) and [5] (13): 50 > 45.
    assert oracle.plan_cost(a, p, oracle.PAPER_WEIGHTS) == 45
    alt = oracle.Plan(oracle.SPMV, np.array([
        [0, 2, 0, 1, -1, 1, 0, 1, 0, 0, 0, 0], [0, 0, 1, 1, 2, 1, 0, 1, 0, 1, 0, 1],
        [0, 2, 2, 2, -1, 1, 1, 0, 0, 0, 0, 0], [0, 0, 4, 1, 1, 1, 0, 1, 0, 3, 0, 0],
        [0, 2, 5, 1, -1, 1, 0, 1, 0, 0, 0, 0]]), p.perm, p.level_ptr, p.gs)
    assert oracle.check_plan(a, oracle.SPMV, alt.perm, alt.level_ptr, alt.gs, alt.records) == (0, -1)
    assert oracle.plan_cost(a, alt, oracle.PAPER_WEIGHTS) == 50


def test_allowed_masks():
    a = synth.laplacian_7pt(6)
    only2 = oracle.inspect(a, oracle.SPMV, t=32, allowed=oracle.ALLOW_PSC2)
    assert set(only2.records[:, 1].tolist()) == {oracle.PSC2}
    assert only2.records.shape[0] == -(-a.n_rows // 32)
    blas_only = oracle.inspect(a, oracle.SPMV, t=32, allowed=oracle.ALLOW_BLAS | oracle.ALLOW_PSC2)
    assert oracle.PSC1 not in set(blas_only.records[:, 1].tolist())
    with pytest.raises(oracle.OracleError):
        oracle.inspect(a, oracle.SPMV, allowed=oracle.ALLOW_BLAS)


# ---------------------------------------------------------------------------
# plan validity: expansion == trace, re-derived classes, planted mistakes
# ---------------------------------------------------------------------------

def rederive(a, kind, plan, allowed=oracle.ALLOW_ALL):
    """Check every record's claims against the trace-level definitions."""
    off = kind == oracle.SPTRSV
    lens = np.diff(a.rowptr.astype(np.int64))[plan.perm] - (1 if off else 0)
    for r in plan.records:
        rec = dict(zip(oracle.FIELDS, r.tolist()))
        q0, m = rec["q0"], rec["m"]
        seqs = plan.perm[q0:q0 + m]
        assert bool(rec["f_str"]) == fopd.is_strided_1d(seqs)
        eq = bool(np.all(lens[q0:q0 + m] == lens[q0]))
        if eq:
            f, g, h = fopd.sequence_tables(a.rowptr, a.colidx, plan.perm, plan.gs, q0, m, off)
            gstr = fopd.is_strided(g) and fopd.is_strided_1d(plan.gs[q0:q0 + m])
        else:
            gstr = False
        assert bool(rec["g_str"]) == gstr
        if rec["type"] == oracle.BLAS:
            assert rec["f_str"] and gstr and fopd.is_strided(h)
        elif rec["type"] == oracle.PSC1:
            assert rec["f_str"] and gstr
            # a fully strided run is typed PSC I only when BLAS is not allowed
            assert (not fopd.is_strided(h)) or not (allowed & oracle.ALLOW_BLAS)
            so = fopd.shared_offsets(h)
            assert so is not None and so[0] == rec["h0"] and so[1] == rec["delta"]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("t", [1, 3, 16, 64])
def test_plan_valid_random(seed, t):
    a = synth.random_pattern(90, 90, 0.06, seed, diag=True, empty_rows=0.1)
    for kind, mat in ((oracle.SPMV, a), (oracle.SPTRSV, synth.lower_triangle(a))):
        for allowed in (7, 5, 6, 4):
            p = oracle.inspect(mat, kind, t=t, allowed=allowed)
            assert oracle.check_plan(mat, kind, p.perm, p.level_ptr, p.gs, p.records) == (0, -1)
            rederive(mat, kind, p, allowed)


@pytest.mark.parametrize("builder", [lambda: synth.laplacian_7pt(7), lambda: synth.elasticity_blocks(4),
                                     lambda: synth.stencil_27pt(5), lambda: synth.powerlaw(3000)])
def test_plan_valid_structured(builder):
    a = builder()
    for kind, mat in ((oracle.SPMV, a), (oracle.SPTRSV, synth.lower_triangle(a))):
        p = oracle.inspect(mat, kind, t=64)
        assert oracle.check_plan(mat, kind, p.perm, p.level_ptr, p.gs, p.records) == (0, -1)
        rederive(mat, kind, p)
        if kind == oracle.SPTRSV:
            lev, depth = oracle.levels(mat)
            assert p.nparts == depth


def test_checker_catches_planted_mistakes():
    a = synth.laplacian_7pt(6)
    p = oracle.inspect(a, oracle.SPMV, t=64)
    ok = oracle.check_plan(a, oracle.SPMV, p.perm, p.level_ptr, p.gs, p.records)
    assert ok == (0, -1)
    i = int(np.flatnonzero(p.records[:, 1] == oracle.PSC1)[0])
    for field, delta in (("delta", 1), ("h0", 1), ("m", 1), ("m", -1), ("gamma", 1), ("rho", 1),
                         ("n", 1), ("q0", 1), ("type", -1)):
        bad = p.records.copy()
        bad[i, oracle.FIELDS.index(field)] += delta
        rc, where = oracle.check_plan(a, oracle.SPMV, p.perm, p.level_ptr, p.gs, bad)
        assert rc != 0, field
    # dropping a record leaves positions uncovered
    rc, _ = oracle.check_plan(a, oracle.SPMV, p.perm, p.level_ptr, p.gs, np.delete(p.records, i, 0))
    assert rc == 9


# ---------------------------------------------------------------------------
# Coarsened SpTRSV partitions (LBC-style, Sec. IV-A): (block of R rows, level)
# ---------------------------------------------------------------------------

def brute_levels(lo):
    """Longest incoming path of every row by repeated relaxation (no ordering)."""
    n = lo.n_rows
    lev = np.zeros(n, np.int64)
    changed = True
    while changed:
        changed = False
        for i in range(n):
            for k in range(lo.rowptr[i], lo.rowptr[i + 1]):
                j = lo.colidx[k]
                if j < i and lev[j] + 1 > lev[i]:
                    lev[i] = lev[j] + 1
                    changed = True
    return lev


COARSE_MATS = {
    "lap5_9": lambda: synth.lower_triangle(synth.laplacian_5pt(9)),
    "lap7_5": lambda: synth.lower_triangle(synth.laplacian_7pt(5)),
    "elast_3": lambda: synth.lower_triangle(synth.elasticity_blocks(3)),
    "powerlaw_300": lambda: synth.lower_triangle(synth.powerlaw(300), "unit_dominant"),
}


@pytest.mark.parametrize("name", sorted(COARSE_MATS))
@pytest.mark.parametrize("R", [1, 7, 32, 100])
def test_coarse_order_is_sorted_by_block_level_row(name, R):
    lo = COARSE_MATS[name]()
    lev = brute_levels(lo)
    depth = int(lev.max()) + 1
    pp, perm = oracle.coarse_order(lev.astype(np.int32), depth, R)
    keys = [(i // R, int(lev[i]), i) for i in range(lo.n_rows)]
    want = sorted(range(lo.n_rows), key=lambda i: keys[i])
    assert perm.tolist() == want
    starts = [q for q in range(lo.n_rows) if q == 0 or keys[want[q]][:2] != keys[want[q - 1]][:2]]
    assert pp.tolist() == starts + [lo.n_rows]
    assert oracle.check_schedule(lo, perm, pp) == (0, -1)


@pytest.mark.parametrize("name", sorted(COARSE_MATS))
def test_one_block_equals_level_sets(name):
    lo = COARSE_MATS[name]()
    plain = oracle.inspect(lo, oracle.SPTRSV)
    for R in (lo.n_rows, lo.n_rows + 5, 1 << 20):
        c = oracle.inspect(lo, oracle.SPTRSV, coarsen=R)
        assert np.array_equal(c.perm, plain.perm)
        assert np.array_equal(c.level_ptr, plain.level_ptr)
        assert np.array_equal(c.records, plain.records)


@pytest.mark.parametrize("name", sorted(COARSE_MATS))
@pytest.mark.parametrize("R", [16, 50])
def test_coarse_plans_expand_to_the_trace(name, R):
    lo = COARSE_MATS[name]()
    c = oracle.inspect(lo, oracle.SPTRSV, coarsen=R)
    assert oracle.check_plan(lo, oracle.SPTRSV, c.perm, c.level_ptr, c.gs, c.records) == (0, -1)
    assert oracle.check_schedule(lo, c.perm, c.level_ptr) == (0, -1)
    # every partition holds rows of one block and one level
    lev, _ = oracle.levels(lo)
    for p in range(c.nparts):
        rows = c.perm[c.level_ptr[p]:c.level_ptr[p + 1]]
        assert len({int(r) // R for r in rows}) == 1
        assert len({int(lev[r]) for r in rows}) == 1
        assert np.all(np.diff(rows) > 0)


@pytest.mark.parametrize("k", [4, 6, 9])
def test_lap7_plane_blocks_partition_count(k):
    # 7-point lower triangle on a k^3 grid, level(x, y, z) = x + y + z.  With
    # one z-plane per block (R = k^2) the plane holds levels z .. z + 2k - 2:
    # 2k - 1 partitions per block, k (2k - 1) in total.
    lo = synth.lower_triangle(synth.laplacian_7pt(k))
    c = oracle.inspect(lo, oracle.SPTRSV, coarsen=k * k)
    assert c.nparts == k * (2 * k - 1)
    plain = oracle.inspect(lo, oracle.SPTRSV)
    assert plain.nparts == 3 * k - 2


def test_schedule_check_catches_planted_mistakes():
    lo = COARSE_MATS["lap7_5"]()
    plain = oracle.inspect(lo, oracle.SPTRSV)
    perm, pp = plain.perm.copy(), plain.level_ptr.copy()
    assert oracle.check_schedule(lo, perm, pp) == (0, -1)
    # a row moved into the partition before its own level
    q = int(pp[3])
    r = int(perm[q])
    bad = perm.copy()
    bad[q], bad[q - 1] = bad[q - 1], bad[q]
    code, row = oracle.check_schedule(lo, bad, pp)
    assert code == 1
    # two partitions merged into one (a row then shares a partition with a dependency)
    merged = np.delete(pp, 2)
    assert oracle.check_schedule(lo, perm, merged)[0] == 1
    # rows sorted by (row, level): not a schedule
    assert oracle.check_schedule(lo, np.arange(lo.n_rows, dtype=np.int32),
                                 np.array([0, lo.n_rows], np.int32))[0] == 1
    # a row listed twice is malformed
    dup = perm.copy()
    dup[1] = dup[0]
    assert oracle.check_schedule(lo, dup, pp)[0] == 2
    assert r >= 0
