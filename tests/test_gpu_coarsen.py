"""GPU checks of coarsened SpTRSV plans (partitions = (block of R rows, level),
the LBC-style coarsening of Sec. IV-A) and of the block-per-CTA solve.

Plans must equal the oracle's Algorithm 1 with the same coarsening bit for
bit; solves must match the oracle's forward substitution within 1e-12
normwise, across block sizes that leave ragged last blocks, one row per
block, a single block, rows whose out-of-block part spans several producer
batches, and rows whose in-block part is longer than a warp.
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


def banded_lower(n, band, seed):
    """Lower triangle with every column j in [i - band, i]: long rows."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        c = np.arange(max(0, i - band), i + 1)
        rows.append(np.full(c.size, i))
        cols.append(c)
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = rng.standard_normal(r.size) / (2.0 * band)
    v[r == c] = 1.0 + rng.random(n)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, r + 1, 1)
    return synth.CSR(n, n, np.cumsum(rp).astype(np.int32), c.astype(np.int32), v)


MATS = {
    "lap5_40": lambda: synth.lower_triangle(synth.laplacian_5pt(40)),
    "lap7_14": lambda: synth.lower_triangle(synth.laplacian_7pt(14)),
    "elast_6": lambda: synth.lower_triangle(synth.elasticity_blocks(6)),
    "st27_10": lambda: synth.lower_triangle(synth.stencil_27pt(10)),
    "powerlaw_6000": lambda: synth.lower_triangle(synth.powerlaw(6000), "unit_dominant"),
    "random_2000": lambda: synth.random_pattern(2000, 2000, 0.004, 9, diag=True, lower=True, empty_rows=0.1),
}


def plan(lo, R, **kw):
    o = ddf.ddf_opts_default(coarsen_rows=R, **kw)
    return ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), dev(lo.values), lo.n_cols, ddf.DDF_SPTRSV, o)


def solve(q, b):
    x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
    ddf.ddf_sptrsv(q, dev(b), x)
    st = ddf.ddf_get_status(q)
    assert st == 0, ddf.ddf_status_string(st)
    return x.cpu().numpy()


def relerr(y, ref):
    return np.linalg.norm(y - ref) / max(np.linalg.norm(ref), 1e-300)


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("R", [1, 61, 512, 16384])
def test_coarse_plan_and_solve(name, R):
    lo = MATS[name]()
    q = plan(lo, R)
    got = ddf.ddf_plan_export(q)
    ref = oracle.inspect(lo, oracle.SPTRSV, coarsen=R)
    assert np.array_equal(got["seq"], ref.perm)
    assert np.array_equal(got["part_ptr"], ref.level_ptr)
    assert np.array_equal(got["gs"], ref.gs)
    assert np.array_equal(got["records"], ref.records)
    assert oracle.check_schedule(lo, got["seq"], got["part_ptr"]) == (0, -1)
    st = ddf.ddf_plan_stats(q)
    assert st["blocks"] == -(-lo.n_rows // R)
    assert st["levels"] == oracle.levels(lo)[1]
    assert st["depth"] == ref.nparts
    b = synth.uniform_vector(lo.n_rows, 3)
    assert relerr(solve(q, b), oracle.sptrsv(lo, b)) <= TOL


@pytest.mark.parametrize("R", [64, 1000, 16384])
def test_long_rows(R):
    # band 700: the out-of-block part of a row spans several producer batches
    # (more than 8 points per lane at 32 lanes) and the in-block part is longer
    # than one warp pass
    lo = banded_lower(3000, 700, 4)
    q = plan(lo, R)
    b = synth.uniform_vector(lo.n_rows, 5)
    assert relerr(solve(q, b), oracle.sptrsv(lo, b)) <= TOL


def test_coarse_equals_plain_solution_and_repeats():
    lo = MATS["lap7_14"]()
    b = synth.uniform_vector(lo.n_rows, 8)
    x0 = solve(plan(lo, 0), b)
    q = plan(lo, 300)
    x1 = solve(q, b)
    x2 = solve(q, b)
    assert np.array_equal(x1, x2)                      # deterministic
    assert relerr(x1, x0) <= TOL


def test_edge_cases():
    # empty, one row, diagonal only (one level, every row its own producer work)
    for n in (0, 1, 5000):
        rp = np.arange(n + 1, dtype=np.int32)
        ci = np.arange(n, dtype=np.int32)
        v = 1.0 + np.arange(n, dtype=np.float64)
        lo = synth.CSR(n, n, rp, ci, v)
        q = plan(lo, 128)
        b = synth.uniform_vector(n, 1)
        x = solve(q, b) if n else np.zeros(0)
        assert np.allclose(x, b / v, rtol=1e-15, atol=0)
    # a chain: each row depends on the previous one (depth n, one row per level)
    n = 3000
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([1] + [2] * (n - 1))
    ci = np.concatenate([[0]] + [[i - 1, i] for i in range(1, n)]).astype(np.int32)
    v = np.tile([-0.5, 1.0], n)[1:].astype(np.float64)
    lo = synth.CSR(n, n, rp, ci, v)
    for R in (7, 1024, 16384):
        q = plan(lo, R)
        b = synth.uniform_vector(n, 2)
        assert relerr(solve(q, b), oracle.sptrsv(lo, b)) <= TOL


@pytest.mark.parametrize("vdt", [ddf.DDF_F32, ddf.DDF_BF16])
def test_coarse_refinement(vdt):
    lo = MATS["elast_6"]()
    q = plan(lo, 200, store_dtype=vdt)
    b = synth.uniform_vector(lo.n_rows, 4)
    x = torch.zeros(lo.n_rows, dtype=torch.float64, device="cuda")
    st, iters, rel = ddf.ddf_sptrsv_refine(q, dev(b), x, tol=1e-12, max_iter=30)
    assert st == 0 and rel <= 1e-12
    r = b - oracle.spmv(lo, x.cpu().numpy())
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)


def test_coarse_multi_rhs_and_update_values():
    lo = MATS["powerlaw_6000"]()
    q = ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), None, lo.n_cols, ddf.DDF_SPTRSV,
                        ddf.ddf_opts_default(coarsen_rows=500))
    ddf.ddf_update_values(q, dev(lo.values))
    nrhs = 5
    B = np.random.default_rng(1).uniform(-1, 1, (lo.n_rows, nrhs))
    X = torch.zeros((lo.n_rows, nrhs), dtype=torch.float64, device="cuda")
    ddf.ddf_sptrsm(q, dev(B), X, nrhs)
    assert ddf.ddf_get_status(q) == 0
    Xh = X.cpu().numpy()
    for k in range(nrhs):
        assert relerr(Xh[:, k], oracle.sptrsv(lo, B[:, k])) <= TOL
    assert relerr(solve(q, B[:, 0]), oracle.sptrsv(lo, B[:, 0])) <= TOL
