"""GPU checks of the batched and multi-RHS forms against the FP64 oracle.

A batch is inspected as its block-diagonal matrix, so its plan must equal the
oracle's Algorithm 1 on that matrix bit for bit.  Multi-RHS results are
checked column by column against the oracle's single-vector SpMV and forward
substitution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2111_12243_gb300 as ddf
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12
U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_12243_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def block_diag(mats):
    rp = [np.zeros(1, np.int64)]
    ci, va = [], []
    r = c = z = 0
    for m in mats:
        rp.append(m.rowptr[1:].astype(np.int64) + z)
        ci.append(m.colidx.astype(np.int64) + c)
        va.append(m.values)
        r += m.n_rows
        c += m.n_cols
        z += m.nnz
    return synth.CSR(r, c, np.concatenate(rp).astype(np.int32), np.concatenate(ci).astype(np.int32),
                     np.concatenate(va))


@pytest.fixture(scope="module")
def small_batch():
    kinds = ["2d", "3d", "powerlaw", "3d", "2d", "powerlaw", "2d"]
    sizes = [1000, 1500, 1200, 2500, 900, 3000, 1100]
    return [synth.batch_member(n, k, 100 + i) for i, (n, k) in enumerate(zip(sizes, kinds))]


def batch_plan(mats, kind, on_device=True, **opts):
    tup = [((dev(m.rowptr), dev(m.colidx), dev(m.values)) if on_device else (m.rowptr, m.colidx, m.values))
           + (m.n_cols,) for m in mats]
    return ddf.ddf_inspect_batch(tup, kind, ddf.ddf_opts_default(**opts))


@pytest.mark.parametrize("on_device", [True, False])
def test_batch_plans_equal_block_diagonal_inspection(small_batch, on_device):
    lows = [synth.lower_triangle(m) for m in small_batch]
    for mats, kind, okind in ((small_batch, ddf.DDF_SPMV, oracle.SPMV), (lows, ddf.DDF_SPTRSV, oracle.SPTRSV)):
        p = batch_plan(mats, kind, on_device)
        got = ddf.ddf_plan_export(p)
        bd = block_diag(mats)
        ref = oracle.inspect(bd, okind)
        assert np.array_equal(got["seq"], ref.perm)
        assert np.array_equal(got["part_ptr"], ref.level_ptr)
        assert np.array_equal(got["records"], ref.records)
        assert oracle.check_plan(bd, okind, got["seq"], got["part_ptr"], got["gs"], got["records"]) == (0, -1)


# nrhs 4, 8, 16, 32 run the vector executors (2 right-hand sides per lane,
# 2 .. 16 lanes per row of X), 1 and 5 the scalar ones
@pytest.mark.parametrize("nrhs", [1, 4, 5, 8, 16, 32])
def test_spmm_and_sptrsm_f64(small_batch, nrhs):
    bd = block_diag(small_batch)
    lo = block_diag([synth.lower_triangle(m) for m in small_batch])
    rng = np.random.default_rng(nrhs)
    X = rng.uniform(-1, 1, (bd.n_cols, nrhs))
    B = rng.uniform(-1, 1, (lo.n_rows, nrhs))
    p = batch_plan(small_batch, ddf.DDF_SPMV)
    Y = torch.full((bd.n_rows, nrhs), float("nan"), dtype=torch.float64, device="cuda")
    ddf.ddf_spmm(p, dev(X), Y, nrhs)
    Yh = Y.cpu().numpy()
    q = batch_plan([synth.lower_triangle(m) for m in small_batch], ddf.DDF_SPTRSV)
    Xs = torch.zeros((lo.n_rows, nrhs), dtype=torch.float64, device="cuda")
    ddf.ddf_sptrsm(q, dev(B), Xs, nrhs)
    assert ddf.ddf_get_status(q) == 0
    Xh = Xs.cpu().numpy()
    for k in range(nrhs):
        ry = oracle.spmv(bd, X[:, k])
        assert np.linalg.norm(Yh[:, k] - ry) <= TOL * np.linalg.norm(ry)
        rx = oracle.sptrsv(lo, B[:, k])
        assert np.linalg.norm(Xh[:, k] - rx) <= TOL * np.linalg.norm(rx)


def f32_block(a, shift):
    """a on the device, starting `shift` floats past a 16-byte boundary."""
    flat = torch.zeros(a.size + 4, dtype=torch.float32, device="cuda")
    v = flat[shift:shift + a.size].view(a.shape)
    v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return v


# nrhs 8, 16, 32 on aligned blocks run the vector executors (4 right-hand
# sides per lane); shifted blocks and nrhs 3 the scalar ones
@pytest.mark.parametrize("nrhs,shift", [(32, 0), (16, 0), (8, 0), (32, 1), (3, 0)])
def test_spmm_and_sptrsm_f32(small_batch, nrhs, shift):
    bd = block_diag(small_batch)
    lo = block_diag([synth.lower_triangle(m) for m in small_batch])
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, (bd.n_cols, nrhs)).astype(np.float32)
    B = rng.uniform(-1, 1, (lo.n_rows, nrhs)).astype(np.float32)
    p = batch_plan(small_batch, ddf.DDF_SPMV, store_dtype=ddf.DDF_F32)
    Y = f32_block(np.zeros((bd.n_rows, nrhs), np.float32), shift)
    ddf.ddf_spmm(p, f32_block(X, shift), Y, nrhs)
    Yh = Y.double().cpu().numpy()
    y2 = Y.clone()
    ddf.ddf_spmm(p, f32_block(X, shift), Y, nrhs)
    assert torch.equal(Y, y2)                           # fixed summation order
    absa = synth.CSR(bd.n_rows, bd.n_cols, bd.rowptr, bd.colidx, np.abs(bd.values))
    k_row = np.maximum(np.diff(bd.rowptr), 1)
    for k in range(0, nrhs, 7):
        xk = X[:, k].astype(np.float64)
        ref = oracle.spmv(bd, xk)                       # batch values are exact in FP32
        bound = 2 * k_row * U32 * oracle.spmv(absa, np.abs(xk)) + 1e-30
        assert np.all(np.abs(Yh[:, k] - ref) <= bound)
    q = batch_plan([synth.lower_triangle(m) for m in small_batch], ddf.DDF_SPTRSV, store_dtype=ddf.DDF_F32)
    Xs = f32_block(np.zeros((lo.n_rows, nrhs), np.float32), shift)
    ddf.ddf_sptrsm(q, f32_block(B, shift), Xs, nrhs)
    assert ddf.ddf_get_status(q) == 0
    Xh = Xs.double().cpu().numpy()
    x2 = Xs.clone()
    ddf.ddf_sptrsm(q, f32_block(B, shift), Xs, nrhs)
    assert torch.equal(Xs, x2)
    for k in range(0, nrhs, 5):
        bk = B[:, k].astype(np.float64)
        r = bk - oracle.spmv(lo, Xh[:, k])
        assert np.linalg.norm(r) <= 1e-5 * np.linalg.norm(bk)


def test_tune_and_graph_capture(small_batch):
    nrhs = 32
    bd = block_diag(small_batch)
    lows = [synth.lower_triangle(m) for m in small_batch]
    lo = block_diag(lows)
    rng = np.random.default_rng(3)
    X = dev(rng.uniform(-1, 1, (bd.n_cols, nrhs)).astype(np.float32))
    B = dev(rng.uniform(-1, 1, (lo.n_rows, nrhs)).astype(np.float32))
    p = batch_plan(small_batch, ddf.DDF_SPMV, store_dtype=ddf.DDF_F32)
    q = batch_plan(lows, ddf.DDF_SPTRSV, store_dtype=ddf.DDF_F32)
    Y = torch.empty((bd.n_rows, nrhs), dtype=torch.float32, device="cuda")
    Xs = torch.empty((lo.n_rows, nrhs), dtype=torch.float32, device="cuda")
    assert ddf.ddf_tune(p, X, Y, nrhs) in (64, 128, 256, 512, 1024, 2048)
    assert ddf.ddf_tune(q, B, Xs, nrhs) in (1, 2, 4, 8)
    ddf.ddf_spmm(p, X, Y, nrhs)
    ddf.ddf_sptrsm(q, B, Xs, nrhs)
    torch.cuda.synchronize()
    y0, x0 = Y.clone(), Xs.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ddf.ddf_spmm(p, X, Y, nrhs, stream=s)
            ddf.ddf_sptrsm(q, B, Xs, nrhs, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        Y.zero_()
        Xs.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(Y, y0)
        assert torch.equal(Xs, x0)
    assert ddf.ddf_get_status(q) == 0


def test_multi_rhs_argument_errors(small_batch):
    p = batch_plan(small_batch[:2], ddf.DDF_SPMV)
    n = p.n_rows
    X = torch.zeros((p.n_cols, 33), dtype=torch.float64, device="cuda")
    Y = torch.zeros((n, 33), dtype=torch.float64, device="cuda")
    with pytest.raises(ddf.DDFError):
        ddf.ddf_spmm(p, X, Y, 33)
    Xf = torch.zeros((p.n_cols, 4), dtype=torch.float32, device="cuda")
    Yf = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_spmm(p, Xf, Yf, 4)                         # FP64-only plan
    assert e.value.status == 1
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_sptrsm(p, Xf, Yf, 4)
    assert e.value.status in (1, 8)
    bad = synth.CSR(2, 3, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.ones(2))
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_inspect_batch([(bad.rowptr, bad.colidx, bad.values, 3)], ddf.DDF_SPTRSV)
    assert e.value.status == 2


@pytest.mark.parametrize("nrhs", [32, 3])
def test_sptrsm_wait_times_out_and_recovers(nrhs):
    # Point the first off-diagonal entry of a row r at a row d that itself
    # reads r: r waits for d and d for r, so the bounded waits must run out,
    # latch DDF_ERR_TIMEOUT, leave NaN in X and the context usable.  nrhs 32
    # runs the 16-byte lane layout, 3 the one-element layout.
    lo = synth.random_pattern(3000, 3000, 0.003, 17, diag=True, lower=True)
    o = ddf.ddf_opts_default(store_dtype=ddf.DDF_F32, spin_cap_ns=50_000_000)
    q = ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), dev(lo.values), lo.n_cols, ddf.DDF_SPTRSV, o)
    exp = ddf.ddf_plan_export(q)
    seq, gs = exp["seq"], exp["gs"]
    offl = np.diff(lo.rowptr) - 1
    rows_of = np.repeat(np.arange(lo.n_rows), np.diff(lo.rowptr))
    target = None
    for pos in range(lo.n_rows):
        row = int(seq[pos])
        if offl[row] < 1:
            continue
        deps = rows_of[(lo.colidx == row) & (rows_of != row)]
        if deps.size:
            target = (int(gs[pos]), int(deps[0]))
            break
    assert target is not None
    ddf.ddf_debug_set_dependency(q, *target)
    B = np.random.default_rng(2).uniform(-1, 1, (lo.n_rows, nrhs)).astype(np.float32)
    X = torch.zeros((lo.n_rows, nrhs), dtype=torch.float32, device="cuda")
    ddf.ddf_sptrsm(q, dev(B), X, nrhs)
    assert ddf.ddf_get_status(q) == 11
    assert torch.isnan(X).any()
    # the device is still usable: a clean plan solves to the FP32 bound
    q2 = ddf.ddf_inspect(dev(lo.rowptr), dev(lo.colidx), dev(lo.values), lo.n_cols, ddf.DDF_SPTRSV,
                         ddf.ddf_opts_default(store_dtype=ddf.DDF_F32))
    ddf.ddf_sptrsm(q2, dev(B), X, nrhs)
    assert ddf.ddf_get_status(q2) == 0
    Xh = X.double().cpu().numpy()
    for k in range(0, nrhs, 7):
        bk = B[:, k].astype(np.float64)
        assert np.linalg.norm(bk - oracle.spmv(lo, Xh[:, k])) <= 1e-5 * np.linalg.norm(bk)


@pytest.mark.parametrize("nrhs,dt", [(32, torch.float32), (3, torch.float32), (8, torch.float64)])
def test_batch_run_equals_separate_calls(small_batch, nrhs, dt):
    # the one-launch form runs the same row computations as ddf_spmm and
    # ddf_sptrsm, so its results are bit-identical; also recorded in a graph
    lows = [synth.lower_triangle(m) for m in small_batch]
    opts = {"store_dtype": ddf.DDF_F32} if dt == torch.float32 else {}
    p = batch_plan(small_batch, ddf.DDF_SPMV, **opts)
    q = batch_plan(lows, ddf.DDF_SPTRSV, **opts)
    rng = np.random.default_rng(nrhs)
    X = torch.from_numpy(rng.uniform(-1, 1, (p.n_cols, nrhs))).to(dt).cuda()
    B = torch.from_numpy(rng.uniform(-1, 1, (q.n_rows, nrhs))).to(dt).cuda()
    Y1 = torch.empty((p.n_rows, nrhs), dtype=dt, device="cuda")
    X1 = torch.empty((q.n_rows, nrhs), dtype=dt, device="cuda")
    ddf.ddf_spmm(p, X, Y1, nrhs)
    ddf.ddf_sptrsm(q, B, X1, nrhs)
    Y2 = torch.full_like(Y1, float("nan"))
    X2 = torch.full_like(X1, float("nan"))
    ddf.ddf_batch_run(p, X, Y2, q, B, X2, nrhs)
    torch.cuda.synchronize()
    assert ddf.ddf_get_status(q) == 0
    assert torch.equal(Y1, Y2) and torch.equal(X1, X2)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ddf.ddf_batch_run(p, X, Y2, q, B, X2, nrhs, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        Y2.zero_()
        X2.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(Y1, Y2) and torch.equal(X1, X2)
    assert ddf.ddf_get_status(q) == 0


def test_batch_run_argument_errors(small_batch):
    lows = [synth.lower_triangle(m) for m in small_batch[:2]]
    p = batch_plan(small_batch[:2], ddf.DDF_SPMV)
    q = batch_plan(lows, ddf.DDF_SPTRSV)
    X = torch.zeros((p.n_cols, 4), dtype=torch.float64, device="cuda")
    Y = torch.zeros((p.n_rows, 4), dtype=torch.float64, device="cuda")
    B = torch.zeros((q.n_rows, 4), dtype=torch.float64, device="cuda")
    Xs = torch.zeros((q.n_rows, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_batch_run(q, X, Y, p, B, Xs, 4)           # plans swapped
    assert e.value.status == 8
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_batch_run(p, X, Y, q, B, B, 4)            # Xs overlaps B
    assert e.value.status == 1
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_batch_run(p, X, Y, q, B, Y, 4)            # Xs overlaps Y
    assert e.value.status == 1
    ddf.ddf_batch_run(p, X, Y, q, B, Xs, 4)
    assert ddf.ddf_get_status(q) == 0


def long_row_lower(n=2500, seed=21):
    """A diagonally dominant lower triangle whose every 17th row reads the
    previous 70 .. 1100 rows (rows longer than a solve segment), the rest a
    band of 3."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        if i % 17 == 0 and i > 70:
            k = int(min(i, rng.integers(70, 1100)))
            cols = np.sort(rng.choice(i, k, replace=False))
        else:
            cols = np.arange(max(0, i - 3), i)
        rows.append(np.concatenate([cols, [i]]).astype(np.int32))
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.concatenate(rows)
    v = rng.standard_normal(ci.size) * 0.01
    v[rp[1:] - 1] = 1.0 + np.abs(rng.standard_normal(n))
    return synth.CSR(n, n, rp.astype(np.int32), ci, v)


@pytest.mark.parametrize("nrhs,dt", [(32, torch.float32), (5, torch.float64), (16, torch.float64)])
def test_sptrsm_long_rows_in_segments(small_batch, nrhs, dt):
    # a batch whose rows of more than 64 points are solved in segments on
    # several warps, their partial sums added in a fixed order: results
    # within the oracle's tolerance and the same on every call
    lows = [long_row_lower(), synth.lower_triangle(small_batch[2]), long_row_lower(1800, 22)]
    lo = block_diag(lows)
    opts = {"store_dtype": ddf.DDF_F32} if dt == torch.float32 else {}
    q = batch_plan(lows, ddf.DDF_SPTRSV, **opts)
    B = np.random.default_rng(nrhs).uniform(-1, 1, (lo.n_rows, nrhs))
    Bd = torch.from_numpy(B).to(dt).cuda()
    Xs = torch.empty((lo.n_rows, nrhs), dtype=dt, device="cuda")
    ddf.ddf_sptrsm(q, Bd, Xs, nrhs)
    x0 = Xs.clone()
    for _ in range(2):
        ddf.ddf_sptrsm(q, Bd, Xs, nrhs)
        assert torch.equal(Xs, x0)
    assert ddf.ddf_get_status(q) == 0
    Xh = Xs.double().cpu().numpy()
    for k in range(nrhs):
        bk = Bd[:, k].double().cpu().numpy()
        rx = oracle.sptrsv(lo, bk)
        tol = 1e-5 if dt == torch.float32 else TOL
        assert np.linalg.norm(Xh[:, k] - rx) <= tol * np.linalg.norm(rx)
