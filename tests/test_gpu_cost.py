"""GPU recalibration of Eq. 1 (ddf_tune_cost) against the CPU oracle.

ddf_tune_cost mines plans with candidate weight sets for the cost model of
Sec. III-C, times the executor on each and returns the fastest set.  The
weights it returns must be one of the candidates, and a plan mined with them
must equal the oracle's Algorithm 1 with the same weights, bit for bit, and
compute what the oracle computes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2111_12243_gb300 as ddf
import synth

pytestmark = pytest.mark.gpu

CANDIDATES = [(8, 32, 4), (8, 8, 4), (8, 128, 4), (8, 32, 1), (8, 32, 16), (1, 3, 1)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_12243_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name,kind", [("st27_11", 1), ("lap7_12", 1), ("elast_5", 2), ("powerlaw_3000", 2)])
def test_tuned_weights_give_oracle_plans(name, kind):
    a = {"st27_11": lambda: synth.stencil_27pt(11), "lap7_12": lambda: synth.laplacian_7pt(12),
         "elast_5": lambda: synth.elasticity_blocks(5), "powerlaw_3000": lambda: synth.powerlaw(3000)}[name]()
    if kind == 2:
        a = synth.lower_triangle(a, "unit_dominant") if name.startswith("powerlaw") else synth.lower_triangle(a)
    o, pick = ddf.ddf_tune_cost(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, kind,
                                ddf.ddf_opts_default(window_t=64))
    assert 0 <= pick < len(CANDIDATES)
    w = (o.w_op, o.w_codelet, o.w_index)
    assert w == CANDIDATES[pick]
    assert o.window_t == 64                      # the other options are kept
    p = ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, kind, o)
    got = ddf.ddf_plan_export(p)
    ref = oracle.inspect(a, oracle.SPMV if kind == 1 else oracle.SPTRSV, t=64, weights=w)
    assert np.array_equal(got["records"], ref.records)
    x = synth.uniform_vector(a.n_cols, 4)
    y = torch.empty(a.n_rows, dtype=torch.float64, device="cuda")
    if kind == 1:
        ddf.ddf_spmv(p, dev(x), y)
        r = oracle.spmv(a, x)
    else:
        ddf.ddf_sptrsv(p, dev(x), y)
        r = oracle.sptrsv(a, x)
    assert np.linalg.norm(y.cpu().numpy() - r) <= 1e-12 * np.linalg.norm(r)


def test_tune_cost_argument_errors():
    a = synth.laplacian_7pt(6)
    with pytest.raises(ValueError):
        ddf.ddf_tune_cost(dev(a.rowptr), dev(a.colidx), None, a.n_cols, 1)
    with pytest.raises(ddf.DDFError):
        ddf.ddf_tune_cost(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, 7)
