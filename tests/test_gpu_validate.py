"""Plan validation on the GPU (ddf_plan_validate, and ddf_plan_load, which runs
it).  Plans the inspector builds pass; a plan whose SpTRSV copy names a row
that is not solved earlier fails with DDF_ERR_NOT_LOWER; serialised buffers
altered so that the checksum still matches are rejected at load time with the
status of the check that caught them, before any executor can run them."""
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2111_12243_gb300 as ddf
import synth

pytestmark = pytest.mark.gpu

OUT_OF_RANGE, NOT_LOWER = 4, 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_12243_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def inspect(a, kind, **opts):
    return ddf.ddf_inspect(dev(a.rowptr), dev(a.colidx), dev(a.values), a.n_cols, kind,
                           ddf.ddf_opts_default(**opts))


def fnv1a(b: bytes) -> int:
    # 64-bit FNV-1a (Fowler, Noll, Vo): the checksum the plan buffer ends with
    h = 0xcbf29ce484222325
    for c in b:
        h = ((h ^ c) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def reseal(buf: bytearray) -> bytes:
    body = bytes(buf[:-8])
    return body + struct.pack("<Q", fnv1a(body))


MATS = {
    "lap5_40": lambda: synth.laplacian_5pt(40),
    "lap7_14": lambda: synth.laplacian_7pt(14),
    "st27_10": lambda: synth.stencil_27pt(10),
    "elast_5": lambda: synth.elasticity_blocks(5),
    "powerlaw_4000": lambda: synth.powerlaw(4000, 3),
    "random_2000": lambda: synth.random_pattern(2000, 2000, 0.004, 5, diag=True),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("coarsen", [0, 64])
def test_inspected_plans_pass(name, coarsen):
    a = MATS[name]()
    lo = synth.lower_triangle(a)
    if coarsen == 0:
        assert ddf.ddf_plan_validate(inspect(a, ddf.DDF_SPMV)) == 0
        assert ddf.ddf_plan_validate(inspect(a, ddf.DDF_SPMV, store_dtype=ddf.DDF_F32)) == 0
    q = inspect(lo, ddf.DDF_SPTRSV, coarsen_rows=coarsen)
    assert ddf.ddf_plan_validate(q) == 0
    if coarsen:
        assert ddf.ddf_plan_stats(q)["blocks"] > 0


def test_batched_and_empty_plans_pass():
    mats = [synth.batch_member(n, k, 40 + i) for i, (n, k) in enumerate([(700, "2d"), (1600, "3d"), (1000, "powerlaw")])]
    for kind, ms in ((ddf.DDF_SPMV, mats), (ddf.DDF_SPTRSV, [synth.lower_triangle(m) for m in mats])):
        p = ddf.ddf_inspect_batch([(dev(m.rowptr), dev(m.colidx), dev(m.values), m.n_cols) for m in ms], kind)
        assert ddf.ddf_plan_validate(p) == 0
    e = synth.CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    for kind in (ddf.DDF_SPMV, ddf.DDF_SPTRSV):
        assert ddf.ddf_plan_validate(ddf.ddf_inspect(e.rowptr, e.colidx, e.values, 0, kind)) == 0


def psc2_entry(lo, q):
    """(position k in the plan's level-ordered copy, row, earliest later row
    that reads it) for the first off-diagonal entry of a PSC II row."""
    exp = ddf.ddf_plan_export(q)
    rec, seq, gs = exp["records"], exp["seq"], exp["gs"]
    offl = np.diff(lo.rowptr) - 1
    rows_of = np.repeat(np.arange(lo.n_rows), np.diff(lo.rowptr))
    for r in rec[rec[:, 1] == 2]:
        for pos in range(r[2], r[2] + r[3]):
            row = int(seq[pos])
            if offl[row] < 1:
                continue
            later = rows_of[(lo.colidx == row) & (rows_of != row)]
            if later.size:
                return int(gs[pos]), row, int(later[0])
    return None


@pytest.mark.parametrize("coarsen", [0, 256])
def test_planted_dependency_fails_and_is_caught_at_load(coarsen):
    lo = synth.random_pattern(3000, 3000, 0.003, 17, diag=True, lower=True)
    q = inspect(lo, ddf.DDF_SPTRSV, coarsen_rows=coarsen)
    assert ddf.ddf_plan_validate(q) == 0
    k, row, later = psc2_entry(lo, q)
    ddf.ddf_debug_set_dependency(q, k, later)      # row now reads a row solved after it
    assert ddf.ddf_plan_validate(q) == NOT_LOWER
    # the altered plan saves with a valid checksum, and load refuses it
    data = ddf.ddf_plan_save(q)
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_plan_load(data, lo.n_rows, lo.n_cols, ddf.DDF_SPTRSV)
    assert e.value.status == NOT_LOWER


def test_resealed_column_out_of_range_is_rejected():
    # A PSC II row of a SpMV plan reads its columns from the plan's copy of
    # colidx; pointing one past n_cols and recomputing the checksum must fail
    # validation on load with DDF_ERR_OUT_OF_RANGE.
    a = synth.powerlaw(3000, 11)
    p = inspect(a, ddf.DDF_SPMV)
    exp = ddf.ddf_plan_export(p)
    rec = exp["records"]
    psc2 = rec[rec[:, 1] == 2]
    assert psc2.shape[0] > 0
    q0 = int(psc2[0][2])                           # the codelet's first position
    row = int(exp["seq"][q0])
    assert a.rowptr[row + 1] > a.rowptr[row]
    data = bytearray(ddf.ddf_plan_save(p))
    at = bytes(data).find(a.colidx.astype(np.int32).tobytes())
    assert at > 0 and at % 8 == 0
    good = reseal(data)
    assert good == bytes(data)                     # the same checksum as the library's
    assert ddf.ddf_plan_validate(ddf.ddf_plan_load(good, a.n_rows, a.n_cols, ddf.DDF_SPMV)) == 0
    k = at + 4 * int(exp["gs"][q0])
    data[k:k + 4] = struct.pack("<i", a.n_cols + 7)
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_plan_load(reseal(data), a.n_rows, a.n_cols, ddf.DDF_SPMV)
    assert e.value.status == OUT_OF_RANGE
    # an altered checksum alone is still a plain DDF_ERR_ARG
    bad = bytearray(good)
    bad[-1] ^= 1
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_plan_load(bytes(bad), a.n_rows, a.n_cols, ddf.DDF_SPMV)
    assert e.value.status == 1
