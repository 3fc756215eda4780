"""The cell plan (batches of per-query ranges over a two-column grid,
vrs_build_grid) against the float64 oracle: bf16-stored and float32 tables,
L2 and IP, per-query k, edge cases of the rectangles (empty ranges, no
terms, one column, repeated values), and agreement with the batched mask
plan on the same batch."""
import numpy as np
import pytest

import gen
import oracle
from _parity import check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, BF16 = 1, 2


@pytest.fixture(scope="module")
def vrs():
    from paper_2403_15807_gb300 import build, vrs as v
    build.build()
    v.load()
    return v


def _bf16_table(n, d, seed):
    mix = gen.Mixture(d, seed=seed)
    x = gen.vectors(n, mix)
    t = torch.from_numpy(x).to(torch.bfloat16)
    xb = t.view(torch.int16).numpy().view(np.uint16).copy()
    xv = t.to(torch.float32).numpy()
    return mix, xb, xv


def _run(vrs, e, q, preds, ks, metric="l2"):
    m = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    ids, dist = e.query(torch.from_numpy(q).cuda(), preds, ks, metric=m, compute=vrs.VRS_BF16)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


def _check(x, attrs, q, preds, ks, metric, ids, dist):
    k_max = int(ks.max())
    rid, rdist, rcnt = oracle.query(x, attrs, q, preds, ks + 1, metric, k_max=k_max + 1,
                                    n_threads=16)
    check_topk(x, q, attrs, preds, ks, metric, ids, dist, rid, rdist, rcnt)


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_cells_bf16_table_matches_oracle(vrs, metric):
    """200k x 96 bf16 rows, 300 queries with their own two-range predicates
    (selectivity 1e-3 .. 0.5) and k in {1, 10, 100}; about 10 x 10 cells."""
    n, d, b = 200_000, 96, 300
    mix, xb, xv = _bf16_table(n, d, 3)
    if metric == "ip":
        # unit rows in bf16 (the stored values are the data)
        xv = xv / np.linalg.norm(xv, axis=1, keepdims=True)
        t = torch.from_numpy(xv.astype(np.float32)).to(torch.bfloat16)
        xb = t.view(torch.int16).numpy().view(np.uint16).copy()
        xv = t.to(torch.float32).numpy()
    attrs = gen.attributes(n, 2, 10_000, seed=3)
    q = gen.to_bf16_values(gen.queries(b, mix))
    preds, _ = gen.per_query_preds(b, attr_range=10_000, s_min=1e-3, s_max=0.5, seed=3)
    ks = gen.per_query_k(b, seed=3)
    with vrs.Engine(0) as e:
        vrs.vrs_load_vectors(e.h, xb, dtype=vrs.VRS_BF16, copies=1 << vrs.VRS_BF16)
        for c in range(2):
            vrs.vrs_load_attribute(e.h, c, attrs[c])
        vrs.vrs_build_grid(e.h, 0, 1)
        ids, dist = _run(vrs, e, q, preds, ks, metric)
        assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_CELLS
        cert = vrs.vrs_last_cert(e.h)
        assert sum(cert.values()) == b
        # the batched mask plan on the same batch gives the same answer
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_CELL_PLAN, 0)
        ids2, dist2 = _run(vrs, e, q, preds, ks, metric)
        assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_MASK_GEMM
    _check(xv, attrs, q, preds, ks, metric, ids, dist)
    assert np.array_equal(ids, ids2)
    assert np.array_equal(dist, dist2)


def test_cells_edge_rectangles(vrs):
    """Empty ranges (no rows), no terms (every cell fully covered), a range
    on one column only, a single value, ranges past the value domain, and an
    explicit bin count; float32 table with a bf16 copy (re-ranked from the
    float32 rows)."""
    n, d = 60_000, 64
    mix = gen.Mixture(d, seed=5)
    x = gen.vectors(n, mix)
    attrs = gen.attributes(n, 2, 1000, seed=5)
    P = gen.Pred
    preds = [
        P([0, 1], [10, 500], [10, 600]),            # empty on column 0
        P([], [], []),                              # every row
        P([1], [100], [900]),                       # column 1 only
        P([0, 1], [77, 0], [78, 1000]),             # one value of column 0
        P([0, 1], [-5000, 990], [5000, 100000]),    # past the domain
        P([0, 0, 1], [100, 150, 0], [400, 300, 50]),  # two terms on column 0
        P([1, 0], [300, 300], [700, 700]),          # terms in the other order
    ]
    b = len(preds)
    q = gen.queries(b, mix)
    ks = np.int32([5, 10, 1, 20, 3, 7, 64])
    for bins in (0, 4):
        with vrs.Engine(0) as e:
            e.load(x, attrs, dtype=vrs.VRS_F32, copies=F32 | BF16)
            vrs.vrs_build_grid(e.h, 0, 1, bins)
            ids, dist = _run(vrs, e, q, preds, ks)
            assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_CELLS
        _check(x, attrs, q, preds, ks, "l2", ids, dist)
        assert np.all(ids[0] == -1)


def test_cells_repeated_values_and_reload(vrs):
    """A column with three distinct values gives at most three bins; a
    reload of a grid column drops the grid (the mask plan runs) until it is
    built again."""
    n, d, b = 50_000, 32, 40
    mix = gen.Mixture(d, seed=6)
    x = gen.vectors(n, mix)
    attrs = np.stack([gen.attributes(n, 1, 3, seed=6)[0], gen.attributes(n, 1, 500, seed=7)[0]])
    q = gen.queries(b, mix)
    rng = np.random.default_rng(6)
    preds = []
    for _ in range(b):
        a0 = int(rng.integers(0, 3))
        lo1 = int(rng.integers(0, 400))
        preds.append(gen.Pred([0, 1], [a0, lo1], [a0 + 1, lo1 + int(rng.integers(1, 100))]))
    ks = np.full(b, 10, dtype=np.int32)
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=F32 | BF16)
        vrs.vrs_build_grid(e.h, 0, 1, 64)
        ids, dist = _run(vrs, e, q, preds, ks)
        assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_CELLS
        _check(x, attrs, q, preds, ks, "l2", ids, dist)
        vrs.vrs_load_attribute(e.h, 1, attrs[1])
        ids2, dist2 = _run(vrs, e, q, preds, ks)
        assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_MASK_GEMM
        assert np.array_equal(ids, ids2)
        vrs.vrs_build_grid(e.h, 0, 1)
        _run(vrs, e, q, preds, ks)
        assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_CELLS


def test_cells_argument_errors(vrs):
    n, d = 1000, 16
    x = np.random.default_rng(0).standard_normal((n, d)).astype(np.float32)
    attrs = gen.attributes(n, 2, 10)
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=F32)
        with pytest.raises(vrs.VrsError) as ei:   # no bf16 copy
            vrs.vrs_build_grid(e.h, 0, 1)
        assert ei.value.status == vrs.VRS_ESTATE
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=F32 | BF16)
        for c0, c1, bins in ((0, 0, 0), (0, 9, 0), (0, 1, 65), (0, 1, -1)):
            with pytest.raises(vrs.VrsError) as ei:
                vrs.vrs_build_grid(e.h, c0, c1, bins)
            assert ei.value.status == vrs.VRS_EINVAL
        with pytest.raises(vrs.VrsError) as ei:   # column 2 not loaded
            vrs.vrs_build_grid(e.h, 0, 2)
        assert ei.value.status == vrs.VRS_ESTATE
