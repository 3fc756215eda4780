"""GPU parity of the filtered range search (sigma_eps with eps a bound on the
score, Sec. 3) against the float64 oracle.

The library decides with exact FP32 scores, the oracle with float64 ones:
the result sets must agree except for rows whose float64 score lies within
1e-5 (relative to ||q||^2 + ||x||^2) of the bound, and every reported score
must match the oracle's within the same tolerance.
"""
import numpy as np
import pytest

import gen
import oracle
from _parity import check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def vrs():
    from paper_2403_15807_gb300 import build, vrs as v
    build.build()
    v.load()
    return v


def _check(x, attrs, q, pred, eps, metric, offs, ids, dist):
    ref = oracle.range_query(x, attrs, q, pred, eps, metric)
    xn = oracle.sqnorm(x)
    qn = oracle.sqnorm(q)
    assert offs[0] == 0 and np.all(np.diff(offs) >= 0)
    for i, (rid, rsc) in enumerate(ref):
        gid = ids[offs[i]:offs[i + 1]]
        gsc = dist[offs[i]:offs[i + 1]].astype(np.float64)
        assert len(np.unique(gid)) == len(gid), f"q{i}: duplicate rows"
        # every returned row satisfies the predicate
        for c, lo, hi in zip(pred.cols, pred.lo, pred.hi):
            assert np.all((attrs[c, gid] >= lo) & (attrs[c, gid] < hi))
        gs, rs = set(gid.tolist()), set(rid.tolist())
        # rows on one side only: their exact score must sit on the bound
        for r in gs ^ rs:
            s = oracle.pair_dist(x, q, np.int64([i]), np.int64([r]), metric)[0]
            assert abs(s - eps) <= TOL * (qn[i] + xn[r]) + 1e-30, (i, r, s, eps)
        # reported scores against the oracle's
        ref_of = dict(zip(rid.tolist(), rsc.tolist()))
        for r, s in zip(gid.tolist(), gsc.tolist()):
            exact = ref_of.get(r)
            if exact is None:
                exact = oracle.pair_dist(x, q, np.int64([i]), np.int64([r]), metric)[0]
            assert abs(s - exact) <= TOL * (qn[i] + xn[r]) + 1e-30, (i, r, s, exact)
    return [len(r) for r, _ in ref]


def _eps_from_rank(x, attrs, q, pred, metric, rank):
    """A bound between the oracle's rank-th and (rank+1)-th score of query 0."""
    _, dist, _ = oracle.query(x, attrs, q[:1], [pred], rank + 1, metric)
    return float(0.5 * (dist[0, rank - 1] + dist[0, rank]))


@pytest.mark.parametrize("on_device", [True, False])
@pytest.mark.parametrize("n,d,b,s,metric,rank", [
    (100_003, 128, 16, 0.1, "l2", 50),
    (50_000, 144, 5, 0.3, "ip", 30),
    (20_000, 64, 64, 1.0, "l2", 20),
    (30_001, 96, 1, 0.5, "ip", 200),
])
def test_range_matches_oracle(vrs, on_device, n, d, b, s, metric, rank):
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=n % 89 + b)
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, 1, 1000, seed=d)
    pred = gen.pred_less_than(int(s * 1000)) if s < 1 else gen.pred_all()
    eps = _eps_from_rank(x, attrs, q, pred, metric, rank)
    m = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    with vrs.Engine(0) as e:
        e.load(x, attrs)
        qq = torch.from_numpy(q).cuda() if on_device else q
        offs, ids, dist = e.range_query(qq, pred, eps, metric=m)
        if on_device:
            torch.cuda.synchronize()
            ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    counts = _check(x, attrs, q, pred, eps, metric, offs, ids, dist)
    assert counts[0] == rank


def test_range_edge_bounds_and_capacity(vrs):
    """No result (L2 bound below zero, or an empty selection), every
    selected row (infinite bound), and a capacity too small for the results
    (ESIZE with the offsets filled, then the retry the binding makes)."""
    n, d, b = 12_345, 32, 3
    mix = gen.Mixture(d, seed=3)
    x = gen.vectors(n, mix)
    q = gen.queries(b, mix)
    attrs = gen.attributes(n, 1, 1000, seed=3)
    pred = gen.pred_less_than(400)
    sel = np.flatnonzero(attrs[0] < 400)
    with vrs.Engine(0) as e:
        e.load(x, attrs)
        offs, ids, dist = e.range_query(q, pred, -1.0)
        assert np.all(offs == 0) and len(ids) == 0
        offs, ids, _ = e.range_query(q, gen.Pred([0], [2000], [3000]), np.inf)
        assert np.all(offs == 0)
        offs, ids, dist = e.range_query(q, pred, np.inf)
        for i in range(b):
            assert np.array_equal(np.sort(ids[offs[i]:offs[i + 1]]), sel)
        # the raw call with a small capacity reports the size needed
        import ctypes as C
        parr, keep = vrs.make_preds([pred])
        o2 = np.zeros(b + 1, dtype=np.int64)
        i2 = np.empty(4, dtype=np.int64)
        d2 = np.empty(4, dtype=np.float32)
        st = vrs.load().vrs_range_query(e.h, q.ctypes.data_as(C.c_void_p), b, d, parr,
                                        C.c_float(np.inf), vrs.VRS_L2, 4,
                                        o2.ctypes.data_as(C.c_void_p),
                                        i2.ctypes.data_as(C.c_void_p),
                                        d2.ctypes.data_as(C.c_void_p), 0, None)
        assert st == vrs.VRS_ESIZE and o2[-1] == b * sel.size
        # a small first guess is retried at the reported size
        eps = _eps_from_rank(x, attrs, q, pred, "l2", 40)
        offs, ids, dist = e.range_query(q, pred, eps, cap=8)
        # and a top-k query afterwards still sees a clean state
        tid, tdist = e.query(q, [pred], np.int32([10]))
    _check(x, attrs, q, pred, eps, "l2", offs, ids, dist)
    kk = np.full(b, 10, np.int32)
    rid, rdist, rcnt = oracle.query(x, attrs, q, [pred], kk + 1, "l2")
    check_topk(x, q, attrs, [pred], kk, "l2", tid, tdist, rid, rdist, rcnt)
