"""GPU parity of the vector join (queries drawn from a relation by its own
predicate, each with the filtered top-k of the loaded rows) against the
oracle's composition: the selected query ids exactly, the top-k under the
tolerance rule of the top-k tests."""
import numpy as np
import pytest

import gen
import oracle
from _parity import check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL = (1 << 0) | (1 << 1) | (1 << 2)


@pytest.fixture(scope="module")
def vrs():
    from paper_2403_15807_gb300 import build, vrs as v
    build.build()
    v.load()
    return v


def _check(x, attrs, qrel, qattrs, qpred, rpred, k, metric, qids, ids, dist):
    rq, _, _ = oracle.join_topk(x, attrs, qrel, qattrs, qpred, rpred, k, metric)
    assert np.array_equal(qids, rq)
    if rq.size == 0:
        return 0
    q = qrel[rq]
    kk = np.full(rq.size, k, np.int32)
    rid, rdist, rcnt = oracle.query(x, attrs, q, [rpred], kk + 1, metric, n_threads=8)
    check_topk(x, q, attrs, [rpred], kk, metric, ids, dist, rid, rdist, rcnt)
    return rq.size


@pytest.mark.parametrize("on_device", [True, False])
@pytest.mark.parametrize("n,d,m,k,qs,rs,metric,compute", [
    (50_000, 64, 3_000, 10, 0.1, 0.2, "l2", "f32"),      # 300 query rows, GEMV plan
    (20_000, 96, 10_001, 5, 0.5, 0.5, "l2", "bf16"),     # ~5000 query rows: two batches
    (30_000, 128, 777, 10, 1.0, 0.3, "ip", "bf16"),      # every query row
])
def test_join_matches_oracle(vrs, on_device, n, d, m, k, qs, rs, metric, compute):
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=m % 97)
    x = gen.vectors(n, mix, unit=unit)
    attrs = gen.attributes(n, 1, 1000, seed=d)
    qrel = gen.queries(m, mix, unit=unit)
    qattrs = gen.attributes(m, 2, 1000, seed=m)
    qpred = gen.Pred([1], [0], [int(qs * 1000)]) if qs < 1 else gen.pred_all()
    rpred = gen.pred_less_than(int(rs * 1000))
    cd = {"f32": vrs.VRS_F32, "bf16": vrs.VRS_BF16}[compute]
    mt = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=ALL)
        if on_device:
            qids, ids, dist = e.join_topk(torch.from_numpy(qrel).cuda(),
                                          torch.from_numpy(qattrs).cuda(), qpred, rpred, k,
                                          metric=mt, compute=cd)
            torch.cuda.synchronize()
            ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
        else:
            qids, ids, dist = e.join_topk(qrel, qattrs, qpred, rpred, k, metric=mt, compute=cd)
    nq = _check(x, attrs, qrel, qattrs, qpred, rpred, k, metric, qids, ids, dist)
    assert nq > 0


def test_join_empty_and_capacity(vrs):
    n, d, m = 5_000, 32, 400
    mix = gen.Mixture(d, seed=5)
    x = gen.vectors(n, mix)
    attrs = gen.attributes(n, 1, 100, seed=5)
    qrel = gen.queries(m, mix)
    qattrs = gen.attributes(m, 1, 100, seed=6)
    rpred = gen.pred_less_than(50)
    with vrs.Engine(0) as e:
        e.load(x, attrs)
        qids, ids, _ = e.join_topk(qrel, qattrs, gen.Pred([0], [200], [300]), rpred, 4)
        assert qids.size == 0 and ids.shape[0] == 0
        with pytest.raises(vrs.VrsError) as ei:
            e.join_topk(qrel, qattrs, gen.pred_less_than(50), rpred, 4, cap=3)
        assert ei.value.status == vrs.VRS_ESIZE
        qids, ids, dist = e.join_topk(qrel, qattrs, gen.pred_less_than(50), rpred, 4)
    _check(x, attrs, qrel, qattrs, gen.pred_less_than(50), rpred, 4, "l2", qids, ids, dist)
