"""vrs_query_noalloc: the filtered top-k for callers that cannot allocate
device memory while they run -- a host whose allocator owns the whole
device pool, a service that fixes its memory budget at start-up, a loop that
must not stall on the driver's allocator.  Its results are held to the float64 oracle with the
same rule as every other parity test, on two calls in a row (the second
call reuses the shared scratch array the first one left behind), and to
the engine's vrs_query on the same inputs.  This file is collected last on
purpose."""
import ctypes as C

import numpy as np
import pytest

import gen
import oracle
from _parity import check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def vrs():
    from paper_2403_15807_gb300 import build, vrs as v
    build.build()
    v.load()
    return v


def _noalloc(vrs, xd, n, d, ad, n_cols, pred, qd, b, k, metric):
    L = vrs.load()
    parr, keep = vrs.make_preds([pred])
    oid = torch.full((b, k), -7, dtype=torch.int64, device="cuda")
    od = torch.full((b, k), -7.0, dtype=torch.float32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = L.vrs_query_noalloc(_p(xd), n, d, _p(ad), n_cols, parr, _p(qd), b, k, metric, _p(oid),
                             _p(od), _p(status), None)
    assert st == vrs.VRS_OK, L.vrs_last_error()
    torch.cuda.synchronize()
    return oid.cpu().numpy(), od.cpu().numpy(), int(status.item())


@pytest.mark.parametrize("n,d,n_cols,k,metric", [
    (200_000, 128, 2, 10, "l2"),   # two columns: n a multiple of 4
    (123_457, 64, 1, 1, "l2"),     # ragged n, k = 1
    (50_003, 256, 1, 4, "ip"),     # ragged n, k = 4, unit vectors
])
def test_noalloc_matches_oracle_twice(vrs, n, d, n_cols, k, metric):
    b = 16
    mix = gen.Mixture(d, seed=21)
    unit = metric == "ip"
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, n_cols, 1000, seed=21)
    preds = [gen.Pred([0], [0], [300])]
    if n_cols == 2:
        preds.append(gen.Pred([0, 1], [100, 0], [800, 500]))
    m = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    xd = torch.from_numpy(x).cuda()
    ad = torch.from_numpy(attrs).cuda()
    qd = torch.from_numpy(q).cuda()
    for pred in preds:
        rid, rdist, rcnt = oracle.query(x, attrs, q, [pred], k + 1, metric, n_threads=16)
        for _ in range(2):
            ids, dist, status = _noalloc(vrs, xd, n, d, ad, n_cols, pred, qd, b, k, m)
            assert status == 0
            check_topk(x, q, attrs, [pred], np.int32([k]), metric, ids, dist, rid, rdist, rcnt)
    # and the engine agrees
    with vrs.Engine(0) as e:
        e.load(x, attrs)
        ref_ids, ref_dist = e.query(qd, [preds[-1]], np.int32([k]),
                                    metric=m)
        torch.cuda.synchronize()
    ids, dist, _ = _noalloc(vrs, xd, n, d, ad, n_cols, preds[-1], qd, b, k, m)
    np.testing.assert_allclose(dist, ref_dist.cpu().numpy(), rtol=1e-4, atol=1e-6)


def test_noalloc_rejects_sizes_beyond_limits(vrs):
    L = vrs.load()
    x = torch.zeros((64, 16), device="cuda")
    q = torch.zeros((1, 16), device="cuda")
    oid = torch.empty((1, 4), dtype=torch.int64, device="cuda")
    od = torch.empty((1, 4), dtype=torch.float32, device="cuda")
    parr, keep = vrs.make_preds([gen.pred_all()])
    a = torch.zeros((1, 64), dtype=torch.int32, device="cuda")
    bad = [
        (x, 2 ** 20 + 1, 16, 1, 4),   # n too large
        (x, 64, 24, 1, 4),            # d not a multiple of 16
        (x, 64, 16, 33, 4),           # batch too large
        (x, 64, 16, 1, 65),           # k too large
    ]
    for xx, n, d, bb, k in bad:
        st = L.vrs_query_noalloc(_p(xx), n, d, _p(a), 1, parr, _p(q), bb, k, vrs.VRS_L2,
                                 _p(oid), _p(od), None, None)
        assert st == vrs.VRS_EINVAL
        assert b"vrs_query_noalloc" in L.vrs_last_error()
