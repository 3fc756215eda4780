"""vrs_query_noalloc: the filtered top-k for callers that cannot allocate
device memory (inside a CUDA graph capture, under an allocator that owns the
pool, or with a memory budget fixed at start-up).  Its results must match
the engine's vrs_query (GEMV plan, FP32) on the same inputs, on two calls in
a row (the second call reuses the shared scratch array the first one left
behind).  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_matches_engine_twice():
    from paper_2403_15807_gb300 import build, vrs
    build.build()
    L = vrs.load()
    n, d, b, k = 200_000, 128, 16, 10
    mix = gen.Mixture(d, seed=21)
    x = gen.vectors(n, mix)
    q = gen.queries(b, mix)
    attrs = gen.attributes(n, 2, 1000, seed=21)
    preds = [gen.Pred([0], [0], [300]), gen.Pred([0, 1], [100, 0], [800, 500])]
    xd = torch.from_numpy(x).cuda()
    ad = torch.from_numpy(attrs).cuda()
    qd = torch.from_numpy(q).cuda()
    with vrs.Engine(0) as e:
        e.load(x, attrs)
        vrs.vrs_set_plan(e.h, vrs.VRS_PLAN_GEMV)
        for pred in preds:
            ref_ids, ref_dist = e.query(qd, [pred], np.int32([k]))
            torch.cuda.synchronize()
            ref_ids, ref_dist = ref_ids.cpu().numpy(), ref_dist.cpu().numpy()
            parr, keep = vrs.make_preds([pred])
            for _ in range(2):
                oid = torch.full((b, k), -7, dtype=torch.int64, device="cuda")
                od = torch.full((b, k), -7.0, dtype=torch.float32, device="cuda")
                st = L.vrs_query_noalloc(_p(xd), n, d, _p(ad), 2, parr, _p(qd), b, k,
                                         vrs.VRS_L2, _p(oid), _p(od), None)
                assert st == vrs.VRS_OK, L.vrs_last_error()
                torch.cuda.synchronize()
                assert np.array_equal(oid.cpu().numpy(), ref_ids)
                np.testing.assert_allclose(od.cpu().numpy(), ref_dist, rtol=1e-4)


def test_noalloc_rejects_sizes_beyond_limits():
    from paper_2403_15807_gb300 import vrs
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
                                 _p(oid), _p(od), None)
        assert st == vrs.VRS_EINVAL
        assert b"vrs_query_noalloc" in L.vrs_last_error()
