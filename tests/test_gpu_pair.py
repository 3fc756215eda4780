"""The tensor-core GEMV pass over the bf16 pair copy (VRS_OPT_PAIR_COPY):
parity with the float64 oracle across batch sizes (one to four query
tiles of 16/32/64), ragged dimensions (the pair row pads d to a multiple of
64), both metrics, and the full 1M-row headline shape on a sample."""
import numpy as np
import pytest

import gen
import oracle
from _parity import check_topk, recall

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vrs():
    from paper_2403_15807_gb300 import build, vrs as v
    build.build()
    v.load()
    return v


def _engine(vrs, x, attrs):
    e = vrs.Engine(0)
    vrs.vrs_set_option(e.h, vrs.VRS_OPT_PAIR_COPY, 1)
    e.load(x, attrs)
    return e


@pytest.mark.parametrize("n,d,b,k,s,metric", [
    (30011, 128, 1, 10, 0.3, "l2"),
    (30011, 128, 16, 10, 0.1, "l2"),
    (30011, 128, 17, 7, 0.5, "ip"),
    (20000, 144, 33, 10, 0.4, "l2"),
    (20000, 64, 64, 100, 0.9, "l2"),
    (12000, 960, 16, 10, 0.5, "l2"),
    (40000, 96, 50, 1, 1.0, "ip"),
])
def test_pair_gemv_matches_oracle(vrs, n, d, b, k, s, metric):
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=n % 97 + d)
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, 1, 1000, seed=b)
    pred = gen.pred_less_than(int(s * 1000))
    m = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    e = _engine(vrs, x, attrs)
    try:
        vrs.vrs_set_plan(e.h, vrs.VRS_PLAN_GEMV)
        stream = torch.cuda.Stream()
        qd = torch.from_numpy(q).cuda()
        for _ in range(3):   # eager, captured, replayed
            ids, dist = e.query(qd, [pred], np.int32([k]), metric=m, stream=stream)
            stream.synchronize()
        cert = vrs.vrs_last_cert(e.h)
    finally:
        e.close()
    assert sum(cert.values()) == b
    rid, rdist, rcnt = oracle.query(x, attrs, q, [pred], k + 1, metric, n_threads=16)
    check_topk(x, q, attrs, [pred], np.int32([k]), metric, ids.cpu().numpy(),
               dist.cpu().numpy(), rid, rdist, rcnt)
    assert recall(ids.cpu().numpy(), rid, k) == 1.0


@pytest.mark.parametrize("n,d,b,k,lo,hi,metric", [
    (50_000, 128, 16, 10, 1234, 3000, "l2"),    # a run in the middle (TMA and cp.async tiles)
    (50_000, 128, 16, 10, 0, 4999, "ip"),       # every row
    (30_011, 960, 8, 5, 17, 2_100, "l2"),       # 15 stages per tile
])
def test_pair_gemv_row_runs(vrs, n, d, b, k, lo, hi, metric):
    """A column that follows row order (row // 10): a range on it selects one
    run of consecutive rows (the id list is then runs of ascending rows, one
    per filter block, in the blocks' atomic order), ragged at both ends."""
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=d + 7)
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = (np.arange(n, dtype=np.int64) // 10).astype(np.int32)[None, :]
    pred = gen.Pred([0], [lo], [hi])
    m = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    e = _engine(vrs, x, attrs)
    try:
        vrs.vrs_set_plan(e.h, vrs.VRS_PLAN_GEMV)
        stream = torch.cuda.Stream()
        qd = torch.from_numpy(q).cuda()
        for _ in range(3):   # eager, captured, replayed
            ids, dist = e.query(qd, [pred], np.int32([k]), metric=m, stream=stream)
            stream.synchronize()
        assert sum(vrs.vrs_last_cert(e.h).values()) == b
    finally:
        e.close()
    rid, rdist, rcnt = oracle.query(x, attrs, q, [pred], k + 1, metric, n_threads=16)
    check_topk(x, q, attrs, [pred], np.int32([k]), metric, ids.cpu().numpy(), dist.cpu().numpy(),
               rid, rdist, rcnt)


def test_pair_gemv_headline_sampled(vrs):
    """1M x 128 fp32, 10 % selected, 16 queries: every query against the oracle."""
    wl = gen.sweep_cell(16, 0.1)
    mix = wl.mixture()
    x = gen.vectors(wl.n, mix)
    q = gen.queries(wl.batch, mix)
    attrs = gen.attributes(wl.n, 1, wl.attr_range)
    pred = wl.pred()
    e = _engine(vrs, x, attrs)
    try:
        ids, dist = e.query(torch.from_numpy(q).cuda(), [pred], np.int32([10]))
        torch.cuda.synchronize()
    finally:
        e.close()
    rid, rdist, rcnt = oracle.query(x, attrs, q, [pred], 11, "l2", n_threads=16)
    check_topk(x, q, attrs, [pred], np.int32([10]), "l2", ids.cpu().numpy(), dist.cpu().numpy(),
               rid, rdist, rcnt)


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_large_fp32_batch_in_tensor_sub_batches(vrs, metric):
    """300k x 128 fp32, 256 queries: the batch's key matrix (307 MB) is
    past the dense-key limit, so it runs as four 64-query sub-batches on
    the pair-copy kernel; per-query k, results equal to the CUDA-core scan
    (VRS_OPT_TENSOR_GEMV = 0) and to the oracle on a sample."""
    n, d, b = 300_000, 128, 256
    mix = gen.Mixture(d, seed=11)
    unit = metric == "ip"
    x = gen.vectors(n, mix, unit=unit)
    attrs = gen.attributes(n, 1, 100, seed=11)
    q = gen.queries(b, mix, unit=unit)
    pred = gen.pred_less_than(20)
    ks = np.random.default_rng(11).choice(np.int32([1, 10, 25]), size=b).astype(np.int32)
    m = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    with _engine(vrs, x, attrs) as e:
        qd = torch.from_numpy(q).cuda()
        ids, dist = e.query(qd, [pred], ks, k_max=25, metric=m)
        torch.cuda.synchronize()
        assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_GEMV
        assert sum(vrs.vrs_last_cert(e.h).values()) == b
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_TENSOR_GEMV, 0)
        ids2, dist2 = e.query(qd, [pred], ks, k_max=25, metric=m)
        torch.cuda.synchronize()
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    assert np.array_equal(ids, ids2.cpu().numpy())
    assert np.array_equal(dist, dist2.cpu().numpy())
    pick = np.linspace(0, b - 1, 24).astype(int)
    rid, rdist, rcnt = oracle.query(x, attrs, q[pick], [pred], ks[pick] + 1, metric, k_max=26,
                                    n_threads=16)
    check_topk(x, q[pick], attrs, [pred], ks[pick], metric, ids[pick], dist[pick], rid, rdist, rcnt)


@pytest.mark.parametrize("zero_copy", [1, 0])
def test_pinned_host_buffers_through_the_graph(vrs, zero_copy):
    """A host-buffer call with page-locked queries and outputs (the captured
    GEMV form: eager, captured, replayed): with VRS_OPT_ZERO_COPY the kernels
    read and write the host buffers in place, without it the graph copies;
    both equal the device-buffer call and the oracle."""
    import ctypes as C
    n, d, b, k = 200_000, 128, 16, 10
    mix = gen.Mixture(d, seed=12)
    x = gen.vectors(n, mix)
    attrs = gen.attributes(n, 1, 100, seed=12)
    q = gen.queries(b, mix)
    pred = gen.pred_less_than(10)
    qh = torch.from_numpy(q).pin_memory()
    with _engine(vrs, x, attrs) as e:
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_ZERO_COPY, zero_copy)
        ref_ids, ref_dist = e.query(torch.from_numpy(q).cuda(), [pred], np.int32([k]))
        torch.cuda.synchronize()
        parr, keep = vrs.make_preds([pred])
        kk = np.int32([k])
        L = vrs.load()
        for rep in range(4):
            oid = torch.full((b, k), -7, dtype=torch.int64).pin_memory()
            od = torch.full((b, k), -7.0, dtype=torch.float32).pin_memory()
            st = L.vrs_query(e.h, C.c_void_p(qh.data_ptr()), b, d, parr, 1,
                             kk.ctypes.data_as(C.c_void_p), 1, k, vrs.VRS_L2, vrs.VRS_F32,
                             C.c_void_p(oid.data_ptr()), C.c_void_p(od.data_ptr()), 0, None)
            assert st == vrs.VRS_OK, L.vrs_last_error()
            assert torch.equal(oid, ref_ids.cpu()), rep
            assert torch.equal(od, ref_dist.cpu()), rep
    ids = oid.numpy()
    rid, rdist, rcnt = oracle.query(x, attrs, q, [pred], np.int32([k + 1]), "l2", n_threads=16)
    check_topk(x, q, attrs, [pred], k, "l2", ids, od.numpy(), rid, rdist, rcnt)
