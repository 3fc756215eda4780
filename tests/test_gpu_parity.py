"""GPU parity: the CUDA path through the C ABI against the float64 oracle.

Inputs are seeded and synthetic (gen/); expected values come from oracle/
only.  Bit-exact for bitmaps, counts, ids lists and encodings; top-k under
the tolerance rule in tests/_parity.py.
"""
import numpy as np
import pytest

import gen
import oracle
from _parity import check_topk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vrs():
    from paper_2403_15807_gb300 import build, vrs as v
    build.build()
    v.load()
    return v


def _engine(vrs, x, attrs, dtype=None, copies=None):
    e = vrs.Engine(0)
    if dtype is None:
        e.load(x, attrs)
    else:
        e.load(x, attrs, dtype=dtype, copies=copies)
    return e


# ------------------------------------------------------------------ filter

@pytest.mark.parametrize("n", [1, 31, 4096, 4097, 100_003])
def test_predicate_bitmap_and_count(vrs, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, 8)).astype(np.float32)
    attrs = rng.integers(-50, 50, size=(3, n), dtype=np.int32)
    with _engine(vrs, x, attrs) as e:
        for pred in [gen.pred_all(), gen.Pred([0], [-10], [25]), gen.Pred([0, 2], [-50, 0], [0, 50]),
                     gen.Pred([1], [5], [5]), gen.Pred([0, 1, 2], [-40, -40, -40], [40, 40, 40])]:
            bm, cnt = vrs.vrs_eval_predicate(e.h, pred, n)
            rbm, rcnt = oracle.predicate(attrs, pred.cols, pred.lo, pred.hi)
            assert cnt == rcnt
            assert np.array_equal(bm, rbm)
            ids = vrs.vrs_select_ids(e.h, pred, n)
            assert np.array_equal(ids, oracle.compact(rbm, n))


def test_predicate_mod100_closed_form(vrs):
    n = 1_000_000
    x = np.zeros((n, 4), np.float32)
    attrs = (np.arange(n) % 100).astype(np.int32)[None, :]
    with _engine(vrs, x, attrs) as e:
        _, cnt = vrs.vrs_eval_predicate(e.h, gen.pred_less_than(10), n)
        assert cnt == n // 10


# ------------------------------------------------------------------ load

@pytest.mark.parametrize("d", [1, 7, 96, 128, 960])
def test_norms_compensated(vrs, d):
    mix = gen.Mixture(d, seed=d)
    x = gen.vectors(3000, mix)
    with _engine(vrs, x, np.zeros((1, 3000), np.int32)) as e:
        got = vrs.vrs_get_norms(e.h, 3000).astype(np.float64)
    ref = oracle.sqnorm(x)
    # compensated float32 sum of exactly split squares: within 2 ulp-units
    assert np.all(np.abs(got - ref) <= 2.0 ** -23 * ref + 1e-30)


def test_encodings_bit_exact(vrs):
    mix = gen.Mixture(100, seed=3)
    x = gen.vectors(2000, mix)
    x[5] = 0.0
    x[6, :3] = [1e-9, -3e-7, 2e-8]
    with _engine(vrs, x, np.zeros((1, 2000), np.int32), dtype=vrs.VRS_F32,
                 copies=(1 << vrs.VRS_F32) | (1 << vrs.VRS_BF16) | (1 << vrs.VRS_FP8E4M3)) as e:
        f32, _ = vrs.vrs_get_encoded(e.h, vrs.VRS_F32, 2000, 100)
        b16, _ = vrs.vrs_get_encoded(e.h, vrs.VRS_BF16, 2000, 100)
        e8, s8 = vrs.vrs_get_encoded(e.h, vrs.VRS_FP8E4M3, 2000, 100)
    assert np.array_equal(f32, x)
    assert np.array_equal(b16, oracle.bf16_encode(x))
    rc, rs = oracle.e4m3_rows(x)
    assert np.array_equal(s8, rs)
    assert np.array_equal(e8, rc)


# ------------------------------------------------------------------ top-k

def _run(vrs, x, attrs, q, preds, k, metric="l2", on_device=True, **kw):
    with _engine(vrs, x, attrs) as e:
        m = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
        kk = np.atleast_1d(k).astype(np.int32)
        if on_device:
            ids, dist = e.query(torch.from_numpy(q).cuda(), preds, kk, metric=m, **kw)
            torch.cuda.synchronize()
            return ids.cpu().numpy(), dist.cpu().numpy()
        return e.query(q, preds, kk, metric=m, **kw)


def _check(x, attrs, q, preds, k, metric, gids, gdist):
    kk = np.broadcast_to(np.atleast_1d(k), (q.shape[0],)).astype(np.int32)
    rid, rdist, rcnt = oracle.query(x, attrs, q, preds, kk + 1, metric, n_threads=8)
    check_topk(x, q, attrs, preds, kk, metric, gids, gdist, rid, rdist, rcnt)


@pytest.mark.parametrize("on_device", [True, False])
def test_small_workload(vrs, on_device):
    wl = gen.small_l2()
    mix = wl.mixture()
    x = gen.vectors(wl.n, mix)
    q = gen.queries(wl.batch, mix)
    attrs = gen.attributes(wl.n, 1, wl.attr_range)
    pred = wl.pred()
    ids, dist = _run(vrs, x, attrs, q, [pred], wl.k, on_device=on_device)
    _check(x, attrs, q, [pred], wl.k, "l2", ids, dist)


@pytest.mark.parametrize("n,d,b,k,s,metric", [
    (1, 4, 1, 1, 1.0, "l2"),
    (33, 7, 3, 5, 1.0, "l2"),
    (1000, 100, 17, 10, 0.5, "l2"),
    (5000, 64, 33, 100, 0.3, "ip"),
    (20011, 96, 64, 10, 0.01, "l2"),
    (20011, 96, 5, 256, 1.0, "ip"),
    (70001, 128, 2, 10, 0.001, "l2"),
    (30000, 960, 9, 10, 0.2, "l2"),
    (12345, 32, 200, 7, 0.6, "ip"),
])
def test_shapes(vrs, n, d, b, k, s, metric):
    mix = gen.Mixture(d, seed=n % 97)
    unit = metric == "ip"
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, 1, 1000, seed=d)
    pred = gen.pred_less_than(int(s * 1000)) if s < 1 else gen.pred_all()
    ids, dist = _run(vrs, x, attrs, q, [pred], k, metric)
    _check(x, attrs, q, [pred], k, metric, ids, dist)


def test_empty_selection_pads(vrs):
    mix = gen.Mixture(16, seed=1)
    x = gen.vectors(500, mix)
    q = gen.queries(4, mix)
    attrs = gen.attributes(500, 1, 100)
    ids, dist = _run(vrs, x, attrs, q, [gen.Pred([0], [200], [300])], 10)
    assert np.all(ids == -1) and np.all(np.isinf(dist))


def test_fewer_rows_than_k(vrs):
    mix = gen.Mixture(16, seed=2)
    x = gen.vectors(3000, mix)
    q = gen.queries(3, mix)
    attrs = np.arange(3000, dtype=np.int32)[None, :]
    pred = gen.Pred([0], [100], [106])
    ids, dist = _run(vrs, x, attrs, q, [pred], 10)
    _check(x, attrs, q, [pred], 10, "l2", ids, dist)
    assert np.all(ids[:, 6:] == -1)


def test_duplicate_rows_tie_break(vrs):
    rng = np.random.default_rng(4)
    base = rng.integers(-4, 5, size=(50, 16)).astype(np.float32)
    x = np.repeat(base, 40, axis=0)           # every row appears 40 times
    attrs = np.zeros((1, x.shape[0]), np.int32)
    q = base[:5] + 0.25
    ids, dist = _run(vrs, x, attrs, q, [gen.pred_all()], 30)
    rid, rdist, _ = oracle.query(x, attrs, q, [gen.pred_all()], 30, "l2")
    assert np.array_equal(ids, rid)           # exact ties -> smallest ids first
    np.testing.assert_allclose(dist, rdist, rtol=1e-6)


def test_per_query_predicates_and_k(vrs):
    mix = gen.Mixture(48, seed=8)
    n = 40000
    x = gen.vectors(n, mix)
    attrs = gen.attributes(n, 2, 1_000_000, seed=8)
    preds, _ = gen.per_query_preds(12, seed=8)
    ks = gen.per_query_k(12, seed=8)
    q = gen.queries(12, mix)
    ids, dist = _run(vrs, x, attrs, q, preds, ks)
    _check(x, attrs, q, preds, ks, "l2", ids, dist)


def test_full_size_sampled_1m(vrs):
    """1M x 128 fp32, B=16, s=10% and 100%: oracle on all 16 queries."""
    wl = gen.sweep_cell(16, 0.1)
    mix = wl.mixture()
    x = gen.vectors(wl.n, mix)
    q = gen.queries(wl.batch, mix)
    attrs = gen.attributes(wl.n, 1, wl.attr_range)
    with _engine(vrs, x, attrs) as e:
        for pred in [wl.pred(), gen.pred_all()]:
            ids, dist = e.query(torch.from_numpy(q).cuda(), [pred], np.int32([10]))
            torch.cuda.synchronize()
            _check(x, attrs, q, [pred], 10, "l2", ids.cpu().numpy(), dist.cpu().numpy())


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("n,d,b,k,s", [(100_003, 128, 16, 10, 0.1), (50_000, 64, 5, 20, 0.9),
                                       (30_001, 112, 1, 7, 0.02), (9_000, 192, 12, 64, 1.0)])
def test_fused_and_predicate_first_gemv(vrs, fused, n, d, b, k, s):
    """The GEMV plan with the predicate evaluated inside the distance kernel
    (Sec. 3.2 on the fly) and as separate predicate/compaction kernels
    (predicate first) both match the oracle."""
    mix = gen.Mixture(d, seed=d + b)
    x = gen.vectors(n, mix)
    q = gen.queries(b, mix)
    attrs = gen.attributes(n, 2, 1000, seed=n % 13)
    pred = gen.Pred([0, 1], [0, 0], [int(s * 1000), 1000])
    with _engine(vrs, x, attrs) as e:
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_FUSED_SCAN, fused)
        ids, dist = e.query(torch.from_numpy(q).cuda(), [pred], np.int32([k]))
        torch.cuda.synchronize()
    _check(x, attrs, q, [pred], k, "l2", ids.cpu().numpy(), dist.cpu().numpy())


@pytest.mark.parametrize("dense", [1, 0])
@pytest.mark.parametrize("n,d,b,k,s,metric", [(200_003, 128, 16, 10, 0.1, "l2"),
                                              (50_000, 96, 3, 100, 1.0, "ip"),
                                              (9_000, 64, 40, 7, 0.002, "l2")])
def test_dense_key_and_in_scan_selection(vrs, dense, n, d, b, k, s, metric):
    """The GEMV plan with every first-pass key written and selected per
    partition, and with selection inside the scan, both match the oracle."""
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=b + d)
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, 1, 1000, seed=5)
    pred = gen.pred_less_than(int(s * 1000)) if s < 1 else gen.pred_all()
    with _engine(vrs, x, attrs) as e:
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_DENSE_KEYS, dense)
        ids, dist = e.query(torch.from_numpy(q).cuda(), [pred], np.int32([k]),
                            metric=vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP)
        torch.cuda.synchronize()
    _check(x, attrs, q, [pred], k, metric, ids.cpu().numpy(), dist.cpu().numpy())


def test_graph_replay_with_changing_predicates(vrs):
    """On a non-default stream the dense-key GEMV pipeline is run eagerly,
    then captured into a CUDA graph and replayed; the predicate lives in a
    device buffer, so replays with other predicates stay exact."""
    n, d, b = 120_000, 128, 16
    mix = gen.Mixture(d, seed=44)
    x = gen.vectors(n, mix)
    q = gen.queries(b, mix)
    attrs = gen.attributes(n, 1, 1000, seed=44)
    st = torch.cuda.Stream()
    qd = torch.from_numpy(q).cuda()
    oid = torch.empty((b, 10), dtype=torch.int64, device="cuda")
    od = torch.empty((b, 10), dtype=torch.float32, device="cuda")
    with _engine(vrs, x, attrs) as e:
        for rep, hi in enumerate([100, 100, 100, 130, 90, 120]):
            pred = gen.pred_less_than(hi)
            with torch.cuda.stream(st):
                vrs.vrs_query(e.h, qd, [pred], np.int32([10]), out_ids=oid, out_dist=od,
                              stream=st)
            st.synchronize()
            _check(x, attrs, q, [pred], 10, "l2", oid.cpu().numpy(), od.cpu().numpy())


@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("cap", [1, 64, 250, 1 << 30])
def test_dense_key_list_capacity(vrs, graph, cap):
    """List capacities in the dense-key merge: at 1 and 64 the chunk minima
    are read from global memory and the candidates overflow, so the merge
    selects from the whole key row; at 250 the minima are staged in shared
    memory and the candidate chunks fit; a huge request is clamped to the
    shared memory the CTA can have.  Results stay exact, eagerly and through
    the captured graph."""
    n, d, b, k = 150_000, 128, 12, 10
    mix = gen.Mixture(d, seed=cap + 7)
    x = gen.vectors(n, mix)
    q = gen.queries(b, mix)
    attrs = gen.attributes(n, 1, 1000, seed=cap)
    pred = gen.pred_less_than(200)
    st = torch.cuda.Stream()
    qd = torch.from_numpy(q).cuda()
    oid = torch.empty((b, k), dtype=torch.int64, device="cuda")
    od = torch.empty((b, k), dtype=torch.float32, device="cuda")
    with _engine(vrs, x, attrs) as e:
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_SELECT_CAP, cap)
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_GRAPH, graph)
        for _ in range(3):
            with torch.cuda.stream(st):
                vrs.vrs_query(e.h, qd, [pred], np.int32([k]), out_ids=oid, out_dist=od,
                              stream=st)
            st.synchronize()
            _check(x, attrs, q, [pred], k, "l2", oid.cpu().numpy(), od.cpu().numpy())


@pytest.mark.parametrize("staged", [1, 0])
@pytest.mark.parametrize("n,d,b,k,s,metric,compute", [
    (70_001, 128, 16, 10, 0.1, "l2", "f32"),
    (33_333, 64, 1, 5, 0.5, "ip", "f32"),
    (40_000, 144, 3, 10, 0.3, "l2", "bf16"),
    (25_000, 128, 32, 20, 0.05, "l2", "f32"),
    (9_000, 96, 40, 7, 0.02, "ip", "bf16"),
])
def test_staged_dense_key_scan(vrs, staged, n, d, b, k, s, metric, compute):
    """The dense-key GEMV distance pass with rows staged through shared
    memory by bulk copies, and with rows read into registers, match the
    oracle: float32 and bf16 rows (d = 144 in bf16 is 288-byte rows, whose
    last 64-byte step runs past the row), one to two query groups, selected
    counts that end inside a 128-position chunk."""
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=b * 7 + d)
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, 1, 1000, seed=b + 3)
    pred = gen.pred_less_than(int(s * 1000))
    cd = vrs.VRS_F32 if compute == "f32" else vrs.VRS_BF16
    with _engine(vrs, x, attrs, dtype=vrs.VRS_F32,
                 copies=(1 << vrs.VRS_F32) | (1 << vrs.VRS_BF16)) as e:
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_STAGED_SCAN, staged)
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_TENSOR_GEMV, 0)
        vrs.vrs_set_plan(e.h, vrs.VRS_PLAN_GEMV)
        ids, dist = e.query(torch.from_numpy(q).cuda(), [pred], np.int32([k]),
                            metric=vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP, compute=cd)
        torch.cuda.synchronize()
        assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_GEMV
    _check(x, attrs, q, [pred], k, metric, ids.cpu().numpy(), dist.cpu().numpy())


@pytest.mark.parametrize("tensor", [1, 0])
@pytest.mark.parametrize("n,d,b,k,s,metric", [
    (100_003, 128, 16, 10, 0.1, "l2"),
    (30_001, 128, 5, 10, 0.3, "ip"),
    (50_000, 144, 17, 10, 0.2, "l2"),
    (20_000, 64, 64, 10, 0.5, "l2"),
    (12_345, 32, 33, 3, 0.9, "ip"),
    (8_000, 960, 16, 10, 0.4, "l2"),
    (40_000, 256, 1, 50, 0.05, "l2"),
])
def test_tensor_gemv_dense_keys(vrs, tensor, n, d, b, k, s, metric):
    """The float32 GEMV plan with its dense-key distance pass on the tensor
    cores (3xTF32: rows as MMA M, queries as N; one to four query tiles;
    d = 144 ends in half a 128-byte K block; d = 960 keeps two stages) and on
    the CUDA cores, both matching the oracle."""
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=b * 11 + d)
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, 1, 1000, seed=b + 9)
    pred = gen.pred_less_than(int(s * 1000))
    with _engine(vrs, x, attrs) as e:
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_TENSOR_GEMV, tensor)
        vrs.vrs_set_plan(e.h, vrs.VRS_PLAN_GEMV)
        ids, dist = e.query(torch.from_numpy(q).cuda(), [pred], np.int32([k]),
                            metric=vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP)
        torch.cuda.synchronize()
    _check(x, attrs, q, [pred], k, metric, ids.cpu().numpy(), dist.cpu().numpy())


def test_float_attribute_ranges(vrs):
    """A float attribute column (loaded as its order-preserving int32 image,
    with -0, NaN and +inf among its values) under a float range, combined
    with an int range on another column: the selection equals the float
    semantics lo <= a < hi, and the top-k equals the oracle's over it."""
    n, d, b, k = 60_000, 64, 16, 10
    mix = gen.Mixture(d, seed=31)
    x = gen.vectors(n, mix)
    q = gen.queries(b, mix)
    rng = np.random.default_rng(31)
    fcol = (rng.standard_normal(n) * 3).astype(np.float32)
    fcol[::97] = -0.0
    fcol[5], fcol[7], fcol[11] = np.nan, np.inf, -np.inf
    icol = gen.attributes(n, 1, 100, seed=32)[0]
    lo, hi = -1.25, 2.5
    sel = (fcol >= lo) & (fcol < hi) & (icol < 60)
    with _engine(vrs, x, icol[None, :]) as e:
        vrs.vrs_load_attribute_f32(e.h, 1, fcol)
        c, klo, khi = vrs.float_range(1, lo, hi)
        pred = vrs.Pred([0, c], [gen.INT32_MIN, klo], [60, khi])
        _, cnt = vrs.vrs_eval_predicate(e.h, pred, n)
        ids, dist = e.query(torch.from_numpy(q).cuda(), [pred], np.int32([k]))
        torch.cuda.synchronize()
    assert cnt == int(sel.sum())
    # the oracle sees the float semantics as a 0/1 column
    sattr = sel.astype(np.int32)[None, :]
    spred = gen.Pred([0], [1], [2])
    _check(x, sattr, q, [spred], k, "l2", ids.cpu().numpy(), dist.cpu().numpy())


@pytest.mark.parametrize("on_device", [True, False])
@pytest.mark.parametrize("compute,metric", [("f32", "l2"), ("bf16", "ip")])
def test_disjunction_and_in_list(vrs, compute, metric, on_device):
    """Top-k under a disjunction of conjunctions (two of them overlapping, so
    rows come back from several lists and must be kept once) and under an
    IN-list; the oracle searches the rows the disjunction selects."""
    n, d, b, k = 50_000, 64, 16, 10
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=51)
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, 2, 1000, seed=51)
    cd = vrs.VRS_F32 if compute == "f32" else vrs.VRS_BF16
    mt = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    cases = [
        [gen.Pred([0], [gen.INT32_MIN], [100]), gen.Pred([0], [50], [300]),
         gen.Pred([0, 1], [900, 3], [1000, 40])],
        vrs.in_list(1, [7, 77, 500, 999]),
    ]
    with _engine(vrs, x, attrs, dtype=vrs.VRS_F32, copies=7) as e:
        for conjs in cases:
            qq = torch.from_numpy(q).cuda() if on_device else q
            ids, dist = e.query_dnf(qq, conjs, k, metric=mt, compute=cd)
            if on_device:
                torch.cuda.synchronize()
                ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
            sel = np.zeros(n, bool)
            for c in conjs:
                m = np.ones(n, bool)
                for col, lo, hi in zip(c.cols, c.lo, c.hi):
                    m &= (attrs[col] >= lo) & (attrs[col] < hi)
                sel |= m
            sattr = sel.astype(np.int32)[None, :]
            _check(x, sattr, q, [gen.Pred([0], [1], [2])], k, metric, ids, dist)
            for i in range(b):
                got = ids[i][ids[i] >= 0]
                assert len(np.unique(got)) == len(got)


# ------------------------------------------------------- measurement hook
@pytest.mark.parametrize("n,cols,m", [(10_000, 40, 3_000), (50_000, 128, 50_000), (7, 4, 0)])
def test_probe_gather_reads_every_listed_row(vrs, n, cols, m):
    """vrs_probe_gather adds the sum of every listed row to *out: rows of
    160 bytes (a partial warp), 512 bytes, and an empty list.  Entries are 0
    or 1, so every partial sum is an integer below 2^24 and exact in float32:
    one row left out or read twice changes the total."""
    g = torch.Generator(device="cpu").manual_seed(n)
    X = torch.randint(0, 2, (n, cols), generator=g).float().cuda()
    ids = torch.randperm(n, generator=g)[:m].to(torch.int32).cuda()
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    vrs.vrs_probe_gather(X, ids, out)
    torch.cuda.synchronize()
    assert float(out) == float(X.double()[ids.long()].sum())


def test_probe_gather_rejects_bad_rows(vrs):
    X = torch.rand(100, 5).cuda()   # 20-byte rows
    ids = torch.arange(10, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(vrs.VrsError) as ei:
        vrs.vrs_probe_gather(X, ids, out)
    assert ei.value.status == vrs.VRS_EINVAL


def test_probe_gather_skips_ids_outside_the_table(vrs):
    """Ids at or past the table's row count (and negative ones) are not read."""
    X = torch.randint(0, 2, (1000, 32)).float().cuda()
    ids = torch.tensor([0, 1, 999, 1000, 5000, -3, 2_000_000_000], dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    vrs.vrs_probe_gather(X, ids, out)
    torch.cuda.synchronize()
    assert float(out) == float(X.double()[[0, 1, 999]].sum())
