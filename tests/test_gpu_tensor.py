"""GPU parity of the tensor-core (tcgen05) plans against the float64 oracle.

COMPACT_GEMM (predicate first, qualifying rows gathered) and MASK_GEMM
(every row, predicate applied to the scores) with BF16 and FP8 E4M3
operands; the k' = 4k first-pass candidates are re-ranked exactly in FP32
from the float32 master (or from the stored bf16 values), so the final
result is held to the same rule as the FP32 path (tests/_parity.py).
"""
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


ALL = (1 << 0) | (1 << 1) | (1 << 2)


def _query(vrs, e, q, preds, k, metric, compute, plan):
    vrs.vrs_set_plan(e.h, plan)
    m = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    ids, dist = e.query(torch.from_numpy(q).cuda(), preds, np.atleast_1d(k).astype(np.int32),
                        metric=m, compute=compute)
    torch.cuda.synchronize()
    assert vrs.vrs_last_plan(e.h) == plan
    return ids.cpu().numpy(), dist.cpu().numpy()


def _check(x, attrs, q, preds, k, metric, gids, gdist):
    kk = np.broadcast_to(np.atleast_1d(k), (q.shape[0],)).astype(np.int32)
    rid, rdist, rcnt = oracle.query(x, attrs, q, preds, kk + 1, metric, n_threads=8)
    check_topk(x, q, attrs, preds, kk, metric, gids, gdist, rid, rdist, rcnt)
    return recall(gids, rid, int(kk.max()))


@pytest.mark.parametrize("plan", ["compact", "mask"])
@pytest.mark.parametrize("compute", ["bf16", "fp8"])
@pytest.mark.parametrize("n,d,b,k,s,metric", [
    (5000, 64, 1, 10, 0.3, "l2"),
    (20011, 128, 130, 10, 0.1, "l2"),
    (20011, 128, 300, 10, 0.6, "ip"),
    (30000, 960, 129, 10, 0.05, "l2"),
    (8000, 96, 64, 100, 0.5, "l2"),
])
def test_tensor_plans(vrs, plan, compute, n, d, b, k, s, metric):
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=(n + d) % 89)
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, 1, 1000, seed=b)
    pred = gen.pred_less_than(int(s * 1000))
    pl = vrs.VRS_PLAN_COMPACT_GEMM if plan == "compact" else vrs.VRS_PLAN_MASK_GEMM
    cd = vrs.VRS_BF16 if compute == "bf16" else vrs.VRS_FP8E4M3
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=ALL)
        ids, dist = _query(vrs, e, q, [pred], k, metric, cd, pl)
    assert _check(x, attrs, q, [pred], k, metric, ids, dist) == 1.0


def test_bf16_storage_full_scan(vrs):
    """bf16-stored rows and bf16-valued queries; re-rank from the stored values."""
    n, d = 50000, 96
    mix = gen.Mixture(d, seed=11)
    x = gen.to_bf16_values(gen.vectors(n, mix))
    q = gen.to_bf16_values(gen.queries(200, mix))
    attrs = gen.attributes(n, 2, 1_000_000, seed=11)
    pred = gen.Pred([0, 1], [0, 100_000], [700_000, 900_000])
    xb = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    with vrs.Engine(0) as e:
        vrs.vrs_load_vectors(e.h, np.ascontiguousarray(xb), dtype=vrs.VRS_BF16, copies=1 << 1)
        for c in range(2):
            vrs.vrs_load_attribute(e.h, c, attrs[c])
        for pl in (vrs.VRS_PLAN_COMPACT_GEMM, vrs.VRS_PLAN_MASK_GEMM):
            ids, dist = _query(vrs, e, q, [pred], 10, "l2", vrs.VRS_BF16, pl)
            _check(x, attrs, q, [pred], 10, "l2", ids, dist)


def test_tensor_empty_and_tiny(vrs):
    mix = gen.Mixture(32, seed=5)
    x = gen.vectors(700, mix)
    q = gen.queries(3, mix)
    attrs = np.arange(700, dtype=np.int32)[None, :]
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=ALL)
        for pl in (vrs.VRS_PLAN_COMPACT_GEMM, vrs.VRS_PLAN_MASK_GEMM):
            ids, dist = _query(vrs, e, q, [gen.Pred([0], [900], [1000])], 5, "l2", vrs.VRS_BF16, pl)
            assert np.all(ids == -1) and np.all(np.isinf(dist))
            pred = gen.Pred([0], [10], [13])
            ids, dist = _query(vrs, e, q, [pred], 5, "l2", vrs.VRS_FP8E4M3, pl)
            _check(x, attrs, q, [pred], 5, "l2", ids, dist)


def test_tensor_first_pass_recall(vrs):
    """Without re-rank the first-pass order is approximate; the first-pass
    top-k' at each dtype's default width (4k BF16, 16k FP8) still contains
    the exact top-k."""
    n, d, k = 40000, 128, 10
    mix = gen.Mixture(d, seed=3)
    x = gen.vectors(n, mix)
    q = gen.queries(256, mix)
    attrs = gen.attributes(n, 1, 1000, seed=3)
    pred = gen.pred_less_than(500)
    rid, _, _ = oracle.query(x, attrs, q, [pred], k, "l2", n_threads=8)
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=ALL)
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_RERANK, 0)
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_KPRIME_FACTOR, 1)
        for cd, f in ((vrs.VRS_BF16, 4), (vrs.VRS_FP8E4M3, 16)):
            idsk, _ = _query(vrs, e, q, [pred], f * k, "l2", cd, vrs.VRS_PLAN_COMPACT_GEMM)
            hit = np.mean([len(set(rid[i]) & set(idsk[i])) / k for i in range(256)])
            assert hit == 1.0, (cd, hit)


@pytest.mark.parametrize("compute", ["bf16", "fp8"])
@pytest.mark.parametrize("graph", [1, 0])
def test_batched_per_query_predicates(vrs, compute, graph):
    """One launch for a batch whose queries carry their own conjunctions on
    two columns and their own k (1, 10 or 100)."""
    n, d, b = 60_000, 96, 300
    mix = gen.Mixture(d, seed=17)
    x = gen.vectors(n, mix)
    q = gen.queries(b, mix)
    attrs = gen.attributes(n, 2, 1_000_000, seed=17)
    preds, _ = gen.per_query_preds(b, seed=17)
    ks = gen.per_query_k(b, seed=17)
    cd = vrs.VRS_BF16 if compute == "bf16" else vrs.VRS_FP8E4M3
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=ALL)
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_GRAPH, graph)
        for rep in range(2):   # second call replays the captured graph
            ids, dist = e.query(torch.from_numpy(q).cuda(), preds, ks, metric=vrs.VRS_L2,
                                compute=cd)
            torch.cuda.synchronize()
            assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_MASK_GEMM
            _check(x, attrs, q, preds, ks, "l2", ids.cpu().numpy(), dist.cpu().numpy())


def test_batched_matches_per_query_passes(vrs):
    n, d, b = 20_000, 64, 130
    mix = gen.Mixture(d, seed=23)
    x = gen.vectors(n, mix)
    q = gen.queries(b, mix)
    attrs = gen.attributes(n, 3, 1000, seed=23)
    rng = np.random.default_rng(23)
    preds = []
    for i in range(b):
        cols = list(rng.choice(3, size=rng.integers(0, 3), replace=False))
        los = [int(rng.integers(0, 500)) for _ in cols]
        preds.append(gen.Pred(cols, los, [lo + int(rng.integers(100, 500)) for lo in los]))
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=ALL)
        out = []
        for batched in (1, 0):
            vrs.vrs_set_option(e.h, vrs.VRS_OPT_BATCHED, batched)
            ids, dist = e.query(torch.from_numpy(q).cuda(), preds, np.int32([10]),
                                compute=vrs.VRS_BF16)
            torch.cuda.synchronize()
            out.append((ids.cpu().numpy(), dist.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0])
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-6)
    _check(x, attrs, q, preds, 10, "l2", out[0][0], out[0][1])


@pytest.mark.parametrize("plan", ["compact", "mask"])
def test_tma_and_cp_async_loads_agree(vrs, plan):
    """Query and dense row tiles loaded by TMA or by cp.async give the same
    results (and both match the oracle)."""
    n, d, b = 30_000, 192, 200
    mix = gen.Mixture(d, seed=31)
    x = gen.vectors(n, mix)
    q = gen.queries(b, mix)
    attrs = gen.attributes(n, 1, 1000, seed=31)
    pred = gen.pred_less_than(700)
    pl = vrs.VRS_PLAN_COMPACT_GEMM if plan == "compact" else vrs.VRS_PLAN_MASK_GEMM
    outs = []
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=ALL)
        for tma in (1, 0):
            vrs.vrs_set_option(e.h, vrs.VRS_OPT_TMA, tma)
            outs.append(_query(vrs, e, q, [pred], 10, "l2", vrs.VRS_BF16, pl))
    assert np.array_equal(outs[0][0], outs[1][0])
    _check(x, attrs, q, [pred], 10, "l2", outs[0][0], outs[0][1])


@pytest.mark.parametrize("n,d,b,k,s,metric,compute,plan,grid", [
    (100_003, 64, 40, 10, 1.0, "l2", "bf16", "mask", 4),
    (120_001, 128, 300, 5, 0.5, "ip", "bf16", "mask", 3),
    (60_000, 96, 17, 1, 0.9, "l2", "bf16", "mask", 2),
    (20_011, 128, 130, 10, 1.0, "l2", "fp8", "mask", 2),
    (20_011, 128, 40, 3, 0.9, "ip", "fp8", "mask", 2),
    (100_003, 64, 40, 10, 1.0, "l2", "bf16", "compact", 4),
    (20_011, 128, 130, 10, 0.5, "l2", "fp8", "compact", 2),
])
def test_seed_pass(vrs, n, d, b, k, s, metric, compute, plan, grid):
    """The sample pass that seeds every query's bound before the full
    pass (grids held to a few CTAs per query tile so that each sees enough
    selected rows; E4M3 with k' = 16k keeps its heaps in global memory and
    uses it on both plans).  With and without it the results match the
    oracle; the sample pass adds exactly its three launches, and none to
    BF16 COMPACT_GEMM."""
    unit = metric == "ip"
    mix = gen.Mixture(d, seed=(n + b) % 83)
    x = gen.vectors(n, mix, unit=unit)
    q = gen.queries(b, mix, unit=unit)
    attrs = gen.attributes(n, 1, 1000, seed=d)
    pred = gen.pred_less_than(int(s * 1000)) if s < 1 else gen.pred_all()
    pl = vrs.VRS_PLAN_COMPACT_GEMM if plan == "compact" else vrs.VRS_PLAN_MASK_GEMM
    cd = vrs.VRS_BF16 if compute == "bf16" else vrs.VRS_FP8E4M3
    launches = {}
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=ALL)
        # the bound-seeding sample pass of a first pass of default width (the
        # sample-seeded exact form replaces it when left on)
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_CERT_SAMPLE, 0)
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_GRID_CTAS, grid)
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_PROFILE, 1)
        for seed in (1, 0):
            vrs.vrs_set_option(e.h, vrs.VRS_OPT_SEED_BOUND, seed)
            ids, dist = _query(vrs, e, q, [pred], k, metric, cd, pl)
            launches[seed] = vrs.vrs_last_profile(e.h)[1]
            assert _check(x, attrs, q, [pred], k, metric, ids, dist) == 1.0
    assert launches[1] == launches[0] + (3 if plan == "mask" or compute == "fp8" else 0)
