"""Pins for the CPU oracle's predicate, compaction and exact top-k.

The oracle is held to things other than itself: pure-Python brute force with
exact rational arithmetic, closed-form datasets, invariants of the selection
operator (Sec. 3, eqs. "Brute force selection" and "Brute force similarity
search with relational predicate"), and the cosine identity of Sec. 3.1.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import gen
import oracle

INT32_MIN = gen.INT32_MIN


def _bits(bm, n):
    return np.array([(bm[i // 32] >> (i % 32)) & 1 for i in range(n)], dtype=np.uint8)


# ---------------------------------------------------------------- predicate

def test_predicate_closed_form_mod100():
    n = 100_000
    attrs = (np.arange(n) % 100).astype(np.int32)[None, :]
    bm, cnt = oracle.predicate(attrs, [0], [INT32_MIN], [10])
    assert cnt == n // 10
    bits = _bits(bm, n)
    assert np.array_equal(np.flatnonzero(bits), np.flatnonzero(np.arange(n) % 100 < 10))


@pytest.mark.parametrize("n", [1, 31, 32, 33, 95, 200])
def test_predicate_brute_force_all_ranges(n):
    rng = np.random.default_rng(n)
    attrs = rng.integers(-3, 4, size=(2, n), dtype=np.int32)
    for lo0, hi0 in itertools.product(range(-4, 5), repeat=2):
        lo1, hi1 = -2, 3
        bm, cnt = oracle.predicate(attrs, [0, 1], [lo0, lo1], [hi0, hi1])
        want = [int(lo0 <= attrs[0, i] < hi0 and lo1 <= attrs[1, i] < hi1) for i in range(n)]
        assert list(_bits(bm, n)) == want
        assert cnt == sum(want)
        # popcount of the words equals the count; no bit set past n
        assert sum(bin(int(w)).count("1") for w in bm) == cnt
        if n % 32:
            assert int(bm[-1]) >> (n % 32) == 0


def test_predicate_zero_terms_and_empty_range():
    attrs = np.arange(70, dtype=np.int32)[None, :]
    _, cnt = oracle.predicate(attrs, [], [], [])
    assert cnt == 70
    _, cnt = oracle.predicate(attrs, [0], [5], [5])
    assert cnt == 0
    _, cnt = oracle.predicate(attrs, [0], [9], [3])
    assert cnt == 0


def test_compact_matches_flatnonzero():
    rng = np.random.default_rng(1)
    for n in (0, 1, 32, 33, 1000):
        attrs = rng.integers(0, 10, size=(1, max(n, 1)), dtype=np.int32)[:, :n]
        attrs = np.ascontiguousarray(attrs)
        bm, cnt = oracle.predicate(attrs, [0], [0], [3]) if n else (np.zeros(0, np.uint32), 0)
        ids = oracle.compact(bm, n)
        assert ids.size == cnt
        if n:
            assert np.array_equal(ids, np.flatnonzero(attrs[0] < 3).astype(np.int32))


# ---------------------------------------------------------------- top-k

def _exact_topk(x, attrs, q, pred, k, metric):
    """Pure-Python twin: exact rationals, explicit loops, full sort."""
    n, d = x.shape
    res = []
    for qi in range(q.shape[0]):
        cand = []
        for i in range(n):
            if not all(lo <= attrs[c, i] < hi for c, lo, hi in zip(pred.cols, pred.lo, pred.hi)):
                continue
            if metric == "l2":
                key = sum((Fraction(float(q[qi, t])) - Fraction(float(x[i, t]))) ** 2
                          for t in range(d))
            else:
                key = -sum(Fraction(float(q[qi, t])) * Fraction(float(x[i, t])) for t in range(d))
            cand.append((key, i))
        cand.sort()
        res.append(cand[:k])
    return res


@pytest.mark.parametrize("metric", ["l2", "ip"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_topk_brute_force_tiny(metric, seed):
    rng = np.random.default_rng(seed)
    n, d, b, k = 48, 6, 4, 7
    x = rng.standard_normal((n, d)).astype(np.float32)
    q = rng.standard_normal((b, d)).astype(np.float32)
    attrs = rng.integers(0, 8, size=(1, n), dtype=np.int32)
    for lo, hi in [(0, 8), (2, 5), (7, 8), (3, 3)]:
        pred = gen.Pred([0], [lo], [hi])
        ids, dist, cnt = oracle.query(x, attrs, q, [pred], k, metric)
        want = _exact_topk(x, attrs, q, pred, k, metric)
        for qi in range(b):
            w = want[qi]
            assert cnt[qi] == sum(lo <= a < hi for a in attrs[0])
            assert list(ids[qi, :len(w)]) == [i for _, i in w]
            for j, (key, _) in enumerate(w):
                ref = float(key) if metric == "l2" else -float(key)
                assert dist[qi, j] == pytest.approx(ref, rel=1e-12, abs=1e-12)
            assert np.all(ids[qi, len(w):] == -1)
            assert np.all(np.isinf(dist[qi, len(w):]))


def test_topk_integer_data_is_exact():
    # small integers: every product and sum is exact in float64
    rng = np.random.default_rng(5)
    n, d, b, k = 60, 8, 5, 10
    x = rng.integers(-9, 10, size=(n, d)).astype(np.float32)
    q = rng.integers(-9, 10, size=(b, d)).astype(np.float32)
    attrs = rng.integers(0, 4, size=(1, n), dtype=np.int32)
    pred = gen.Pred([0], [1], [3])
    for metric in ("l2", "ip"):
        ids, dist, _ = oracle.query(x, attrs, q, [pred], k, metric)
        want = _exact_topk(x, attrs, q, pred, k, metric)
        for qi in range(b):
            got = list(zip(dist[qi], ids[qi]))[:len(want[qi])]
            exp = [((float(kk) if metric == "l2" else -float(kk)), i) for kk, i in want[qi]]
            assert got == exp


def test_topk_line_dataset_closed_form():
    # x_i = i * e1; the k nearest rows to t*e1 among even rows are known
    n, d, k = 1000, 4, 5
    x = np.zeros((n, d), np.float32)
    x[:, 0] = np.arange(n)
    attrs = (np.arange(n) % 2).astype(np.int32)[None, :]
    q = np.zeros((1, d), np.float32)
    q[0, 0] = 500.25
    ids, dist, cnt = oracle.query(x, attrs, q, [gen.Pred([0], [0], [1])], k, "l2")
    assert cnt[0] == 500
    assert list(ids[0]) == [500, 502, 498, 504, 496]
    assert list(dist[0]) == [0.0625, 3.0625, 5.0625, 14.0625, 18.0625]


def test_tie_break_smallest_id():
    n, d = 40, 3
    x = np.ones((n, d), np.float32)
    x[::3] = 2.0                       # rows 0,3,6,.. tie at distance 3, others tie at 0
    attrs = np.zeros((1, n), np.int32)
    q = np.ones((1, d), np.float32)
    ids, dist, _ = oracle.query(x, attrs, q, [gen.pred_all()], 30, "l2")
    others = [i for i in range(n) if i % 3]
    assert list(ids[0, :len(others)]) == others
    assert list(ids[0, len(others):30]) == [i for i in range(n) if i % 3 == 0][:30 - len(others)]


def test_invariants_mixture():
    wl = gen.Workload("t", 3000, 16, 6, 10, "l2", 0.3, 100)
    mix = wl.mixture()
    x = gen.vectors(wl.n, mix)
    q = gen.queries(wl.batch, mix)
    attrs = gen.attributes(wl.n, 1, 100)
    pred = gen.pred_less_than(30)
    ids, dist, cnt = oracle.query(x, attrs, q, [pred], 10, "l2")
    # every returned id satisfies the predicate
    assert np.all(attrs[0, ids] < 30)
    # keys are non-decreasing with rank
    assert np.all(np.diff(dist, axis=1) >= 0)
    # selectivity 100% (no terms) equals the unfiltered search (eq. 2 vs eq. 3)
    full_pred = gen.pred_less_than(100)
    i1, d1, c1 = oracle.query(x, attrs, q, [full_pred], 10, "l2")
    i2, d2, c2 = oracle.query(x, attrs, q, [gen.pred_all()], 10, "l2")
    assert np.array_equal(i1, i2) and np.array_equal(d1, d2)
    assert np.all(c1 == 3000)
    # the filtered result equals the unfiltered search over the selected rows
    sel = np.flatnonzero(attrs[0] < 30)
    i3, d3, _ = oracle.query(x[sel], np.zeros((1, sel.size), np.int32), q, [gen.pred_all()],
                             10, "l2")
    assert np.array_equal(sel[i3], ids) and np.array_equal(d3, dist)


def test_cosine_identity_unit_vectors():
    # on unit vectors ||q-x||^2 = 2 - 2 q.x, so L2 and IP rank alike (Sec. 3.1)
    mix = gen.Mixture(32, seed=3)
    x = gen.vectors(2000, mix, unit=True)
    q = gen.queries(8, mix, unit=True)
    attrs = gen.attributes(2000, 1, 100)
    pred = gen.pred_less_than(50)
    il2, dl2, _ = oracle.query(x, attrs, q, [pred], 10, "l2")
    iip, dip, _ = oracle.query(x, attrs, q, [pred], 10, "ip")
    assert np.array_equal(il2, iip)
    np.testing.assert_allclose(dl2, 2.0 - 2.0 * dip, rtol=1e-5, atol=1e-5)


def test_per_query_predicates_and_k():
    rng = np.random.default_rng(9)
    n, d, b = 300, 5, 6
    x = rng.standard_normal((n, d)).astype(np.float32)
    q = rng.standard_normal((b, d)).astype(np.float32)
    attrs = rng.integers(0, 20, size=(2, n), dtype=np.int32)
    preds = [gen.Pred([0, 1], [i, 0], [i + 8, 10 + i]) for i in range(b)]
    ks = np.array([1, 3, 10, 2, 7, 4], np.int32)
    ids, dist, cnt = oracle.query(x, attrs, q, preds, ks, "l2")
    for qi in range(b):
        want = _exact_topk(x, attrs, q[qi:qi + 1], preds[qi], int(ks[qi]), "l2")[0]
        assert list(ids[qi, :len(want)]) == [i for _, i in want]
        assert np.all(ids[qi, len(want):] == -1)


def test_fewer_rows_than_k_pads():
    x = np.arange(12, dtype=np.float32).reshape(6, 2)
    attrs = np.arange(6, dtype=np.int32)[None, :]
    ids, dist, cnt = oracle.query(x, attrs, x[:1], [gen.Pred([0], [0], [2])], 5, "l2")
    assert cnt[0] == 2
    assert list(ids[0]) == [0, 1, -1, -1, -1]
    assert dist[0, 0] == 0 and dist[0, 1] == 8 and np.all(np.isinf(dist[0, 2:]))


def test_threads_do_not_change_results():
    mix = gen.Mixture(24, seed=4)
    x = gen.vectors(1500, mix)
    q = gen.queries(9, mix)
    attrs = gen.attributes(1500, 1, 100)
    a = oracle.query(x, attrs, q, [gen.pred_less_than(40)], 10, "l2", n_threads=1)
    b = oracle.query(x, attrs, q, [gen.pred_less_than(40)], 10, "l2", n_threads=4)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_pair_dist_matches_query():
    mix = gen.Mixture(16, seed=6)
    x = gen.vectors(500, mix)
    q = gen.queries(3, mix)
    attrs = np.zeros((1, 500), np.int32)
    ids, dist, _ = oracle.query(x, attrs, q, [gen.pred_all()], 4, "l2")
    qi = np.repeat(np.arange(3), 4)
    got = oracle.pair_dist(x, q, qi, ids.ravel(), "l2")
    assert np.array_equal(got, dist.ravel())


def test_sqnorm_closed_form():
    x = np.array([[3, 4, 0, 0], [1, 1, 1, 1], [0, 0, 0, 0]], np.float32)
    assert list(oracle.sqnorm(x)) == [25.0, 4.0, 0.0]
    rng = np.random.default_rng(0)
    y = rng.integers(-100, 100, size=(50, 33)).astype(np.float32)
    assert np.array_equal(oracle.sqnorm(y), (y.astype(np.int64) ** 2).sum(1).astype(np.float64))


# ---------------------------------------------------------------- range (sigma_eps)

def _exact_range(x, attrs, q, pred, eps, metric):
    """Pure-Python twin of the range selection: exact rationals, loops."""
    n, d = x.shape
    res = []
    e = Fraction(float(eps))
    for qi in range(q.shape[0]):
        keep = []
        for i in range(n):
            if not all(lo <= attrs[c, i] < hi for c, lo, hi in zip(pred.cols, pred.lo, pred.hi)):
                continue
            if metric == "l2":
                s = sum((Fraction(float(q[qi, t])) - Fraction(float(x[i, t]))) ** 2 for t in range(d))
                if s <= e:
                    keep.append((s, i))
            else:
                s = sum(Fraction(float(q[qi, t])) * Fraction(float(x[i, t])) for t in range(d))
                if s >= e:
                    keep.append((-s, i))
        keep.sort()
        res.append(keep)
    return res


@pytest.mark.parametrize("metric", ["l2", "ip"])
@pytest.mark.parametrize("seed", [0, 1])
def test_range_brute_force_tiny(metric, seed):
    rng = np.random.default_rng(seed + 10)
    n, d, b = 60, 5, 4
    x = rng.standard_normal((n, d)).astype(np.float32)
    q = rng.standard_normal((b, d)).astype(np.float32)
    attrs = rng.integers(0, 6, size=(1, n), dtype=np.int32)
    for pred in [gen.Pred([0], [1], [5]), gen.pred_all(), gen.Pred([0], [3], [3])]:
        for eps in ([2.0, 6.0, 11.0] if metric == "l2" else [-1.0, 0.5, 2.0]):
            got = oracle.range_query(x, attrs, q, pred, eps, metric)
            want = _exact_range(x, attrs, q, pred, eps, metric)
            for qi in range(b):
                ids, sc = got[qi]
                assert list(ids) == [i for _, i in want[qi]]
                ref = [float(k) if metric == "l2" else -float(k) for k, _ in want[qi]]
                np.testing.assert_allclose(sc, ref, rtol=1e-12, atol=1e-12)


def test_range_infinite_bound_is_the_selection():
    mix = gen.Mixture(12, seed=4)
    x = gen.vectors(3000, mix)
    q = gen.queries(3, mix)
    attrs = gen.attributes(3000, 1, 100, seed=4)
    pred = gen.pred_less_than(37)
    sel = np.flatnonzero(attrs[0] < 37)
    for metric, eps in (("l2", np.inf), ("ip", -np.inf)):
        for ids, _ in oracle.range_query(x, attrs, q, pred, eps, metric):
            assert np.array_equal(np.sort(ids), sel)
    assert all(len(ids) == 0 for ids, _ in oracle.range_query(x, attrs, q, pred, -1.0, "l2"))


def test_range_nested_and_equal_to_topk_at_the_kth_distance():
    mix = gen.Mixture(16, seed=6)
    x = gen.vectors(4000, mix)
    q = gen.queries(5, mix)
    attrs = gen.attributes(4000, 1, 100, seed=6)
    pred = gen.pred_less_than(60)
    ids10, dist10, _ = oracle.query(x, attrs, q, [pred], 11, "l2")
    prev = None
    for eps in (0.5, 1.0, 2.0, 4.0):
        cur = [set(ids) for ids, _ in oracle.range_query(x, attrs, q, pred, eps, "l2")]
        if prev is not None:
            assert all(a <= b for a, b in zip(prev, cur))   # nested for growing eps
        prev = cur
    for qi in range(5):
        assert dist10[qi, 9] < dist10[qi, 10]                # no tie at rank 10
        ids, sc = oracle.range_query(x, attrs, q[qi:qi + 1], pred, dist10[qi, 9], "l2")[0]
        assert list(ids) == list(ids10[qi, :10])             # the top-10, in order
        np.testing.assert_array_equal(sc, dist10[qi, :10])


def test_range_line_dataset_closed_form():
    # x_i = i * e1, q = 500.25 e1: the rows within eps are an interval of i
    n, d = 1000, 3
    x = np.zeros((n, d), np.float32)
    x[:, 0] = np.arange(n)
    attrs = np.zeros((1, n), np.int32)
    q = np.zeros((1, d), np.float32)
    q[0, 0] = 500.25
    ids, sc = oracle.range_query(x, attrs, q, gen.pred_all(), 16.0, "l2")[0]
    assert sorted(ids) == list(range(497, 505))              # (i - 500.25)^2 <= 16
    assert list(sc[:3]) == [0.0625, 0.5625, 1.5625]
    assert list(ids[:3]) == [500, 501, 499]


def test_range_cosine_identity_unit_vectors():
    # ||q-x||^2 = 2 - 2 q.x on unit vectors: q.x >= t  <=>  dist <= 2 - 2t
    mix = gen.Mixture(24, seed=8)
    x = gen.vectors(3000, mix, unit=True)
    q = gen.queries(4, mix, unit=True)
    attrs = gen.attributes(3000, 1, 100, seed=8)
    pred = gen.pred_less_than(70)
    for t in (0.5, 0.8):
        ip = oracle.range_query(x, attrs, q, pred, t, "ip")
        l2 = oracle.range_query(x, attrs, q, pred, 2.0 - 2.0 * t, "l2")
        for (i1, s1), (i2, s2) in zip(ip, l2):
            # rows within rounding of the bound may fall on either side
            a, b = set(i1), set(i2)
            amb = {int(i) for i, s in zip(i1, s1) if abs(s - t) < 1e-5} | \
                  {int(i) for i, s in zip(i2, s2) if abs((2.0 - s) / 2.0 - t) < 1e-5}
            assert (a ^ b) <= amb


# ---------------------------------------------------------------- vector join

def test_join_row_by_row_twin():
    """Each query row that its own predicate selects, in order, with the
    exact filtered top-k of the searched relation (rational twin)."""
    rng = np.random.default_rng(21)
    n, d, m, k = 40, 4, 12, 5
    x = rng.standard_normal((n, d)).astype(np.float32)
    attrs = rng.integers(0, 5, size=(1, n), dtype=np.int32)
    qrel = rng.standard_normal((m, d)).astype(np.float32)
    qattrs = rng.integers(0, 4, size=(2, m), dtype=np.int32)
    qpred = gen.Pred([1, 0], [1, 0], [3, 3])
    rpred = gen.Pred([0], [1], [4])
    for metric in ("l2", "ip"):
        qids, ids, dist = oracle.join_topk(x, attrs, qrel, qattrs, qpred, rpred, k, metric)
        want_q = [i for i in range(m) if 1 <= qattrs[1, i] < 3 and 0 <= qattrs[0, i] < 3]
        assert list(qids) == want_q
        want = _exact_topk(x, attrs, qrel[want_q], rpred, k, metric)
        for j, w in enumerate(want):
            assert list(ids[j, :len(w)]) == [i for _, i in w]
            ref = [float(kk) if metric == "l2" else -float(kk) for kk, _ in w]
            np.testing.assert_allclose(dist[j, :len(w)], ref, rtol=1e-12, atol=1e-12)


def test_join_all_and_none():
    mix = gen.Mixture(8, seed=2)
    x = gen.vectors(500, mix)
    attrs = gen.attributes(500, 1, 10, seed=2)
    qrel = gen.queries(30, mix)
    qattrs = np.arange(30, dtype=np.int32)[None, :]
    rp = gen.pred_less_than(5)
    qids, ids, dist = oracle.join_topk(x, attrs, qrel, qattrs, gen.pred_all(), rp, 7)
    r_ids, r_dist, _ = oracle.query(x, attrs, qrel, [rp], 7)
    assert np.array_equal(qids, np.arange(30)) and np.array_equal(ids, r_ids)
    assert np.array_equal(dist, r_dist)
    qids, ids, _ = oracle.join_topk(x, attrs, qrel, qattrs, gen.Pred([0], [40], [50]), rp, 7)
    assert qids.size == 0 and ids.shape == (0, 7)


# ---------------------------------------------------------------- disjunctions

def test_dnf_rational_twin_and_range_union():
    rng = np.random.default_rng(41)
    n, d, b, k = 70, 4, 3, 6
    x = rng.standard_normal((n, d)).astype(np.float32)
    q = rng.standard_normal((b, d)).astype(np.float32)
    attrs = rng.integers(0, 10, size=(2, n), dtype=np.int32)
    conjs = [gen.Pred([0], [0], [2]), gen.Pred([0, 1], [5, 0], [7, 4]), gen.Pred([1], [9], [10])]
    for metric in ("l2", "ip"):
        ids, dist, cnt = oracle.query_dnf(x, attrs, q, conjs, k, metric)
        ok = [i for i in range(n) if any(all(lo <= attrs[c, i] < hi
                                             for c, lo, hi in zip(p.cols, p.lo, p.hi))
                                         for p in conjs)]
        sub = _exact_topk(x[ok], np.zeros((1, len(ok)), np.int32), q, gen.pred_all(), k, metric)
        for qi in range(b):
            assert cnt[qi] == len(ok)
            assert list(ids[qi, :len(sub[qi])]) == [ok[i] for _, i in sub[qi]]
    # [a, b) or [b, c) selects exactly [a, c)
    mix = gen.Mixture(8, seed=4)
    x2 = gen.vectors(2000, mix)
    q2 = gen.queries(4, mix)
    a2 = gen.attributes(2000, 1, 100, seed=4)
    i1, d1, _ = oracle.query_dnf(x2, a2, q2, [gen.Pred([0], [10], [30]), gen.Pred([0], [30], [55])], 9)
    i2, d2, _ = oracle.query(x2, a2, q2, [gen.Pred([0], [10], [55])], 9)
    assert np.array_equal(i1, i2) and np.array_equal(d1, d2)
