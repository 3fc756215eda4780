"""Comparison of a GPU top-k result with the float64 oracle.

Acceptance rule (the tolerances are written here, once):
  * distances: |d_gpu - d_ref| <= 1e-4 * scale, scale = max(|d_ref|, 1e-30)
    for L2 (squared) and max(|d_ref|, ||q|| ||x||) for IP;
  * ids: wherever the float64 gap between ranks j and j+1 exceeds 1e-5
    relative (same scale), the set of the first j+1 ids must equal the
    oracle's -- in particular the whole top-k set when the k-th/(k+1)-th gap
    does;
  * every returned id must be a valid answer: it satisfies the predicate and
    its exact (float64) distance is within 1e-5 relative of the oracle's
    distance at the same rank (a near-tie may swap equal-enough rows);
  * padding (id -1, +inf) exactly where the oracle pads.
"""
import numpy as np

import oracle

DIST_RTOL = 1e-4
GAP_RTOL = 1e-5


def _scale(ref, metric, qnorm=None, xnorm=None):
    if metric == "l2":
        return np.maximum(np.abs(ref), 1e-30)
    return np.maximum(np.abs(ref), qnorm * xnorm if qnorm is not None else 1.0)


def check_topk(x, q, attrs, preds, k, metric, gids, gdist, rid, rdist, rcount):
    """rid/rdist: oracle result with k_max >= max(k) + 1 (for the gap)."""
    b = q.shape[0]
    karr = np.broadcast_to(np.atleast_1d(k), (b,))
    gids = np.asarray(gids)
    gdist = np.asarray(gdist, dtype=np.float64)
    qn = np.sqrt((q.astype(np.float64) ** 2).sum(1))
    for i in range(b):
        kk = int(karr[i])
        pred = preds[0] if len(preds) == 1 else preds[i]
        nv = int(min(kk, rcount[i]))
        # padding
        assert np.all(gids[i, nv:kk] == -1), f"q{i}: expected padding after {nv}"
        assert np.all(np.isinf(gdist[i, nv:kk])), f"q{i}: expected +inf padding"
        if nv == 0:
            continue
        g, gd = gids[i, :nv], gdist[i, :nv]
        r, rd = rid[i, :nv], rdist[i, :nv]
        assert np.all(g >= 0), f"q{i}: missing results"
        assert len(set(g.tolist())) == nv, f"q{i}: duplicate ids"
        # predicate satisfied
        for c, lo, hi in zip(pred.cols, pred.lo, pred.hi):
            a = attrs[c, g]
            assert np.all((lo <= a) & (a < hi)), f"q{i}: id violates predicate"
        xn = np.sqrt((x[g].astype(np.float64) ** 2).sum(1)) if metric == "ip" else None
        sc = _scale(rd, metric, qn[i], xn)
        # distances within tolerance of the oracle's at the same rank
        err = np.abs(gd - rd)
        assert np.all(err <= DIST_RTOL * sc), \
            f"q{i}: distance error {np.max(err / sc):.3g} relative"
        # exact distance of each returned id matches the rank's reference
        ex = oracle.pair_dist(x, q, np.full(nv, i), g, metric)
        assert np.all(np.abs(ex - rd) <= GAP_RTOL * sc), f"q{i}: returned id is not a valid top-k row"
        # ids identical wherever the gap after rank j exceeds GAP_RTOL
        nxt = rdist[i, 1:nv + 1] if rcount[i] > nv else np.append(rdist[i, 1:nv], np.inf)
        gap = np.abs(nxt - rd) > GAP_RTOL * sc
        for j in np.flatnonzero(gap):
            assert set(g[:j + 1].tolist()) == set(r[:j + 1].tolist()), \
                f"q{i}: top-{j + 1} set differs from the oracle"


def recall(gids, rid, k):
    b = gids.shape[0]
    hit = 0
    tot = 0
    for i in range(b):
        r = set(int(v) for v in rid[i, :k] if v >= 0)
        g = set(int(v) for v in gids[i, :k] if v >= 0)
        hit += len(r & g)
        tot += len(r)
    return hit / max(tot, 1)
