"""CPU oracle for exact filtered top-k vector search (float64, full sort).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library
(``paper_2403_15807_gb300``) never does, and this package never imports it.

The arithmetic lives in ``vrs_oracle.c`` (plain C, float64); this module
compiles it with gcc on first use and marshals numpy arrays.  See the C file
for the passage of the paper each routine follows.

Parity status per function (what pins it, in tests/test_oracle_*.py):
  predicate / compact  -- closed form (attr = i mod 100), brute force, popcount
  range_query          -- pure-Python brute force on tiny inputs, eps = +inf
                          equals the selection, nested results for growing
                          eps, the top-k set at eps = k-th distance, line
                          dataset closed form, L2/IP identity on unit vectors
  query_dnf            -- OR of predicate bitmaps, then query: pinned by a
                          rational twin and by [a,b) | [b,c) == [a,c)
  join_topk            -- the composition of predicate + compact + query:
                          pinned through them and by a row-by-row twin
  query (top-k)        -- pure-Python brute force on tiny inputs, exact
                          integer-valued data, line dataset closed form,
                          invariants (s=100% equals unfiltered, monotone keys,
                          every id satisfies the predicate), L2/IP identity on
                          unit vectors, duplicate rows for the tie-break
  sqnorm               -- closed form on integer rows
  bf16 / e4m3 codecs   -- format constants, all 256 E4M3 codes, torch's
                          float8_e4m3fn / bfloat16 conversions
  mlp / adam           -- central finite differences, closed-form linear case,
                          hand-computed Adam step
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vrs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile vrs_oracle.c into liboracle.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i32, i64, f32, f64 = C.c_int32, C.c_int64, C.c_float, C.c_double
            P = C.c_void_p
            L.vrs_oracle_predicate.restype = i64
            L.vrs_oracle_predicate.argtypes = [P, i64, i32, P, P, P, P]
            L.vrs_oracle_compact.restype = i64
            L.vrs_oracle_compact.argtypes = [P, i64, P]
            L.vrs_oracle_query.restype = C.c_int
            L.vrs_oracle_query.argtypes = [P, i64, i32, P, P, i32, P, P, P, P, i32, P, i32, i32,
                                           i32, P, P, P, i32]
            L.vrs_oracle_range.restype = i64
            L.vrs_oracle_range.argtypes = [P, i64, i32, P, P, i32, i32, P, P, P, f64, i32, P, P,
                                           P, i64]
            L.vrs_oracle_pair_dist.restype = None
            L.vrs_oracle_pair_dist.argtypes = [P, i32, P, P, P, i64, i32, P]
            L.vrs_oracle_sqnorm.restype = None
            L.vrs_oracle_sqnorm.argtypes = [P, i64, i32, P]
            L.vrs_oracle_bf16_encode.restype = C.c_uint16
            L.vrs_oracle_bf16_encode.argtypes = [f32]
            L.vrs_oracle_bf16_decode.restype = f32
            L.vrs_oracle_bf16_decode.argtypes = [C.c_uint16]
            L.vrs_oracle_e4m3_encode.restype = C.c_uint8
            L.vrs_oracle_e4m3_encode.argtypes = [f32]
            L.vrs_oracle_e4m3_decode.restype = f64
            L.vrs_oracle_e4m3_decode.argtypes = [C.c_uint8]
            L.vrs_oracle_e4m3_rows.restype = None
            L.vrs_oracle_e4m3_rows.argtypes = [P, i64, i32, P, P]
            L.vrs_oracle_mlp_nparams.restype = i64
            L.vrs_oracle_mlp_nparams.argtypes = [i32, i32, i32, i32]
            L.vrs_oracle_mlp.restype = f64
            L.vrs_oracle_mlp.argtypes = [P, i32, i32, i32, i32, P, i64, P, P, P, P]
            L.vrs_oracle_adam.restype = None
            L.vrs_oracle_adam.argtypes = [P, P, P, P, i64, i32, f64, f64, f64, f64]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def predicate(attrs: np.ndarray, cols, lo, hi):
    """Bitmap (uint32 words, LSB-first) and |S| for a conjunction of [lo,hi)."""
    attrs = _c(np.atleast_2d(attrs), np.int32)
    n = attrs.shape[1]
    cols, lo, hi = _c(cols, np.int32), _c(lo, np.int32), _c(hi, np.int32)
    bm = np.zeros((n + 31) // 32, dtype=np.uint32)
    cnt = lib().vrs_oracle_predicate(_p(attrs), n, len(cols), _p(cols), _p(lo), _p(hi), _p(bm))
    return bm, int(cnt)


def compact(bitmap: np.ndarray, n: int) -> np.ndarray:
    bitmap = _c(bitmap, np.uint32)
    ids = np.empty(max(n, 1), dtype=np.int32)
    c = lib().vrs_oracle_compact(_p(bitmap), n, _p(ids))
    return ids[:c].copy()


def query(x, attrs, q, preds, k, metric: str = "l2", k_max=None, n_threads: int = 1):
    """Exact filtered top-k.

    preds: list of gen.Pred (one shared, or one per query); k: int or per-query
    array.  Returns (ids int64 [b x k_max], dist float64 [b x k_max],
    count int64 [b]); L2 distances are squared, IP values are q.x.
    """
    from gen import pack_preds  # input marshalling only
    x = _c(x, np.float32)
    q = _c(np.atleast_2d(q), np.float32)
    attrs = _c(np.atleast_2d(attrs), np.int32)
    n, d = x.shape
    b = q.shape[0]
    assert q.shape[1] == d
    off, cols, lo, hi = pack_preds(preds)
    karr = _c(np.atleast_1d(k), np.int32)
    if k_max is None:
        k_max = int(karr.max()) if karr.size else 0
    ids = np.empty((b, k_max), dtype=np.int64)
    dist = np.empty((b, k_max), dtype=np.float64)
    cnt = np.empty(b, dtype=np.int64)
    m = 0 if metric == "l2" else 1
    rc = lib().vrs_oracle_query(_p(x), n, d, _p(attrs), _p(q), b, _p(off), _p(cols), _p(lo),
                                _p(hi), len(preds), _p(karr), karr.size, k_max, m, _p(ids),
                                _p(dist), _p(cnt), n_threads)
    if rc != 0:
        raise MemoryError("oracle worker could not allocate")
    return ids, dist, cnt


def range_query(x, attrs, q, pred, eps: float, metric: str = "l2"):
    """Exact filtered range selection with one shared predicate.

    Query i keeps every selected row with squared L2 distance <= eps, or
    q.x >= eps for IP.  Returns a list of (ids int64, score float64) per
    query, in (score, id) order (ascending distance; descending q.x).
    """
    x = _c(x, np.float32)
    q = _c(np.atleast_2d(q), np.float32)
    attrs = _c(np.atleast_2d(attrs), np.int32)
    n, d = x.shape
    b = q.shape[0]
    assert q.shape[1] == d
    cols, lo, hi = _c(pred.cols, np.int32), _c(pred.lo, np.int32), _c(pred.hi, np.int32)
    m = 0 if metric == "l2" else 1
    off = np.zeros(b + 1, dtype=np.int64)
    args = (_p(x), n, d, _p(attrs), _p(q), b, len(pred.cols), _p(cols), _p(lo), _p(hi),
            float(eps), m, _p(off))
    total = lib().vrs_oracle_range(*args, None, None, 0)
    if total < 0:
        raise MemoryError("oracle could not allocate")
    ids = np.empty(max(total, 1), dtype=np.int64)
    dist = np.empty(max(total, 1), dtype=np.float64)
    lib().vrs_oracle_range(*args, _p(ids), _p(dist), total)
    return [(ids[off[i]:off[i + 1]].copy(), dist[off[i]:off[i + 1]].copy()) for i in range(b)]


def query_dnf(x, attrs, q, conjs, k: int, metric: str = "l2", n_threads: int = 8):
    """Exact top-k under a disjunction of conjunctions (one shared predicate
    in disjunctive normal form): a row qualifies when any conjunction holds.
    The selection is the OR of each conjunction's bitmap; the search is
    `query` over it.  Returns (ids, dist, count) like `query`."""
    attrs = _c(np.atleast_2d(attrs), np.int32)
    n = attrs.shape[1]
    words = np.zeros((n + 31) // 32, dtype=np.uint32)
    for c in conjs:
        bm, _ = predicate(attrs, c.cols, c.lo, c.hi)
        words |= bm
    sel = np.zeros((1, n), np.int32)
    sel[0, compact(words, n)] = 1
    from gen import Pred  # input marshalling only
    return query(x, sel, q, [Pred([0], [1], [2])], k, metric, n_threads=n_threads)


def join_topk(x, attrs, qrel, qattrs, qpred, rpred, k: int, metric: str = "l2"):
    """Vector join: the query rows of (qrel, qattrs) that qpred selects, in
    ascending order, each with its exact filtered top-k over (x, attrs) under
    rpred -- the composition sigma_qpred(Q), then the top-k of each selected
    query.  Returns (qids int64, ids [nq x k], dist [nq x k])."""
    qrel = _c(np.atleast_2d(qrel), np.float32)
    m = qrel.shape[0]
    qattrs = np.zeros((0, m), np.int32) if qattrs is None else _c(np.atleast_2d(qattrs), np.int32)
    if qpred.n_terms:
        bm, _ = predicate(qattrs, qpred.cols, qpred.lo, qpred.hi)
    else:
        bm, _ = predicate(np.zeros((1, m), np.int32), [], [], [])
    qids = compact(bm, m).astype(np.int64)
    if qids.size == 0:
        return qids, np.empty((0, k), np.int64), np.empty((0, k), np.float64)
    ids, dist, _ = query(x, attrs, qrel[qids], [rpred], k, metric, n_threads=8)
    return qids, ids, dist


def pair_dist(x, q, qi, xi, metric: str = "l2") -> np.ndarray:
    """Exact float64 distance (L2 squared) or q.x (IP) for (query, row) pairs."""
    x = _c(x, np.float32)
    q = _c(np.atleast_2d(q), np.float32)
    qi, xi = _c(qi, np.int64), _c(xi, np.int64)
    out = np.empty(qi.shape[0], dtype=np.float64)
    lib().vrs_oracle_pair_dist(_p(x), x.shape[1], _p(q), _p(qi), _p(xi), qi.shape[0],
                               0 if metric == "l2" else 1, _p(out))
    return out


def sqnorm(x) -> np.ndarray:
    x = _c(x, np.float32)
    out = np.empty(x.shape[0], dtype=np.float64)
    lib().vrs_oracle_sqnorm(_p(x), x.shape[0], x.shape[1], _p(out))
    return out


def bf16_encode(x) -> np.ndarray:
    L = lib()
    flat = np.asarray(x, dtype=np.float32).ravel()
    return np.array([L.vrs_oracle_bf16_encode(float(v)) for v in flat],
                    dtype=np.uint16).reshape(np.shape(x))


def bf16_decode(h) -> np.ndarray:
    L = lib()
    flat = np.asarray(h, dtype=np.uint16).ravel()
    return np.array([L.vrs_oracle_bf16_decode(int(v)) for v in flat],
                    dtype=np.float32).reshape(np.shape(h))


def e4m3_encode(x) -> np.ndarray:
    L = lib()
    flat = np.asarray(x, dtype=np.float32).ravel()
    return np.array([L.vrs_oracle_e4m3_encode(float(v)) for v in flat],
                    dtype=np.uint8).reshape(np.shape(x))


def e4m3_decode(c) -> np.ndarray:
    L = lib()
    flat = np.asarray(c, dtype=np.uint8).ravel()
    return np.array([L.vrs_oracle_e4m3_decode(int(v)) for v in flat],
                    dtype=np.float64).reshape(np.shape(c))


def e4m3_rows(x):
    """Per-row scaled E4M3 copy: (codes uint8 [n x d], scale float32 [n])."""
    x = _c(x, np.float32)
    n, d = x.shape
    codes = np.empty((n, d), dtype=np.uint8)
    scale = np.empty(n, dtype=np.float32)
    lib().vrs_oracle_e4m3_rows(_p(x), n, d, _p(codes), _p(scale))
    return codes, scale


MLP_SHAPE = (6, 64, 64, 3)


def mlp_nparams(shape=MLP_SHAPE) -> int:
    return int(lib().vrs_oracle_mlp_nparams(*shape))


def mlp(params, X, T=None, mask=None, shape=MLP_SHAPE, want_grad: bool = False):
    """float64 forward (and backward) of the 6-64-64-3 ReLU plan model.

    Returns (Y [m x out], loss, grad or None)."""
    P = _c(params, np.float64)
    X = _c(np.atleast_2d(X), np.float64)
    m = X.shape[0]
    Y = np.empty((m, shape[3]), dtype=np.float64)
    Tt = None if T is None else _c(T, np.float64)
    Mm = None if mask is None else _c(mask, np.float64)
    g = np.empty(P.size, dtype=np.float64) if want_grad else None
    loss = lib().vrs_oracle_mlp(_p(P), *shape, _p(X), m, _p(Tt), _p(Mm), _p(Y), _p(g))
    return Y, float(loss), g


def adam(params, grad, m1, m2, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays."""
    for a in (params, grad, m1, m2):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().vrs_oracle_adam(_p(params), _p(grad), _p(m1), _p(m2), params.size, t, lr, beta1,
                          beta2, eps)
