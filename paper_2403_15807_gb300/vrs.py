"""Thin ctypes binding of libvrs.so (include/vrs.h).

Argument marshalling only: every step of the search runs in the library's
CUDA kernels.  Functions keep the C names (``vrs_create``, ``vrs_query`` ...)
and take numpy arrays (host memory) or torch CUDA tensors (device memory);
a ``Engine`` class wraps them for convenience.  There is no CPU fallback:
if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, NamedTuple, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvrs.so")

VRS_OK, VRS_EINVAL, VRS_ENOMEM, VRS_ECUDA, VRS_ETIMEOUT, VRS_ESTATE, VRS_EIO = \
    0, -1, -2, -3, -4, -5, -6
VRS_EINTERNAL, VRS_ESIZE = -7, -8
VRS_L2, VRS_IP = 0, 1
VRS_F32, VRS_BF16, VRS_FP8E4M3 = 0, 1, 2
VRS_PLAN_AUTO, VRS_PLAN_GEMV, VRS_PLAN_COMPACT_GEMM, VRS_PLAN_MASK_GEMM = -1, 0, 1, 2
VRS_PLAN_CELLS = 3
VRS_OPT_KPRIME_FACTOR, VRS_OPT_RERANK, VRS_OPT_GRID_CTAS, VRS_OPT_PROFILE = 0, 1, 2, 3
VRS_OPT_FUSED_SCAN, VRS_OPT_BATCHED, VRS_OPT_GRAPH, VRS_OPT_TMA = 4, 5, 6, 7
VRS_OPT_DENSE_KEYS = 8
VRS_OPT_SELECT_CAP = 9
VRS_OPT_STAGED_SCAN = 10
VRS_OPT_TENSOR_GEMV = 11
VRS_OPT_SEED_BOUND = 12
VRS_OPT_PAIR_COPY = 13
VRS_OPT_WAIT_TEST = 14
VRS_OPT_CERT_SAMPLE = 15
VRS_OPT_CELL_PLAN = 16
VRS_OPT_ZERO_COPY = 17
VRS_CERT_FFMA, VRS_CERT_TF32X3, VRS_CERT_BF16X3, VRS_CERT_BF16, VRS_CERT_E4M3 = 0, 1, 2, 3, 4
STAGES = ("prepare", "predicate", "offsets", "compact", "distance", "merge")
VRS_N_STAGES = len(STAGES)

_STATUS = {VRS_EINVAL: "EINVAL", VRS_ENOMEM: "ENOMEM", VRS_ECUDA: "ECUDA",
           VRS_ETIMEOUT: "ETIMEOUT", VRS_ESTATE: "ESTATE", VRS_EIO: "EIO",
           VRS_EINTERNAL: "EINTERNAL", VRS_ESIZE: "ESIZE"}

# Every symbol include/vrs.h declares, with (restype, argtypes).
_P = C.c_void_p
_I32, _I64, _U32 = C.c_int32, C.c_int64, C.c_uint32
SIGNATURES = {
    "vrs_version": (C.c_char_p, []),
    "vrs_last_error": (C.c_char_p, []),
    "vrs_create": (C.c_int, [C.c_int, C.POINTER(_P)]),
    "vrs_destroy": (C.c_int, [_P]),
    "vrs_load_vectors": (C.c_int, [_P, _P, _I64, _I32, C.c_int, _U32, C.c_int, _P]),
    "vrs_load_attribute": (C.c_int, [_P, _I32, _P, _I64, C.c_int, _P]),
    "vrs_float_key": (_I32, [C.c_float]),
    "vrs_load_attribute_f32": (C.c_int, [_P, _I32, _P, _I64, C.c_int, _P]),
    "vrs_build_grid": (C.c_int, [_P, _I32, _I32, _I32, _P]),
    "vrs_query": (C.c_int, [_P, _P, _I32, _I32, _P, _I32, _P, _I32, _I32, C.c_int, C.c_int,
                            _P, _P, C.c_int, _P]),
    "vrs_range_query": (C.c_int, [_P, _P, _I32, _I32, _P, C.c_float, C.c_int, _I64, _P, _P, _P,
                                  C.c_int, _P]),
    "vrs_query_dnf": (C.c_int, [_P, _P, _I32, _I32, _P, _I32, _I32, C.c_int, C.c_int, _P, _P,
                                C.c_int, _P]),
    "vrs_join_topk": (C.c_int, [_P, _P, _I64, _I32, _P, _I32, _P, _P, _I32, C.c_int, C.c_int,
                                _I64, C.POINTER(_I64), _P, _P, _P, C.c_int, _P]),
    "vrs_eval_predicate": (C.c_int, [_P, _P, _P, C.POINTER(_I64), C.c_int, _P]),
    "vrs_select_ids": (C.c_int, [_P, _P, _P, C.POINTER(_I64), C.c_int, _P]),
    "vrs_probe_gather": (C.c_int, [_P, _I64, _I64, _P, _I64, _P, _P]),
    "vrs_get_norms": (C.c_int, [_P, _P, C.c_int, _P]),
    "vrs_get_encoded": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "vrs_set_plan": (C.c_int, [_P, C.c_int]),
    "vrs_last_plan": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "vrs_set_option": (C.c_int, [_P, C.c_int, _I64]),
    "vrs_planner_load": (C.c_int, [_P, C.c_char_p]),
    "vrs_last_profile": (C.c_int, [_P, _P, C.POINTER(_I32), C.POINTER(_I64)]),
    "vrs_query_noalloc": (C.c_int, [_P, _I64, _I32, _P, _I32, _P, _P, _I32, _I32, C.c_int, _P,
                                    _P, _P, _P]),
    "vrs_merge_shards": (C.c_int, [_P, _P, _I32, _I32, _I32, _P, C.c_int, _P, _P, C.c_int, _P]),
    "vrs_last_cert": (C.c_int, [_P, _P]),
    "vrs_cert_bound": (C.c_float, [_I32, _I32, C.c_int, C.c_float, C.c_float, C.c_float,
                                   C.c_float]),
    "vrs_mlp_nparams": (C.c_int32, []),
    "vrs_mlp_forward": (C.c_int, [_P, _P, _I64, _I32, _P]),
    "vrs_mlp_grad": (C.c_int, [_P, _P, _P, _P, _I64, _P, _P]),
    "vrs_mlp_train": (C.c_int, [_P, _P, _P, _P, _I64, _I32, C.c_float, _P]),
}


class VrsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class vrs_range(C.Structure):
    _fields_ = [("col", C.c_int32), ("lo", C.c_int32), ("hi", C.c_int32)]


class vrs_pred(C.Structure):
    _fields_ = [("n_terms", C.c_int32), ("terms", C.POINTER(vrs_range))]


_lib = None


def load(path: str = LIB_PATH):
    """Load libvrs.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing; build it with paper_2403_15807_gb300.build")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int):
    if st != VRS_OK:
        raise VrsError(st, load().vrs_last_error().decode())


def _ptr(a) -> tuple:
    """(pointer, on_device) for a numpy array or a torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous, "arrays must be C-contiguous"
        return a.ctypes.data_as(C.c_void_p), 0
    # torch tensor
    assert a.is_contiguous(), "tensors must be contiguous"
    return C.c_void_p(a.data_ptr()), int(a.is_cuda)


def _stream(stream) -> Optional[C.c_void_p]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)   # torch.cuda.Stream


class Pred(NamedTuple):
    """A conjunction of half-open ranges lo[t] <= attr[cols[t]] < hi[t]
    (no terms: every row).  Any object with cols / lo / hi lists will do."""
    cols: List[int]
    lo: List[int]
    hi: List[int]


class PredArray:
    """Predicates marshalled once into the C layout (vrs_pred[] pointing
    into one vrs_range[] block); vrs_query accepts it in place of a list."""

    _DT = np.dtype([("n_terms", "<i4"), ("pad", "<i4"), ("terms", "<u8")])

    def __init__(self, preds):
        n = len(preds)
        nt = np.fromiter((len(p.cols) for p in preds), dtype=np.int64, count=n)
        off = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(nt, out=off[1:])
        tot = int(off[-1])
        self.terms = np.zeros((max(tot, 1), 3), dtype=np.int32)
        if tot:
            for f, name in enumerate(("cols", "lo", "hi")):
                self.terms[:tot, f] = np.fromiter(
                    (int(v) for p in preds for v in getattr(p, name)), dtype=np.int64, count=tot)
        self.arr = np.zeros(n, dtype=self._DT)
        self.arr["n_terms"] = nt
        self.arr["terms"] = self.terms.ctypes.data + off[:-1] * 12
        self.n = n
        self.ptr = self.arr.ctypes.data_as(C.POINTER(vrs_pred))

    def __len__(self):
        return self.n


def make_preds(preds) -> tuple:
    """(pointer to a vrs_pred array, the objects that keep it alive) from
    objects with cols/lo/hi lists, or from a PredArray."""
    pa = preds if isinstance(preds, PredArray) else PredArray(preds)
    return pa.ptr, pa


def vrs_version() -> str:
    return load().vrs_version().decode()


def vrs_last_error() -> str:
    return load().vrs_last_error().decode()


def vrs_create(device: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().vrs_create(device, C.byref(h)))
    return h


def vrs_destroy(h) -> None:
    _check(load().vrs_destroy(h))


def vrs_load_vectors(h, x, dtype: int = VRS_F32, copies: int = 1 << VRS_F32, stream=None):
    p, dev = _ptr(x)
    n, d = x.shape
    _check(load().vrs_load_vectors(h, p, n, d, dtype, copies, dev, _stream(stream)))


def vrs_load_attribute(h, col: int, a, stream=None):
    p, dev = _ptr(a)
    _check(load().vrs_load_attribute(h, col, p, a.shape[-1], dev, _stream(stream)))


def vrs_float_key(v: float) -> int:
    """Order-preserving int32 image of a float attribute value."""
    return int(load().vrs_float_key(C.c_float(v)))


def float_range(col: int, lo: float, hi: float) -> tuple:
    """(col, lo, hi) of the int32 range selecting lo <= a < hi on a float
    column loaded with vrs_load_attribute_f32 (for a Pred's terms)."""
    return col, vrs_float_key(lo), vrs_float_key(hi)


def vrs_load_attribute_f32(h, col: int, a, stream=None):
    p, dev = _ptr(a)
    _check(load().vrs_load_attribute_f32(h, col, p, a.shape[-1], dev, _stream(stream)))


def vrs_build_grid(h, col0: int, col1: int, bins: int = 0, stream=None):
    _check(load().vrs_build_grid(h, col0, col1, bins, _stream(stream)))


def vrs_query(h, q, preds, k, k_max: Optional[int] = None, metric: int = VRS_L2,
              compute: int = VRS_F32, out_ids=None, out_dist=None, stream=None):
    """Filtered top-k.  With host q, returns numpy (ids, dist); with device q
    the outputs are torch tensors on q's device (or the ones passed in)."""
    karr = np.ascontiguousarray(np.atleast_1d(k), dtype=np.int32)
    if k_max is None:
        k_max = int(karr.max())
    b, d = q.shape
    parr, keep = make_preds(preds)
    qp, qdev = _ptr(q)
    if out_ids is None:
        if qdev:
            import torch
            out_ids = torch.empty((b, k_max), dtype=torch.int64, device=q.device)
            out_dist = torch.empty((b, k_max), dtype=torch.float32, device=q.device)
        else:
            out_ids = np.empty((b, k_max), dtype=np.int64)
            out_dist = np.empty((b, k_max), dtype=np.float32)
    ip, _ = _ptr(out_ids)
    dp, _ = _ptr(out_dist)
    _check(load().vrs_query(h, qp, b, d, parr, len(preds), karr.ctypes.data_as(C.c_void_p),
                            karr.size, k_max, metric, compute, ip, dp, qdev, _stream(stream)))
    return out_ids, out_dist


def vrs_range_query(h, q, pred, eps: float, metric: int = VRS_L2, cap: Optional[int] = None,
                    stream=None):
    """Filtered range search with one shared predicate: every selected row
    with squared L2 distance <= eps (IP: q.x >= eps).  Returns (offsets,
    ids, dist): numpy offsets [b + 1]; query i's results are ids / dist
    [offsets[i]:offsets[i + 1]] (numpy for host q, torch tensors on q's
    device for device q).  A first capacity guess that proves too small is
    retried once at the size the library reports."""
    b, d = q.shape
    parr, keep = make_preds([pred])
    qp, qdev = _ptr(q)
    offs = np.zeros(b + 1, dtype=np.int64)
    cap = 4096 * b if cap is None else int(cap)
    while True:
        m = max(cap, 1)
        if qdev:
            import torch
            ids = torch.empty(m, dtype=torch.int64, device=q.device)
            dist = torch.empty(m, dtype=torch.float32, device=q.device)
        else:
            ids = np.empty(m, dtype=np.int64)
            dist = np.empty(m, dtype=np.float32)
        ip, _ = _ptr(ids)
        dp, _ = _ptr(dist)
        st = load().vrs_range_query(h, qp, b, d, parr, C.c_float(eps), metric, cap,
                                    offs.ctypes.data_as(C.c_void_p), ip, dp, qdev,
                                    _stream(stream))
        if st == VRS_ESIZE and int(offs[-1]) > cap:
            cap = int(offs[-1])
            continue
        _check(st)
        total = int(offs[-1])
        return offs, ids[:total], dist[:total]


def in_list(col: int, values) -> list:
    """The conjunctions of the IN-list `attr[col] in values` (one per value),
    for vrs_query_dnf."""
    return [Pred([col], [int(v)], [int(v) + 1]) for v in values]


def vrs_query_dnf(h, q, conjs, k: int, metric: int = VRS_L2, compute: int = VRS_F32,
                  out_ids=None, out_dist=None, stream=None):
    """Filtered top-k under a disjunction of conjunctions (shared by the
    batch).  Host q gives numpy results; device q gives tensors on its device."""
    b, d = q.shape
    carr, keep = make_preds(conjs)
    qp, qdev = _ptr(q)
    if out_ids is None:
        if qdev:
            import torch
            out_ids = torch.empty((b, k), dtype=torch.int64, device=q.device)
            out_dist = torch.empty((b, k), dtype=torch.float32, device=q.device)
        else:
            out_ids = np.empty((b, k), dtype=np.int64)
            out_dist = np.empty((b, k), dtype=np.float32)
    ip, _ = _ptr(out_ids)
    dp, _ = _ptr(out_dist)
    _check(load().vrs_query_dnf(h, qp, b, d, carr, len(conjs), k, metric, compute, ip, dp, qdev,
                                _stream(stream)))
    return out_ids, out_dist


def vrs_join_topk(h, qrel, qattrs, qpred, rpred, k: int, metric: int = VRS_L2,
                  compute: int = VRS_F32, cap: Optional[int] = None, stream=None):
    """Vector join: the query rows of relation (qrel [m x d], qattrs
    [q_cols x m]) that qpred selects, each with its filtered top-k over the
    loaded rows (rpred).  Returns (qids numpy int64 [nq], ids [nq x k],
    dist [nq x k]); ids / dist are numpy for host inputs, torch tensors on
    qrel's device for device inputs."""
    m, d = qrel.shape
    qp, qdev = _ptr(qrel)
    if qattrs is None:
        ap, q_cols = None, 0
    else:
        ap, adev = _ptr(qattrs)
        assert adev == qdev, "qrel and qattrs must both be on the host or both on the device"
        q_cols = 1 if qattrs.ndim == 1 else qattrs.shape[0]
    qarr, keep1 = make_preds([qpred])
    rarr, keep2 = make_preds([rpred])
    cap = m if cap is None else int(cap)
    nq = C.c_int64()
    m_out = max(cap, 1)
    qids = np.empty(m_out, dtype=np.int64)
    if qdev:
        import torch
        ids = torch.empty((m_out, k), dtype=torch.int64, device=qrel.device)
        dist = torch.empty((m_out, k), dtype=torch.float32, device=qrel.device)
    else:
        ids = np.empty((m_out, k), dtype=np.int64)
        dist = np.empty((m_out, k), dtype=np.float32)
    ip, _ = _ptr(ids)
    dp, _ = _ptr(dist)
    _check(load().vrs_join_topk(h, qp, m, d, ap, q_cols, qarr, rarr, k, metric, compute, cap,
                                C.byref(nq), qids.ctypes.data_as(C.c_void_p), ip, dp, qdev,
                                _stream(stream)))
    n = nq.value
    return qids[:n].copy(), ids[:n], dist[:n]


def vrs_eval_predicate(h, pred, n: int, stream=None):
    parr, keep = make_preds([pred])
    bm = np.empty((n + 31) // 32, dtype=np.uint32)
    cnt = C.c_int64()
    _check(load().vrs_eval_predicate(h, parr, bm.ctypes.data_as(C.c_void_p), C.byref(cnt), 0,
                                     _stream(stream)))
    return bm, cnt.value


def vrs_select_ids(h, pred, n: int, stream=None):
    parr, keep = make_preds([pred])
    ids = np.empty(max(n, 1), dtype=np.int32)
    cnt = C.c_int64()
    _check(load().vrs_select_ids(h, parr, ids.ctypes.data_as(C.c_void_p), C.byref(cnt), 0,
                                 _stream(stream)))
    return ids[:cnt.value].copy()


def vrs_probe_gather(rows, ids, out, stream=None):
    """Measurement hook: read rows[ids] in full (device tensors: rows 2-D
    row-major, ids int32, out a float32 scalar the sum is added to)."""
    row_bytes = rows.stride(0) * rows.element_size()
    _check(load().vrs_probe_gather(C.c_void_p(rows.data_ptr()), rows.shape[0], row_bytes,
                                   C.c_void_p(ids.data_ptr()), ids.numel(),
                                   C.c_void_p(out.data_ptr()), _stream(stream)))


def vrs_get_norms(h, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float32)
    _check(load().vrs_get_norms(h, out.ctypes.data_as(C.c_void_p), 0, None))
    return out


def vrs_get_encoded(h, dtype: int, n: int, d: int):
    npdt = {VRS_F32: np.float32, VRS_BF16: np.uint16, VRS_FP8E4M3: np.uint8}[dtype]
    codes = np.empty((n, d), dtype=npdt)
    scale = np.empty(n, dtype=np.float32) if dtype == VRS_FP8E4M3 else None
    _check(load().vrs_get_encoded(h, dtype, codes.ctypes.data_as(C.c_void_p),
                                  None if scale is None else scale.ctypes.data_as(C.c_void_p),
                                  0, None))
    return codes, scale


def vrs_set_plan(h, plan: int):
    _check(load().vrs_set_plan(h, plan))


def vrs_last_plan(h) -> int:
    v = C.c_int()
    _check(load().vrs_last_plan(h, C.byref(v)))
    return v.value


def vrs_set_option(h, key: int, value: int):
    _check(load().vrs_set_option(h, key, value))


def vrs_last_profile(h):
    """(stage_ms dict, kernel launches, selected rows) of the last query."""
    ms = np.zeros(VRS_N_STAGES, dtype=np.float32)
    nl = C.c_int32()
    sel = C.c_int64()
    _check(load().vrs_last_profile(h, ms.ctypes.data_as(C.c_void_p), C.byref(nl), C.byref(sel)))
    return dict(zip(STAGES, ms.tolist())), nl.value, sel.value


def vrs_merge_shards(ids, dist, row_offset, metric: int = VRS_L2, out_ids=None, out_dist=None,
                     stream=None):
    """k best of the shards' top-k lists: ids/dist [n_shards x batch x k]
    (numpy, or torch CUDA tensors), row_offset [n_shards] global id of each
    shard's row 0.  Returns (ids, dist) [batch x k] with global ids."""
    w, b, k = ids.shape
    offs = np.ascontiguousarray(row_offset, dtype=np.int64)
    ip, dev = _ptr(ids)
    dp, _ = _ptr(dist)
    if out_ids is None:
        if dev:
            import torch
            out_ids = torch.empty((b, k), dtype=torch.int64, device=ids.device)
            out_dist = torch.empty((b, k), dtype=torch.float32, device=ids.device)
        else:
            out_ids = np.empty((b, k), dtype=np.int64)
            out_dist = np.empty((b, k), dtype=np.float32)
    oi, _ = _ptr(out_ids)
    od, _ = _ptr(out_dist)
    _check(load().vrs_merge_shards(ip, dp, w, b, k, offs.ctypes.data_as(C.c_void_p), metric, oi,
                                   od, dev, _stream(stream)))
    return out_ids, out_dist


def vrs_last_cert(h) -> dict:
    """How the last call's queries were certified exact."""
    c = np.zeros(4, dtype=np.int64)
    _check(load().vrs_last_cert(h, c.ctypes.data_as(C.c_void_p)))
    return dict(zip(("first_pass", "merge_widening", "wider_pass", "exact_gemv"), c.tolist()))


def vrs_cert_bound(kind: int, d: int, metric: int, qnorm: float, qres: float, xmax: float,
                   xres: float) -> float:
    return float(load().vrs_cert_bound(kind, d, metric, qnorm, qres, xmax, xres))


def vrs_planner_load(h, path):
    _check(load().vrs_planner_load(h, None if path is None else path.encode()))


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def vrs_mlp_nparams() -> int:
    return int(load().vrs_mlp_nparams())


def vrs_mlp_forward(params, X, bf16: bool = False) -> np.ndarray:
    P, X = _f32(params), _f32(X)
    X = X.reshape(-1, 6)
    Y = np.empty((X.shape[0], 3), dtype=np.float32)
    _check(load().vrs_mlp_forward(P.ctypes.data_as(C.c_void_p), X.ctypes.data_as(C.c_void_p),
                                  X.shape[0], int(bf16), Y.ctypes.data_as(C.c_void_p)))
    return Y


def vrs_mlp_grad(params, X, T, mask):
    P, X, T, M = _f32(params), _f32(X).reshape(-1, 6), _f32(T).reshape(-1, 3), _f32(mask).reshape(-1, 3)
    g = np.empty(P.size, dtype=np.float32)
    loss = C.c_float()
    _check(load().vrs_mlp_grad(P.ctypes.data_as(C.c_void_p), X.ctypes.data_as(C.c_void_p),
                               T.ctypes.data_as(C.c_void_p), M.ctypes.data_as(C.c_void_p),
                               X.shape[0], g.ctypes.data_as(C.c_void_p), C.byref(loss)))
    return g, loss.value


def vrs_mlp_train(params, X, T, mask, steps: int, lr: float = 1e-3):
    P = _f32(params).copy()
    X, T, M = _f32(X).reshape(-1, 6), _f32(T).reshape(-1, 3), _f32(mask).reshape(-1, 3)
    loss = C.c_float()
    _check(load().vrs_mlp_train(P.ctypes.data_as(C.c_void_p), X.ctypes.data_as(C.c_void_p),
                                T.ctypes.data_as(C.c_void_p), M.ctypes.data_as(C.c_void_p),
                                X.shape[0], steps, lr, C.byref(loss)))
    return P, loss.value


class Engine:
    """Owning wrapper: ``with Engine(0) as e: e.load(x); e.query(...)``."""

    def __init__(self, device: int = 0):
        self.h = vrs_create(device)
        self.n = 0
        self.d = 0

    def close(self):
        if self.h:
            vrs_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, x, attrs=None, dtype: int = VRS_F32, copies: int = 1 << VRS_F32):
        vrs_load_vectors(self.h, x, dtype, copies)
        self.n, self.d = x.shape
        if attrs is not None:
            for c in range(attrs.shape[0]):
                vrs_load_attribute(self.h, c, attrs[c])

    def query(self, q, preds, k, **kw):
        return vrs_query(self.h, q, preds, k, **kw)

    def range_query(self, q, pred, eps, **kw):
        return vrs_range_query(self.h, q, pred, eps, **kw)

    def query_dnf(self, q, conjs, k, **kw):
        return vrs_query_dnf(self.h, q, conjs, k, **kw)

    def join_topk(self, qrel, qattrs, qpred, rpred, k, **kw):
        return vrs_join_topk(self.h, qrel, qattrs, qpred, rpred, k, **kw)
