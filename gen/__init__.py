"""Seeded synthetic inputs for the filtered exact top-k scan.

This module draws random numbers and nothing else: it holds none of the
search method's arithmetic (no distances, no predicates evaluated, no top-k).
Both the CUDA path's tests/bench and the CPU oracle read what it produces.

Workload shapes follow the paper's evaluation setting (Sec. 5, "Dataset":
in-memory synthetic vectors and relational columns drawn at random with a
fixed seed) with the data distribution replaced by a Gaussian mixture:

* vectors: 64 centres c_j ~ N(0, I_d); row i = c_{z_i} + 0.3 * N(0, I_d),
  z_i uniform on {0..63};
* queries: drawn from the same mixture on an independent stream;
* inner-product workloads: rows and queries normalised to unit length in
  float64, then rounded to float32 (cosine = dot product of normalised
  vectors, Sec. 3.1);
* attributes: int32, uniform on [0, attr_range);
* range predicates: half-open [lo, hi) on an attribute column.

Every stream comes from ``numpy.random.SeedSequence(seed).spawn``, so each
piece (centres, assignments, noise, attributes, queries, predicates) can be
regenerated independently of the others.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Iterator, List, Optional, Tuple

import numpy as np

INT32_MIN = -(2 ** 31)
INT32_MAX = 2 ** 31 - 1

# stream indices inside one SeedSequence
_S_CENTRES, _S_ASSIGN, _S_NOISE, _S_ATTR, _S_QUERY, _S_PRED, _S_K = range(7)


def _streams(seed: int, n: int = 8) -> List[np.random.Generator]:
    ss = np.random.SeedSequence(seed)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(n)]


@dataclasses.dataclass
class Mixture:
    """Parameters of the Gaussian mixture the rows and queries come from."""
    d: int
    n_centres: int = 64
    centre_std: float = 1.0
    within_std: float = 0.3
    seed: int = 0

    def centres(self) -> np.ndarray:
        g = _streams(self.seed)[_S_CENTRES]
        return (self.centre_std * g.standard_normal((self.n_centres, self.d))).astype(np.float32)


def _unit_rows(a: np.ndarray) -> np.ndarray:
    a64 = a.astype(np.float64)
    nrm = np.sqrt((a64 * a64).sum(axis=1, keepdims=True))
    nrm[nrm == 0] = 1.0
    return (a64 / nrm).astype(np.float32)


def vectors_chunks(n: int, mix: Mixture, unit: bool = False,
                   chunk: int = 1 << 20) -> Iterator[Tuple[int, np.ndarray]]:
    """Yield (row_offset, float32 [rows x d]) chunks of the data vectors.

    Chunking keeps host memory bounded for the 10^7..5*10^7-row workloads;
    the concatenation of the chunks does not depend on ``chunk``.
    """
    st = _streams(mix.seed)
    c = mix.centres()
    g_z, g_e = st[_S_ASSIGN], st[_S_NOISE]
    done = 0
    while done < n:
        m = min(chunk, n - done)
        z = g_z.integers(0, mix.n_centres, size=m)
        e = g_e.standard_normal((m, mix.d), dtype=np.float32)
        x = c[z] + np.float32(mix.within_std) * e
        if unit:
            x = _unit_rows(x)
        yield done, x.astype(np.float32, copy=False)
        done += m


def vectors(n: int, mix: Mixture, unit: bool = False) -> np.ndarray:
    out = np.empty((n, mix.d), dtype=np.float32)
    for off, x in vectors_chunks(n, mix, unit):
        out[off:off + x.shape[0]] = x
    return out


def queries(b: int, mix: Mixture, unit: bool = False) -> np.ndarray:
    """Query batch [b x d] drawn from the same mixture on its own stream."""
    g = _streams(mix.seed)[_S_QUERY]
    c = mix.centres()
    z = g.integers(0, mix.n_centres, size=b)
    e = g.standard_normal((b, mix.d), dtype=np.float32)
    q = c[z] + np.float32(mix.within_std) * e
    if unit:
        q = _unit_rows(q)
    return q.astype(np.float32, copy=False)


def attributes(n: int, n_cols: int = 1, attr_range: int = 100, seed: int = 0) -> np.ndarray:
    """int32 attribute columns [n_cols x n], uniform on [0, attr_range)."""
    g = _streams(seed)[_S_ATTR]
    return g.integers(0, attr_range, size=(n_cols, n), dtype=np.int32)


def to_bf16_values(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (round-to-nearest-even) and return the
    decoded float32 values; used to make bf16-*stored* workloads, whose
    stored values are then the input both sides see.  Uses torch's
    conversion so it carries no method arithmetic of this repository."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float32).numpy()


@dataclasses.dataclass
class Pred:
    """A conjunction of half-open ranges lo <= attr[col] < hi (0 terms = all)."""
    cols: List[int]
    lo: List[int]
    hi: List[int]

    @property
    def n_terms(self) -> int:
        return len(self.cols)


def pred_less_than(thresh: int, col: int = 0) -> Pred:
    """attr[col] < thresh, i.e. [INT32_MIN, thresh)."""
    return Pred([col], [INT32_MIN], [int(thresh)])


def pred_all() -> Pred:
    return Pred([], [], [])


def per_query_preds(b: int, attr_range: int = 1_000_000, s_min: float = 1e-4,
                    s_max: float = 0.5, seed: int = 0) -> Tuple[List[Pred], np.ndarray]:
    """Per-query conjunctions of two ranges on columns 0 and 1.

    The target selectivity s_q is log-uniform on [s_min, s_max]; it is split
    into two independent ranges of width sqrt(s_q) * attr_range placed at
    random offsets (the exact selectivity is whatever the rows give).
    Returns the predicates and the target selectivities.
    """
    g = _streams(seed)[_S_PRED]
    ls = g.uniform(math.log(s_min), math.log(s_max), size=b)
    s = np.exp(ls)
    preds = []
    for q in range(b):
        w = max(1, int(round(math.sqrt(s[q]) * attr_range)))
        lo0 = int(g.integers(0, attr_range - w + 1))
        lo1 = int(g.integers(0, attr_range - w + 1))
        preds.append(Pred([0, 1], [lo0, lo1], [lo0 + w, lo1 + w]))
    return preds, s


def per_query_k(b: int, choices=(1, 10, 100), seed: int = 0) -> np.ndarray:
    g = _streams(seed)[_S_K]
    return g.choice(np.asarray(choices, dtype=np.int32), size=b).astype(np.int32)


def pack_preds(preds: List[Pred]) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Flatten predicates into CSR form: (offsets[n+1], cols, lo, hi), int32."""
    off = np.zeros(len(preds) + 1, dtype=np.int32)
    for i, p in enumerate(preds):
        off[i + 1] = off[i] + p.n_terms
    cols = np.array([c for p in preds for c in p.cols], dtype=np.int32)
    lo = np.array([v for p in preds for v in p.lo], dtype=np.int32)
    hi = np.array([v for p in preds for v in p.hi], dtype=np.int32)
    return off, cols, lo, hi


# ---------------------------------------------------------------------------
# Named workloads (sizes of the paper-shaped configurations)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    n: int
    d: int
    batch: int
    k: int
    metric: str          # "l2" or "ip"
    selectivity: float   # fraction of rows the shared predicate keeps
    attr_range: int
    n_cols: int = 1
    seed: int = 0

    @property
    def unit(self) -> bool:
        return self.metric == "ip"

    def mixture(self) -> Mixture:
        return Mixture(self.d, seed=self.seed)

    def pred(self) -> Pred:
        if self.selectivity >= 1.0:
            return pred_less_than(self.attr_range)
        return pred_less_than(int(round(self.selectivity * self.attr_range)))


def small_l2() -> Workload:
    """100k x 128 fp32 rows, 1 attribute on [0,100), attr < 10, 16 queries, k=10, L2."""
    return Workload("n1e5_d128_b16_s10_k10_l2", 100_000, 128, 16, 10, "l2", 0.10, 100)


def sweep_cell(batch: int, selectivity: float, k: int = 10, metric: str = "l2",
               n: int = 1_000_000, d: int = 128) -> Workload:
    """One cell of the 1M x 128 fp32 sweep (attribute on [0, 10^6))."""
    name = f"n{n:.0e}_d{d}_b{batch}_s{selectivity:g}_k{k}_{metric}".replace("+0", "")
    return Workload(name, n, d, batch, k, metric, selectivity, 1_000_000)
