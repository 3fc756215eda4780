"""The exactness certificate's bound E (vrs_cert_bound) dominates the real
first-pass error of the reduced-precision encodings.

For rows and queries of the Gaussian-mixture workloads (and adversarial
ones: aligned rows, large dynamic range), the first-pass key is computed in
float64 from the *encoded* values exactly as the tensor plans form it (BF16
round-to-nearest-even; E4M3 with a per-vector scale max|v|/448), so the only
error left is the encoding's.  E, fed with the norms and residual norms
measured the same way, must bound |key - exact| for every (query, row)
pair; E with the residual terms dropped must not (so the test would catch a
bound that forgot them).  No GPU: vrs_cert_bound is a host function.
"""
import numpy as np
import pytest

import gen
import oracle


@pytest.fixture(scope="module")
def vrs():
    from paper_2403_15807_gb300 import build, vrs as v
    build.build()
    v.load()
    return v


def _bf16(a):
    return oracle.bf16_decode(oracle.bf16_encode(a)).astype(np.float64)


def _e4m3(a):
    codes, scale = oracle.e4m3_rows(a)
    return oracle.e4m3_decode(codes) * scale.astype(np.float64)[:, None]


def _inputs(d, kind):
    if kind == "mixture":
        mix = gen.Mixture(d, seed=d)
        return gen.vectors(600, mix), gen.queries(12, mix)
    g = np.random.default_rng(d)
    if kind == "aligned":
        # rows nearly parallel to the queries: the dot product's error is not
        # averaged away by random signs
        base = g.standard_normal(d).astype(np.float32)
        x = (base[None, :] * (1 + 0.01 * g.standard_normal((600, 1)))).astype(np.float32)
        q = (base[None, :] * (1 + 0.01 * g.standard_normal((12, 1)))).astype(np.float32)
        return x, q
    # wide dynamic range inside a vector
    x = (g.standard_normal((600, d)) * np.exp(g.uniform(-6, 3, (600, d)))).astype(np.float32)
    q = (g.standard_normal((12, d)) * np.exp(g.uniform(-6, 3, (12, d)))).astype(np.float32)
    return x, q


@pytest.mark.parametrize("d", [64, 128, 200])
@pytest.mark.parametrize("kind", ["mixture", "aligned", "wide"])
@pytest.mark.parametrize("enc", ["bf16", "e4m3"])
@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_bound_dominates_first_pass_error(vrs, d, kind, enc, metric):
    x, q = _inputs(d, kind)
    x64, q64 = x.astype(np.float64), q.astype(np.float64)
    f = _bf16 if enc == "bf16" else _e4m3
    xh, qh = f(x), f(q)
    exact_dot = q64 @ x64.T
    enc_dot = qh @ xh.T
    xn2, qn2 = (x64 ** 2).sum(1), (q64 ** 2).sum(1)
    if metric == "l2":
        key = qn2[:, None] + xn2[None, :] - 2 * enc_dot
        ex = qn2[:, None] + xn2[None, :] - 2 * exact_dot
    else:
        key, ex = -enc_dot, -exact_dot
    err = np.abs(key - ex)
    A = float(np.sqrt(xn2.max()))
    Rx = float(np.sqrt(((x64 - xh) ** 2).sum(1)).max())
    rq = np.sqrt(((q64 - qh) ** 2).sum(1))
    kind_id = vrs.VRS_CERT_BF16 if enc == "bf16" else vrs.VRS_CERT_E4M3
    m = vrs.VRS_L2 if metric == "l2" else vrs.VRS_IP
    for i in range(q.shape[0]):
        E = vrs.vrs_cert_bound(kind_id, d, m, float(np.sqrt(qn2[i])), float(rq[i]), A, Rx)
        assert E > 0
        assert err[i].max() <= E, f"query {i}: error {err[i].max():.4g} above the bound {E:.4g}"
    # without the residual terms the bound does not hold (the test is sensitive)
    worst = max(err[i].max() - vrs.vrs_cert_bound(kind_id, d, m, float(np.sqrt(qn2[i])), 0.0,
                                                  A, 0.0) for i in range(q.shape[0]))
    assert worst > 0


def test_bound_grows_with_each_term(vrs):
    """E is monotone in the query norm, both residuals and the row norm, and
    rejects unknown kinds."""
    base = vrs.vrs_cert_bound(vrs.VRS_CERT_BF16, 128, vrs.VRS_L2, 10.0, 0.1, 12.0, 0.2)
    for args in ((11.0, 0.1, 12.0, 0.2), (10.0, 0.2, 12.0, 0.2), (10.0, 0.1, 13.0, 0.2),
                 (10.0, 0.1, 12.0, 0.3)):
        assert vrs.vrs_cert_bound(vrs.VRS_CERT_BF16, 128, vrs.VRS_L2, *args) > base
    assert vrs.vrs_cert_bound(99, 128, vrs.VRS_L2, 1.0, 0.0, 1.0, 0.0) == -1.0
    # the float32 kernel families carry no encoding residual: their bound is
    # the accumulation term alone, far below BF16's
    f32 = vrs.vrs_cert_bound(vrs.VRS_CERT_TF32X3, 128, vrs.VRS_L2, 10.0, 0.0, 12.0, 0.0)
    assert 0 < f32 < base / 10
