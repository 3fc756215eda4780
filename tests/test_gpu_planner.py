"""The plan-selection network's GPU kernels against the float64 oracle, the
planner file, and the gain of the learned plan choice over the fixed rule on
timings the engine measured."""
import json
import os

import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
DATA = os.path.join(os.path.dirname(HERE), "paper_2403_15807_gb300", "data")


@pytest.fixture(scope="module")
def vrs():
    from paper_2403_15807_gb300 import build, vrs as v
    build.build()
    v.load()
    return v


def _problem(seed, m=300):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(oracle.mlp_nparams()) * 0.3).astype(np.float32)
    X = rng.standard_normal((m, 6)).astype(np.float32)
    T = rng.standard_normal((m, 3)).astype(np.float32)
    M = (rng.uniform(size=(m, 3)) < 0.8).astype(np.float32)
    return p, X, T, M


def test_forward_matches_oracle(vrs):
    p, X, _, _ = _problem(0)
    Y = vrs.vrs_mlp_forward(p, X)
    Yr, _, _ = oracle.mlp(p.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(Y, Yr, rtol=1e-4, atol=1e-4)
    Yb = vrs.vrs_mlp_forward(p, X, bf16=True)
    # bf16 inference: 8 significant bits per weight and activation
    assert np.max(np.abs(Yb - Yr)) <= 0.05 * max(1.0, np.max(np.abs(Yr)))


def test_gradient_matches_oracle(vrs):
    p, X, T, M = _problem(1)
    g, loss = vrs.vrs_mlp_grad(p, X, T, M)
    _, lr, gr = oracle.mlp(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                           M.astype(np.float64), want_grad=True)
    assert loss == pytest.approx(lr, rel=1e-4)
    rel = np.linalg.norm(g - gr) / np.linalg.norm(gr)
    assert rel <= 1e-3
    # and element-wise where the gradient is not tiny
    big = np.abs(gr) > 1e-3 * np.abs(gr).max()
    np.testing.assert_allclose(g[big], gr[big], rtol=2e-3, atol=1e-6)


def test_training_fits_a_known_function(vrs):
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (800, 6)).astype(np.float32)
    T = np.stack([X[:, 0] * 2 - X[:, 1], np.abs(X[:, 2]), X[:, 3] * X[:, 4]], 1).astype(np.float32)
    M = np.ones_like(T)
    p0 = (rng.standard_normal(vrs.vrs_mlp_nparams()) * 0.1).astype(np.float32)
    _, l0 = vrs.vrs_mlp_grad(p0, X, T, M)
    p1, l1 = vrs.vrs_mlp_train(p0, X, T, M, steps=1500, lr=3e-3)
    assert l1 < 0.05 * l0
    # the float64 oracle agrees on the trained parameters' loss
    _, lr1, _ = oracle.mlp(p1.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                           M.astype(np.float64))
    assert l1 == pytest.approx(lr1, rel=1e-3)


def test_planner_file_load_and_rejection(vrs, tmp_path):
    from paper_2403_15807_gb300 import planner
    n = vrs.vrs_mlp_nparams()
    params = np.zeros(n, np.float32)
    # a model that predicts GEMV cheapest: b3 = (-5, 0, 0)
    params[n - 3] = -5.0
    m = planner.Model(params, np.zeros(6, np.float32), np.ones(6, np.float32), 0.0, 1.0)
    path = str(tmp_path / "p.bin")
    planner.write_planner(path, m)
    mix = gen.Mixture(32, seed=1)
    x = gen.vectors(4000, mix)
    attrs = gen.attributes(4000, 1, 100)
    q = torch.from_numpy(gen.queries(300, mix)).cuda()
    with vrs.Engine(0) as e:
        e.load(x, attrs, dtype=vrs.VRS_F32, copies=7)
        vrs.vrs_planner_load(e.h, None)   # (the shipped model is loaded by default)
        e.query(q, [gen.pred_less_than(80)], np.int32([10]), compute=vrs.VRS_BF16)
        assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_MASK_GEMM      # fixed rule
        vrs.vrs_planner_load(e.h, path)
        e.query(q, [gen.pred_less_than(80)], np.int32([10]), compute=vrs.VRS_BF16)
        assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_GEMV           # learned choice
        e.query(q, [gen.pred_less_than(80)], np.int32([10]), compute=vrs.VRS_FP8E4M3)
        assert vrs.vrs_last_plan(e.h) != vrs.VRS_PLAN_GEMV           # not available for FP8
        # corrupt / missing files are rejected and the fixed rule comes back
        vrs.vrs_planner_load(e.h, None)
        blob = bytearray(open(path, "rb").read())
        blob[100] ^= 0xFF
        bad = str(tmp_path / "bad.bin")
        open(bad, "wb").write(bytes(blob))
        for pth in (bad, str(tmp_path / "missing.bin")):
            with pytest.raises(vrs.VrsError) as ei:
                vrs.vrs_planner_load(e.h, pth)
            assert ei.value.status == vrs.VRS_EIO
        e.query(q, [gen.pred_less_than(80)], np.int32([10]), compute=vrs.VRS_BF16)
        assert vrs.vrs_last_plan(e.h) == vrs.VRS_PLAN_MASK_GEMM


def test_learned_planner_beats_fixed_rule(vrs):
    """Trained by the library's kernels on the engine's own timing grid, the
    network's plan choices cost less total latency than the fixed rule on
    the held-out half of the cells."""
    path = os.path.join(DATA, "timings_grid_gb300.json")
    if not os.path.exists(path):
        pytest.skip("timing grid not recorded")
    from paper_2403_15807_gb300 import planner
    recs = json.load(open(path))["records"]
    rng = np.random.default_rng(0)
    idx = rng.permutation(len(recs))
    train = [recs[i] for i in idx[: len(recs) // 2]]
    test = [recs[i] for i in idx[len(recs) // 2:]]
    m = planner.fit(train, steps=3000)
    ev = planner.evaluate(m, test)
    print("held-out latency (ms): model %.1f fixed %.1f best %.1f over %d cells"
          % (ev["model"], ev["fixed"], ev["best"], ev["cells"]))
    assert ev["cells"] > 20
    assert ev["model"] <= ev["fixed"]
