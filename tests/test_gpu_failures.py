"""Failure detection without a GPU fault: an injected host-side allocation
failure (VRS_FAULT=alloc) returns VRS_ENOMEM, and a bounded device-side
wait that runs out (VRS_OPT_WAIT_TEST: the distance kernel waits on a
barrier nothing arrives at) returns VRS_ETIMEOUT; in both cases the engine
stays usable and the next query is exact."""
import os

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


def _data():
    n, d, b = 20_000, 128, 8
    mix = gen.Mixture(d, seed=9)
    return gen.vectors(n, mix), gen.queries(b, mix), gen.attributes(n, 1, 100, seed=9)


def _exact(vrs, e, x, q, attrs, pred, k=10):
    ids, dist = e.query(q, [pred], np.int32([k]))   # host buffers: synchronous
    rid, rdist, rcnt = oracle.query(x, attrs, q, [pred], k + 1, "l2", n_threads=16)
    check_topk(x, q, attrs, [pred], np.int32([k]), "l2", ids, dist, rid, rdist, rcnt)


def test_injected_allocation_failure(vrs, monkeypatch):
    x, q, attrs = _data()
    pred = gen.pred_less_than(30)
    with vrs.Engine(0) as e:
        e.load(x, attrs)
        monkeypatch.setenv("VRS_FAULT", "alloc")
        # a batch larger than any seen so far needs new workspace
        with pytest.raises(vrs.VrsError) as ei:
            e.query(np.ascontiguousarray(np.tile(q, (40, 1))), [pred], np.int32([10]))
        assert ei.value.status == vrs.VRS_ENOMEM
        assert "injected" in vrs.vrs_last_error()
        monkeypatch.delenv("VRS_FAULT")
        _exact(vrs, e, x, q, attrs, pred)


def test_bounded_wait_runs_out(vrs):
    x, q, attrs = _data()
    pred = gen.pred_less_than(30)
    with vrs.Engine(0) as e:
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_PAIR_COPY, 1)
        e.load(x, attrs)
        vrs.vrs_set_plan(e.h, vrs.VRS_PLAN_GEMV)
        _exact(vrs, e, x, q, attrs, pred)
        vrs.vrs_set_option(e.h, vrs.VRS_OPT_WAIT_TEST, 1)
        with pytest.raises(vrs.VrsError) as ei:
            e.query(q, [pred], np.int32([10]))
        assert ei.value.status == vrs.VRS_ETIMEOUT
        # the hook is one-shot; the engine and the context stay usable
        for _ in range(2):
            _exact(vrs, e, x, q, attrs, pred)
