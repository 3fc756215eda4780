"""The C-ABI library builds for sm_103a, loads, and exports every symbol
include/vrs.h declares; host-side argument checks work without a GPU."""
import ctypes as C
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_15807_gb300 import build, vrs
    build.build()
    return vrs.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "vrs.h")).read()
    return sorted(set(re.findall(r"^VRS_API[^(]*?\b(vrs_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"


def test_binding_covers_every_declared_symbol():
    from paper_2403_15807_gb300 import vrs
    assert sorted(vrs.SIGNATURES) == declared_symbols()


def test_null_arguments_are_rejected(lib):
    from paper_2403_15807_gb300 import vrs
    assert lib.vrs_destroy(None) == vrs.VRS_OK
    assert lib.vrs_create(0, None) == vrs.VRS_EINVAL
    assert b"NULL" in lib.vrs_last_error()
    assert lib.vrs_query(None, None, 1, 1, None, 1, None, 1, 1, 0, 0, None, None, 0, None) \
        == vrs.VRS_EINVAL
    assert lib.vrs_set_plan(None, 0) == vrs.VRS_EINVAL
    assert lib.vrs_version().decode().count(".") == 2


def _has_gpu():
    import torch
    return torch.cuda.is_available()


@pytest.mark.skipif(_has_gpu(), reason="only meaningful without a GPU")
def test_create_without_gpu_fails_cleanly(lib):
    from paper_2403_15807_gb300 import vrs
    h = C.c_void_p()
    st = lib.vrs_create(0, C.byref(h))
    assert st in (vrs.VRS_ECUDA, vrs.VRS_EINVAL)
    assert lib.vrs_last_error() != b""


def _header_constants():
    """Every `VRS_NAME = value` enumerator of include/vrs.h."""
    src = open(os.path.join(ROOT, "include", "vrs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {m.group(1): int(m.group(2))
            for m in re.finditer(r"\b(VRS_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}


def test_binding_constants_match_the_header():
    """The binding's status codes, options, plans, encodings and metrics have
    the header's values (the binding only marshals, so a stale constant
    would send the wrong option or plan through the ABI)."""
    from paper_2403_15807_gb300 import vrs
    hdr = _header_constants()
    assert len(hdr) >= 25
    # the stages are the binding's STAGES tuple, in the header's order
    stages = {k: v for k, v in hdr.items() if k.startswith("VRS_STAGE_")}
    assert len(vrs.STAGES) == hdr["VRS_N_STAGES"] == len(stages)
    for k, v in stages.items():
        assert vrs.STAGES[v] == k[len("VRS_STAGE_"):].lower(), (k, v)
    rest = {k: v for k, v in hdr.items() if k not in stages}
    missing = [k for k in rest if not hasattr(vrs, k)]
    assert not missing, missing
    for k, v in rest.items():
        assert getattr(vrs, k) == v, (k, getattr(vrs, k), v)


def test_predicates_marshal_into_the_abi_struct():
    """vrs.Pred (or any object with cols / lo / hi) becomes vrs_pred terms;
    an empty conjunction has no terms."""
    from paper_2403_15807_gb300 import vrs
    arr, keep = vrs.make_preds([vrs.Pred([2, 0], [-5, 7], [5, 9]), vrs.Pred([], [], [])])
    assert arr[0].n_terms == 2 and arr[1].n_terms == 0
    t = arr[0].terms
    assert (t[0].col, t[0].lo, t[0].hi, t[1].col, t[1].lo, t[1].hi) == (2, -5, 5, 0, 7, 9)


def test_float_key_orders_like_the_floats(lib):
    """vrs_float_key is strictly increasing over ordered floats (subnormals,
    infinities included), maps -0 and +0 alike, and sends NaN past every
    half-open range."""
    from paper_2403_15807_gb300 import vrs
    f32 = np.float32
    special = [-np.inf, -np.finfo(f32).max, -1e30, -1.5, -1.0, -np.finfo(f32).tiny,
               -1e-45, 0.0, 1e-45, np.finfo(f32).tiny, 1e-10, 1.0, 1.0000001, 3e38,
               np.finfo(f32).max, np.inf]
    rng = np.random.default_rng(0)
    vals = np.concatenate([np.array(special, f32),
                           (rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 30, 2000)).astype(f32)])
    vals = np.unique(vals)                 # sorted, distinct floats
    keys = np.array([vrs.vrs_float_key(float(v)) for v in vals], dtype=np.int64)
    assert np.all(np.diff(keys) > 0)
    assert vrs.vrs_float_key(-0.0) == vrs.vrs_float_key(0.0) == 0
    assert vrs.vrs_float_key(float("nan")) == 2 ** 31 - 1
    assert keys.max() < 2 ** 31 - 1


def test_next_row_entry_points_reject_null_arguments(lib):
    """Range search, vector join, disjunctions and float columns check their
    arguments on the host before touching a device."""
    from paper_2403_15807_gb300 import vrs
    assert lib.vrs_range_query(None, None, 1, 1, None, C.c_float(1.0), 0, 0, None, None, None,
                               0, None) == vrs.VRS_EINVAL
    assert lib.vrs_join_topk(None, None, 1, 1, None, 0, None, None, 1, 0, 0, 0, None, None,
                             None, None, 0, None) == vrs.VRS_EINVAL
    assert lib.vrs_query_dnf(None, None, 1, 1, None, 1, 1, 0, 0, None, None, 0, None) \
        == vrs.VRS_EINVAL
    assert lib.vrs_load_attribute_f32(None, 0, None, 1, 0, None) == vrs.VRS_EINVAL
    assert b"NULL" in lib.vrs_last_error()
