"""Pins for the oracle's number-format codecs (bf16, FP8 E4M3).

These formats have no counterpart in the paper; they serve the reduced-
precision scan.  The oracle's encoders are written from the format
definitions; here they are held to the format's constants, to exhaustive
enumeration of the 256 E4M3 codes, and to torch's CPU conversions (a library
routine).
"""
import numpy as np
import pytest
import torch

import oracle


def test_e4m3_constants():
    dec = oracle.e4m3_decode(np.arange(256, dtype=np.uint8))
    assert dec[0x7E] == 448.0 and dec[0xFE] == -448.0
    assert np.isnan(dec[0x7F]) and np.isnan(dec[0xFF])
    assert dec[0x01] == 2.0 ** -9            # smallest subnormal
    assert dec[0x07] == 7 * 2.0 ** -9        # largest subnormal
    assert dec[0x08] == 2.0 ** -6            # smallest normal
    assert dec[0x38] == 1.0                  # exponent field 7 = bias
    assert dec[0x00] == 0.0 and dec[0x80] == 0.0 and np.signbit(dec[0x80])
    finite = dec[~np.isnan(dec)]
    assert len(np.unique(finite)) == 253     # 254 finite codes, +0 and -0 equal


def test_e4m3_roundtrip_all_codes():
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF)], np.uint8)
    vals = oracle.e4m3_decode(codes).astype(np.float32)
    assert np.array_equal(oracle.e4m3_encode(vals), codes)


def test_e4m3_saturates_and_ties_to_even():
    enc = oracle.e4m3_encode
    assert enc(np.float32(1e6)) == 0x7E and enc(np.float32(-1e6)) == 0xFE
    assert enc(np.float32(np.inf)) == 0x7E
    assert enc(np.float32(460.0)) == 0x7E
    # 1 + 1/16 lies halfway between 1 (mantissa 000) and 1.125 (001): even -> 1
    assert enc(np.float32(1.0625)) == 0x38
    # 1.1875 halfway between 1.125 (001) and 1.25 (010): even -> 1.25
    assert enc(np.float32(1.1875)) == 0x3A
    # halfway between 0 and the smallest subnormal -> 0
    assert enc(np.float32(2.0 ** -10)) == 0x00


def test_e4m3_matches_torch():
    rng = np.random.default_rng(0)
    v = np.concatenate([
        rng.uniform(-447, 447, 20000),
        rng.standard_normal(20000) * 0.01,
        rng.standard_normal(20000) * 2.0 ** -8,
        # exact midpoints between neighbouring codes
        (oracle.e4m3_decode(np.arange(0, 0x7E, dtype=np.uint8))
         + oracle.e4m3_decode(np.arange(1, 0x7F, dtype=np.uint8))) / 2.0,
    ]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(oracle.e4m3_encode(v), ref)


def test_e4m3_rows_scale():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((20, 37)).astype(np.float32)
    x[3] = 0.0
    codes, scale = oracle.e4m3_rows(x)
    amax = np.abs(x).max(1)
    assert scale[3] == 1.0 and np.all(codes[3] == 0)
    rows = [i for i in range(20) if i != 3]
    np.testing.assert_array_equal(scale[rows], (amax[rows] / np.float32(448.0)).astype(np.float32))
    dec = oracle.e4m3_decode(codes) * scale[:, None].astype(np.float64)
    # the largest element of each row maps to +-448 * scale exactly
    for i in rows:
        j = np.argmax(np.abs(x[i]))
        assert abs(dec[i, j]) == pytest.approx(448.0 * float(scale[i]), rel=0, abs=0)
    # relative error of E4M3 is at most 2^-4 for normal values
    big = np.abs(x / scale[:, None]) >= 2.0 ** -6
    err = np.abs(dec - x)[big] / np.abs(x)[big]
    assert err.max() <= 2.0 ** -4 + 1e-12


def test_bf16_matches_torch():
    rng = np.random.default_rng(1)
    v = np.concatenate([
        rng.standard_normal(30000),
        rng.standard_normal(3000) * 1e-39,          # float32 subnormals
        rng.uniform(-3.3e38, 3.3e38, 3000),
        [0.0, -0.0, 1.0, 3.0e38, 3.4e38, np.inf, -np.inf],
    ]).astype(np.float32)
    # exact ties: float32 values whose low 16 bits are 0x8000
    bits = (rng.integers(0, 2 ** 15, 2000, dtype=np.uint32) << 16) | 0x8000
    bits |= rng.integers(0, 2, 2000, dtype=np.uint32) << 31
    bits &= ~np.uint32(0x7F800000) | np.uint32(0x3F800000)
    v = np.concatenate([v, bits.view(np.float32)])
    ref = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = oracle.bf16_encode(v)
    assert np.array_equal(got, ref)
    back = oracle.bf16_decode(got)
    fin = np.isfinite(v) & np.isfinite(back)
    vf, bf = v[fin].astype(np.float64), back[fin].astype(np.float64)
    # round to nearest at 8 significant bits: error <= half an ulp
    assert np.all(np.abs(bf - vf) <= np.abs(vf) * 2.0 ** -8 + 2.0 ** -134)
