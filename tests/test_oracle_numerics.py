"""Pins of the oracle's rounding, scaling and splitting.

Each test checks the oracle against something other than itself: the
half-precision facts the paper prints (Sec. V), IEEE binary16 conversion in
numpy and torch (third-party routines), torch's BF16 and E4M3 conversions,
exhaustive enumeration of the E4M3 codes, and closed forms of the split.
"""
import json
import os

import numpy as np
import pytest
import torch

import synth
from oracle import numerics as nm


@pytest.fixture(scope="module")
def paper(golden_dir):
    with open(os.path.join(golden_dir, "paper_numbers.json")) as f:
        return json.load(f)


def _all_f16_values():
    bits = np.arange(65536, dtype=np.uint16)
    v = bits.view(np.float16).astype(np.float64)
    return v[np.isfinite(v)]


# ---- paper facts (Sec. V) ---------------------------------------------------

def test_fp16_facts_from_paper(paper):
    f = paper["fp16"]
    assert nm.round_to(np.float32(65504.0), "f16") == f["max_finite"]
    # "larger than 65,504 ... set to half infinity" (RNE reading: from 65520 on)
    assert nm.round_to(np.float32(65519.0), "f16") == 65504.0
    assert np.isinf(nm.round_to(np.float32(65520.0), "f16"))
    assert np.isinf(nm.round_to(np.float32(1e6), "f16"))
    # machine epsilon 2^-10: 1 + eps is representable, 1 + eps/2 is a tie to 1
    eps = f["machine_epsilon"]
    assert nm.round_to(np.float32(1.0 + eps), "f16") == 1.0 + eps
    assert nm.round_to(np.float32(1.0 + eps / 2), "f16") == 1.0
    assert nm.round_to(np.float32(1.0 + 3 * eps / 2), "f16") == 1.0 + 2 * eps
    # 1024 values in [1, 2)
    v = _all_f16_values()
    assert np.sum((v >= 1.0) & (v < 2.0)) == f["values_per_binade"]
    # spacing 32 in [2^15, 2^16) and 1 in [1024, 2048)
    hi = np.sort(v[(v >= 32768.0) & (v < 65536.0)])
    assert set(np.diff(hi)) == {float(f["spacing_between_32768_and_65536"])}
    mid = np.sort(v[(v >= 1024.0) & (v < 2048.0)])
    assert set(np.diff(mid)) == {float(f["spacing_between_1024_and_2048"])}
    # "too small to be represented as a half will be set to zero" (gradual underflow reading)
    assert nm.round_to(np.float32(2.0 ** -26), "f16") == 0.0
    assert nm.round_to(np.float32(2.0 ** -25), "f16") == 0.0          # tie -> even (0)
    assert nm.round_to(np.float32(1.5 * 2.0 ** -25), "f16") == 2.0 ** -24


# ---- against library conversions -------------------------------------------

def _f32_from_bits(bits):
    return np.asarray(bits, dtype=np.uint32).view(np.float32)


def _nonnan(x):
    return x[~np.isnan(x)]


def test_f16_matches_numpy_and_torch_on_boundaries():
    v = np.sort(_all_f16_values())
    v = v[v >= 0]
    mids = (v[:-1] + v[1:]) / 2.0                      # exact in FP32 (12 significant bits)
    mids32 = mids.astype(np.float32)
    assert np.array_equal(mids32.astype(np.float64), mids)
    up = np.nextafter(mids32, np.float32(np.inf))
    down = np.nextafter(mids32, np.float32(-np.inf))
    x = np.concatenate([v.astype(np.float32), mids32, up, down, np.float32([65519.996, 65520.0, 70000.0])])
    x = np.concatenate([x, -x])
    ours = nm.round_to(x, "f16")
    ref_np = x.astype(np.float16).astype(np.float64)
    ref_t = torch.from_numpy(x).to(torch.float16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref_np)
    assert np.array_equal(ours, ref_t)
    assert np.array_equal(np.signbit(ours), np.signbit(ref_np))


def test_f16_matches_numpy_on_random_fp32_patterns():
    bits = synth.words(1 << 21, seed=99)
    x = _nonnan(_f32_from_bits(bits))
    assert np.array_equal(nm.round_to(x, "f16"), x.astype(np.float16).astype(np.float64))


def test_bf16_matches_torch():
    bits = synth.words(1 << 21, seed=98)
    # add every tie and near-tie of the BF16 grid around random values
    base = bits & np.uint32(0xFFFF0000)
    extra = np.concatenate([base | np.uint32(0x8000), base | np.uint32(0x7FFF), base | np.uint32(0x8001)])
    x = _nonnan(_f32_from_bits(np.concatenate([bits, extra])))
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(nm.round_to(x, "bf16"), ref)


def test_e4m3_matches_torch_below_saturation():
    x = synth.uniform((1 << 20,), seed=97, lo=-464.0, hi=464.0)
    tiny = synth.uniform((1 << 16,), seed=96, lo=-2.0 ** -5, hi=2.0 ** -5)
    codes = nm.e4m3_value(np.arange(256, dtype=np.uint8))
    codes = codes[np.isfinite(codes)]
    grid = np.sort(np.unique(codes))
    mids = ((grid[:-1] + grid[1:]) / 2.0).astype(np.float32)
    x = np.concatenate([x, tiny, mids, codes.astype(np.float32)])
    x = x[np.abs(x) < 464.0]
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(nm.round_to(x, "e4m3"), ref)


def test_e4m3_saturates_finite():
    x = np.float32([464.0, 480.0, 1e9, np.inf, -500.0])
    assert list(nm.round_to(x, "e4m3")) == [448.0, 448.0, 448.0, 448.0, -448.0]


def test_e4m3_codes_roundtrip():
    codes = np.arange(256, dtype=np.uint8)
    vals = nm.e4m3_value(codes)
    finite = np.isfinite(vals)
    assert finite.sum() == 254                     # 0x7F and 0xFF are NaN
    assert np.array_equal(nm.e4m3_bits(vals[finite]), codes[finite])
    assert np.array_equal(nm.round_to(vals[finite], "e4m3"), vals[finite])
    assert np.nanmax(vals) == 448.0 and np.nanmin(np.abs(vals[vals != 0])) == 2.0 ** -9
    # torch agrees on the decoding
    t = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(t[finite], vals[finite])


def test_bit_encoders():
    v = _all_f16_values()
    assert np.array_equal(nm.f16_bits(v).view(np.float16).astype(np.float64), v)
    b = nm.round_to(synth.uniform((4096,), seed=5), "bf16")
    back = (nm.bf16_bits(b).astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    assert np.array_equal(back, b)


# ---- E4M3 per-tensor scale ----------------------------------------------------

@pytest.mark.parametrize("amax", [1.0, 0.999, 448.0, 448.5, 1e-3, 3.0e5, 2.0 ** -20, 7.0])
def test_e4m3_scale_is_largest_power_of_two(amax):
    j = nm.e4m3_scale_exponent(amax)
    assert amax * 2.0 ** j <= 448.0 < amax * 2.0 ** (j + 1)


def test_e4m3_scale_degenerate():
    assert nm.e4m3_scale(0.0) == 1.0
    assert nm.e4m3_scale(float("inf")) == 1.0
    assert nm.e4m3_scale_exponent(2.0 ** -149) == 127      # capped: s stays finite in FP32


def test_e4m3_quantize_never_saturates():
    x = synth.normal((4096,), seed=8).astype(np.float64) * 1000.0
    q, s = nm.quantize(x, "e4m3")
    assert np.max(np.abs(q)) <= 448.0
    assert np.max(np.abs(x * s)) <= 448.0


# ---- split into hi + lo (Sec. V residual, Eq. 1 / Eq. 2) ----------------------

def test_split_exact_for_22_significant_bits():
    # x = (integer with <= 22 bits) * 2^e and lo stays in the normal FP16 range
    r = synth.words(20000, seed=11)
    ints = (r & np.uint32((1 << 22) - 1)).astype(np.float64) + float(1 << 21)
    e = (synth.words(20000, seed=12) % 8).astype(np.float64) - 24.0
    x = (ints * 2.0 ** e).astype(np.float32)
    hi, lo = nm.split(x, "f16")
    assert np.array_equal(hi + lo, x.astype(np.float64))


def test_split_error_bound_and_fp16_inputs():
    x = synth.log_uniform_pow2((50000,), seed=13)
    hi, lo = nm.split(x, "f16")
    x64 = x.astype(np.float64)
    r = x64 - hi
    # |x - hi - lo| <= half an ulp of lo: 2^-11 |r| (normal lo) or 2^-25 (subnormal lo)
    assert np.all(np.abs(r - lo) <= np.maximum(2.0 ** -11 * np.abs(r), 2.0 ** -25))
    # FP32 difference is exact: the residual is representable in FP32
    assert np.array_equal((x - hi.astype(np.float32)).astype(np.float64), r)
    # a value that is already FP16 has no residual
    hi2, lo2 = nm.split(hi.astype(np.float32), "f16")
    assert np.array_equal(hi2, hi) and not np.any(lo2)


def test_split_bf16_pieces():
    x = synth.uniform((50000,), seed=14)
    hi, lo = nm.split(x, "bf16")
    r = x.astype(np.float64) - hi
    assert np.all(np.abs(r) <= 2.0 ** -8 * np.abs(x.astype(np.float64)))
    assert np.all(np.abs(r - lo) <= 2.0 ** -8 * np.abs(r))
    assert np.array_equal(nm.round_to(hi, "bf16"), hi) and np.array_equal(nm.round_to(lo, "bf16"), lo)


def test_rounding_is_ties_to_even_not_away():
    # 1 + 2^-11 is the midpoint between 1 and 1 + 2^-10; 1 + 3*2^-11 between 1+2^-10 and 1+2^-9
    assert nm.round_to(np.float32(1.0 + 2.0 ** -11), "f16") == 1.0
    assert nm.round_to(np.float32(1.0 + 3 * 2.0 ** -11), "f16") == 1.0 + 2.0 ** -9
    assert nm.round_to(np.float32(-(1.0 + 2.0 ** -11)), "f16") == -1.0
    assert nm.round_to(np.float32(1.0 + 2.0 ** -8), "bf16") == 1.0
    assert nm.round_to(np.float32(1.0 + 2.0 ** -4), "e4m3") == 1.0
    assert nm.round_to(np.float32(1.0 + 3 * 2.0 ** -4), "e4m3") == 1.25


# ---- scaled residual split (Ootomo and Yokota, 2022) ---------------------------

def test_scaled_split_keeps_small_residuals():
    # x with 22 significant bits and |x| ~ 2^-9: the plain FP16 residual is subnormal and
    # loses bits, the scaled one (x 2^11) is normal and exact
    ints = (synth.words(5000, seed=15) & np.uint32((1 << 22) - 1)).astype(np.float64) + float(1 << 21)
    x = (ints * 2.0 ** -31).astype(np.float32)        # in [2^-10, 2^-9)
    x64 = x.astype(np.float64)
    hi, lo = nm.split(x, "f16")
    assert not np.array_equal(hi + lo, x64)
    hs, ls = nm.split_scaled(x, "f16")
    assert np.array_equal(hs, hi)
    assert np.array_equal(hs + np.ldexp(ls, -11), x64)
    # scaling by a power of two commutes with rounding wherever the scaled residual is normal
    big = synth.uniform((5000,), seed=16, lo=-200.0, hi=200.0)
    h1, l1 = nm.split(big, "f16")
    h2, l2 = nm.split_scaled(big, "f16")
    normal = np.abs(l1) >= 2.0 ** -14
    assert np.array_equal(h1, h2) and np.array_equal(np.ldexp(l1[normal], 11), l2[normal])


def test_scaled_split_bf16():
    x = synth.log_uniform_pow2((20000,), seed=17)
    hs, ls = nm.split_scaled(x, "bf16")
    r = x.astype(np.float64) - hs
    assert np.all(np.abs(np.ldexp(r, 8) - ls) <= 2.0 ** -8 * np.abs(np.ldexp(r, 8)))


# ---- three-piece BF16 split (Henry, Tang and Heinecke, 2019) --------------------

def test_bf16x3_pieces_sum_to_x_over_the_fp32_range():
    # FP32 values with random 24-bit significands over 200 binades: three 8-bit pieces hold them
    n = 40000
    ints = (synth.words(n, seed=18) & np.uint32((1 << 23) - 1)).astype(np.float64) + float(1 << 23)
    e = (synth.words(n, seed=19) % 200).astype(np.float64) - 100.0
    sgn = np.where(synth.words(n, seed=20) & np.uint32(1), -1.0, 1.0)
    x = (sgn * ints * 2.0 ** (e - 23)).astype(np.float32)
    x64 = x.astype(np.float64)
    p0, p1, p2 = nm.split_bf16x3(x)
    assert np.array_equal(p0 + p1 + p2, x64)
    for p in (p0, p1, p2):
        assert np.array_equal(nm.round_to(p, "bf16"), p)
    # each piece is at most half an ulp (2^-8 relative) of what is left before it
    assert np.all(np.abs(p1) <= 2.0 ** -8 * np.abs(x64))
    assert np.all(np.abs(p2) <= 2.0 ** -8 * np.abs(x64 - p0))
    # the first piece is the plain BF16 rounding, the second the plain BF16 residual
    h, l = nm.split(x, "bf16")
    assert np.array_equal(p0, h) and np.array_equal(p1, l)


def test_bf16x3_short_significands_leave_zero_pieces():
    n = 5000
    e = (synth.words(n, seed=21) % 60).astype(np.float64) - 30.0
    b8 = (synth.words(n, seed=22) & np.uint32(0x7F)).astype(np.float64) + 128.0        # 8 bits
    b16 = (synth.words(n, seed=23) & np.uint32(0x7FFF)).astype(np.float64) + 32768.0   # 16 bits
    x8 = (b8 * 2.0 ** (e - 7)).astype(np.float32)
    x16 = (b16 * 2.0 ** (e - 15)).astype(np.float32)
    p0, p1, p2 = nm.split_bf16x3(x8)
    assert np.array_equal(p0, x8.astype(np.float64)) and not np.any(p1) and not np.any(p2)
    p0, p1, p2 = nm.split_bf16x3(x16)
    assert np.array_equal(p0 + p1, x16.astype(np.float64)) and not np.any(p2)
