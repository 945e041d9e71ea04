"""Rounding of FP32 values to narrow formats, written from the IEEE-754 definition.

Oracle code (test infrastructure only; see the package header).

Sec. V of the paper: an FP32 value is "rounded" to half precision; half has a
10-bit fraction (machine epsilon 2^-10, 1024 values per binade), range
+-65504, values above the range become infinity and values too small become
zero.  The reading taken here (paper silent on the rounding mode) is IEEE 754
roundTiesToEven with gradual underflow:

* the exact value is rounded to the nearest number of the form
  integer * 2^(max(e, emin) - mbits), e = floor(log2|x|), ties to the even
  integer;
* if that result exceeds the largest finite number it overflows: to +-inf for
  FP16 and BF16 (so 65520 and above become inf, 65504 < x < 65520 give 65504),
  and to +-448 for E4M3 with "satfinite" semantics (E4M3 has no infinity).

FP16: 1 sign, 5 exponent, 10 fraction bits, emin = -14.
BF16: 1 sign, 8 exponent, 7 fraction bits, emin = -126 (not in the paper).
E4M3: 1 sign, 4 exponent, 3 fraction bits, emin = -6, max 448 (not in the paper).

The residual of Sec. V, R_A = A_single - A_half, is stored in half precision
(Eq. 1 and Eq. 2 multiply it on the tensor cores): ``split`` returns
hi = round(x) and lo = round(x - hi).  x - hi is computed exactly (in FP64; it
is also exact in FP32 because |x - hi| is at most half an FP16 ulp of x and a
multiple of the FP32 ulp of x).
"""
from __future__ import annotations

import math

import numpy as np

# mbits: stored fraction bits; emin: exponent of the smallest normal number.
FORMATS = {
    "f16": {"mbits": 10, "emin": -14, "max_finite": 65504.0, "overflow": "inf"},
    "bf16": {"mbits": 7, "emin": -126, "max_finite": (2.0 - 2.0 ** -7) * 2.0 ** 127, "overflow": "inf"},
    "e4m3": {"mbits": 3, "emin": -6, "max_finite": 448.0, "overflow": "satfinite"},
}

E4M3_MAX = 448.0


def round_to(x, fmt: str) -> np.ndarray:
    """Round each value of ``x`` (FP32 values, any float dtype) to format ``fmt``.

    Returns FP64 numbers that are exactly representable in ``fmt``.  NaN stays
    NaN; the sign of zero is kept.
    """
    f = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    with np.errstate(invalid="ignore", over="ignore"):
        _, E = np.frexp(a)                      # a = m * 2^E, m in [0.5, 1)
        e = E.astype(np.int64) - 1              # a in [2^e, 2^(e+1))
        qexp = np.maximum(e, f["emin"]) - f["mbits"]   # exponent of the quantum
        r = np.ldexp(np.rint(np.ldexp(a, -qexp)), qexp)  # np.rint: ties to even
    big = f["max_finite"]
    over = r > big
    if f["overflow"] == "inf":
        r = np.where(over, np.inf, r)
        r = np.where(np.isinf(a), np.inf, r)
    else:
        r = np.where(over | np.isinf(a), big, r)
    r = np.where(np.isnan(a), np.nan, r)
    return np.copysign(r, x)


def absmax(x) -> float:
    """max |x| over all entries (the per-tensor amax of the E4M3 scale)."""
    x = np.asarray(x, dtype=np.float64)
    return float(np.max(np.abs(x))) if x.size else 0.0


def e4m3_scale_exponent(amax: float) -> int:
    """Exponent j of the per-tensor E4M3 scale s = 2^j.

    Reading (the paper has no FP8): s is the largest power of two with
    amax * s <= 448, so scaling is exact and never saturates.  amax = 0 or a
    non-finite amax gives s = 1; j is capped at 127 so s stays a finite FP32.
    """
    if not (amax > 0.0) or not math.isfinite(amax):
        return 0
    j = 0
    while amax * 2.0 ** j > E4M3_MAX:
        j -= 1
    while j < 127 and amax * 2.0 ** (j + 1) <= E4M3_MAX:
        j += 1
    return j


def e4m3_scale(amax: float) -> float:
    return 2.0 ** e4m3_scale_exponent(amax)


def quantize(x, fmt: str, amax: float | None = None):
    """Values of the quantised operand and its scale s.

    FP16/BF16: (round_to(x), 1).  E4M3: (round_to(x * s), s) with s from the
    absmax of ``x`` (or the given ``amax`` when ``x`` is a sample of a larger
    tensor).  The product keeps the scale folded in; the GEMM divides by
    s_A * s_B in its epilogue.
    """
    x = np.asarray(x, dtype=np.float64)
    if fmt == "e4m3":
        s = e4m3_scale(absmax(x) if amax is None else amax)
        return round_to(x * s, "e4m3"), s
    return round_to(x, fmt), 1.0


def split(x, piece: str):
    """(hi, lo) with hi = round(x), lo = round(x - hi) in format ``piece``.

    Definition of the residual matrix R = A_single - A_half (Sec. V), stored in
    the 16-bit format (reading: lo is itself rounded, since Eq. 1 and Eq. 2
    feed it to the tensor cores).
    """
    x = np.asarray(x, dtype=np.float64)
    hi = round_to(x, piece)
    with np.errstate(invalid="ignore"):
        lo = round_to(x - hi, piece)
    return hi, lo


# Exponent of the residual scale of the scaled split: the residual of an
# FP16 hi piece is at most 2^-11 |x|, of a BF16 hi piece 2^-8 |x|.
SPLIT_SCALE_EXP = {"f16": 11, "bf16": 8}


def split_scaled(x, piece: str):
    """(hi, lo_s) with hi = round(x), lo_s = round((x - hi) * 2^s), s = SPLIT_SCALE_EXP[piece].

    Scaled-residual split published by Ootomo and Yokota (2022, "Recovering
    single precision accuracy from Tensor Cores while surpassing the FP32
    theoretical peak performance"): the residual is multiplied by 2^s before
    rounding so that it stays in the normal range of the 16-bit format; the
    products that use it are multiplied by 2^-s afterwards.  The scaling by a
    power of two is exact.
    """
    x = np.asarray(x, dtype=np.float64)
    hi = round_to(x, piece)
    with np.errstate(invalid="ignore"):
        lo = round_to(np.ldexp(x - hi, SPLIT_SCALE_EXP[piece]), piece)
    return hi, lo


def split_bf16x3(x):
    """(p0, p1, p2): three BF16 pieces, p0 = round(x), p1 = round(x - p0),
    p2 = round(x - p0 - p1).

    Generalisation of the residual split of Sec. V (Eq. 1 / Eq. 2) to a third
    piece, in the way Henry, Tang and Heinecke (2019, "Leveraging the bfloat16
    artificial intelligence datatype for higher-precision computations") split
    FP32 into BF16 triples: three 8-bit significands hold the 24 bits of an
    FP32 value, so p0 + p1 + p2 == x whenever no piece falls below the BF16
    normal range.  BF16 has the exponent range of FP32, so unlike FP16 pieces
    nothing overflows.
    """
    x = np.asarray(x, dtype=np.float64)
    p0 = round_to(x, "bf16")
    with np.errstate(invalid="ignore"):
        r = x - p0
        p1 = round_to(r, "bf16")
        p2 = round_to(r - p1, "bf16")
    return p0, p1, p2


# --- bit encodings (used to compare device outputs bit for bit) -------------

def f16_bits(values) -> np.ndarray:
    """IEEE binary16 bit patterns of values already representable in FP16."""
    return np.asarray(values, dtype=np.float64).astype(np.float16).view(np.uint16)


def bf16_bits(values) -> np.ndarray:
    """BF16 bit patterns (top half of the FP32 pattern) of representable values."""
    v = np.asarray(values, dtype=np.float64).astype(np.float32).view(np.uint32)
    return (v >> np.uint32(16)).astype(np.uint16)


def e4m3_bits(values) -> np.ndarray:
    """E4M3 (fn) bit patterns of values already representable in E4M3."""
    v = np.asarray(values, dtype=np.float64)
    out = np.zeros(v.shape, dtype=np.uint8)
    flat_v = v.reshape(-1)
    flat_o = out.reshape(-1)
    for i, val in enumerate(flat_v):
        sign = 0x80 if math.copysign(1.0, val) < 0 else 0
        a = abs(val)
        if math.isnan(a):
            flat_o[i] = sign | 0x7F
            continue
        if a == 0.0:
            flat_o[i] = sign
            continue
        m, E = math.frexp(a)
        e = E - 1
        if e < -6:          # subnormal: a = f * 2^-9, f in 1..7
            f = int(round(a * 2.0 ** 9))
            flat_o[i] = sign | f
        else:
            frac = int(round((a / 2.0 ** e - 1.0) * 8))
            flat_o[i] = sign | ((e + 7) << 3) | frac
    return out


def e4m3_value(bits) -> np.ndarray:
    """Decode E4M3 (fn) bit patterns to FP64 values."""
    b = np.asarray(bits, dtype=np.uint8).astype(np.int64)
    sign = np.where(b & 0x80, -1.0, 1.0)
    ex = (b >> 3) & 0xF
    fr = b & 7
    val = np.where(ex == 0, fr * 2.0 ** -9, (1.0 + fr / 8.0) * np.ldexp(1.0, ex - 7))
    val = np.where((ex == 15) & (fr == 7), np.nan, val)
    return sign * val
