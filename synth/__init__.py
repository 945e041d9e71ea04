"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the GEMM method: it only turns a seed into
FP32 matrices and problem/request shapes.  Every value is a function of
(seed, stream, index) through the Philox4x32-10 counter generator, so the same
call gives the same bits on any machine and in any process.

Distributions (the paper's own workloads are random FP32 matrices, Sec. VI and
VII-B; the shapes below reproduce them and the benchmark configurations):

* ``uniform(shape, seed, lo=-1, hi=1)``: x = lo + (hi-lo) * u with
  u = (r >> 8) * 2^-24, r a 32-bit Philox word.  For the symmetric ranges
  used here ([-1,1) and [-16,16)) every value is an exact FP32 number.
* ``normal(shape, seed)``: Box-Muller in FP64 from two words, rounded to FP32.
* ``log_uniform_pow2(shape, seed, emin=-8, emax=8)``: sign * 2^e * m with e an
  integer uniform in {emin..emax-1} and m uniform in [1, 2) on 23 bits.
* ``group_sizes(count, seed)``: m, n, k uniform over {16, 32, ..., 256}.
* ``serve_stream(count, seed, ...)``: Poisson arrivals, log-uniform sizes
  rounded up to a multiple of 16, a mode per request.

Seeds follow ``seed_for(config_index, matrix_id) = 1803_04014 + 1000 *
config_index + matrix_id`` (A=0, B=1, C0=2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()

BASE_SEED = 1803_04014


def seed_for(config_index: int, matrix_id: int) -> int:
    """Seed of matrix ``matrix_id`` (A=0, B=1, C0=2, ...) of configuration ``config_index``."""
    return BASE_SEED + 1000 * int(config_index) + int(matrix_id)


def build_lib() -> str:
    """Compile the Philox C file into a host shared object (gcc, no GPU)."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "philox.c")
    out = os.path.join(_BUILD, "libsynth_philox.so")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build_lib())
            lib.synth_philox_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                              ctypes.c_uint64, ctypes.c_void_p]
            lib.synth_philox_fill.restype = None
            lib.synth_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_philox4x32_10.restype = None
            _LIB = lib
    return _LIB


def philox_block(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block through the C implementation (4 uint32 words)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _lib().synth_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def philox_block_numpy(ctr, key) -> np.ndarray:
    """Plain restatement of Philox4x32-10 (used to cross-check the C file)."""
    M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
    c = [int(v) & 0xFFFFFFFF for v in ctr]
    k = [int(v) & 0xFFFFFFFF for v in key]
    for r in range(10):
        if r > 0:
            k = [(k[0] + W0) & 0xFFFFFFFF, (k[1] + W1) & 0xFFFFFFFF]
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & 0xFFFFFFFF, p1 & 0xFFFFFFFF,
             ((p0 >> 32) ^ c[3] ^ k[1]) & 0xFFFFFFFF, p0 & 0xFFFFFFFF]
    return np.array(c, dtype=np.uint32)


def words(n: int, seed: int, stream: int = 0, first: int = 0) -> np.ndarray:
    """``n`` consecutive 32-bit Philox words of (seed, stream), starting at word ``first``."""
    out = np.empty(int(n), dtype=np.uint32)
    if n:
        _lib().synth_philox_fill(int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream) & 0xFFFFFFFF, int(first),
                                 int(n), out.ctypes.data)
    return out


def _count(shape) -> int:
    return int(np.prod(shape, dtype=np.int64)) if len(shape) else 1


def unit24(r: np.ndarray) -> np.ndarray:
    """u = (r >> 8) * 2^-24 in [0, 1), exact in FP32 and FP64."""
    return (r >> np.uint32(8)).astype(np.float64) * (2.0 ** -24)


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0, stream: int = 0) -> np.ndarray:
    """FP32 matrix with entries lo + (hi - lo) * u (exact for lo = -hi, hi a power of two)."""
    shape = tuple(int(s) for s in shape)
    r = words(_count(shape), seed, stream)
    m, e = np.frexp(hi)
    if lo == -hi and hi > 0 and m == 0.5:
        # symmetric power-of-two range: (r>>8 - 2^23) * hi * 2^-23, exact in FP32
        x = ((r >> np.uint32(8)).astype(np.int32) - (1 << 23)).astype(np.float32)
        x *= np.float32(hi * 2.0 ** -23)
        return x.reshape(shape)
    x = lo + (hi - lo) * unit24(r)
    return x.astype(np.float32).reshape(shape)


def normal(shape, seed: int, stream: int = 0) -> np.ndarray:
    """FP32 matrix of N(0,1) draws (Box-Muller in FP64, rounded once to FP32)."""
    shape = tuple(int(s) for s in shape)
    n = _count(shape)
    m = (n + 1) // 2
    r = words(2 * m, seed, stream)
    u1 = ((r[0::2] >> np.uint32(8)).astype(np.float64) + 0.5) * (2.0 ** -24)
    u2 = (r[1::2] >> np.uint32(8)).astype(np.float64) * (2.0 ** -24)
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m, dtype=np.float64)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:n].astype(np.float32).reshape(shape)


def log_uniform_pow2(shape, seed: int, emin: int = -8, emax: int = 8, stream: int = 0) -> np.ndarray:
    """FP32 entries sign * 2^e * m, e uniform integer in [emin, emax), m in [1, 2) on 23 bits."""
    shape = tuple(int(s) for s in shape)
    span = emax - emin
    if span <= 0 or span > 256:
        raise ValueError("bad exponent range")
    r = words(_count(shape), seed, stream)
    sign = np.where((r >> np.uint32(31)) & np.uint32(1), -1.0, 1.0)
    # exponent from 8 bits (modulo the span; span 16 divides 256 so it is unbiased)
    e = ((r >> np.uint32(23)) & np.uint32(0xFF)).astype(np.int64) % span + emin
    mant = 1.0 + (r & np.uint32(0x7FFFFF)).astype(np.float64) * (2.0 ** -23)
    return (sign * np.ldexp(mant, e)).astype(np.float32).reshape(shape)


def integers(shape, seed: int, lo: int, hi: int, stream: int = 0) -> np.ndarray:
    """Integer-valued FP32 matrix, entries uniform in [lo, hi] (inclusive)."""
    shape = tuple(int(s) for s in shape)
    span = hi - lo + 1
    r = words(_count(shape), seed, stream).astype(np.uint64)
    v = (r * np.uint64(span)) >> np.uint64(32)
    return (v.astype(np.int64) + lo).astype(np.float32).reshape(shape)


def group_sizes(count: int, seed: int, step: int = 16, top: int = 256) -> np.ndarray:
    """(count, 3) int array of m, n, k uniform over {step, 2*step, ..., top}."""
    levels = top // step
    r = words(3 * int(count), seed, stream=7).astype(np.uint64)
    v = ((r * np.uint64(levels)) >> np.uint64(32)).astype(np.int64) + 1
    return (v * step).reshape(int(count), 3)


SERVE_MODES = ("f16", "bf16", "e4m3", "split3")


def serve_stream(count: int, seed: int, rate_per_s: float, lo: int = 32, hi: int = 4096,
                 align: int = 16):
    """Open-loop request stream.

    Returns (arrival_s, sizes[count,3], modes[count]) where arrivals are a
    Poisson process of the given rate, each of m, n, k is log-uniform in
    [lo, hi] rounded up to a multiple of ``align``, and the mode is uniform
    over ``SERVE_MODES``.
    """
    r = words(5 * int(count), seed, stream=11).reshape(int(count), 5)
    u = (unit24(r[:, 0]) + 2.0 ** -25)
    gaps = -np.log(u) / float(rate_per_s)
    arrival = np.cumsum(gaps) - gaps[0]
    ls = np.log(float(lo)) + (np.log(float(hi)) - np.log(float(lo))) * unit24(r[:, 1:4])
    sizes = np.ceil(np.exp(ls) / align).astype(np.int64) * align
    sizes = np.clip(sizes, align * ((lo + align - 1) // align), hi)
    modes = ((r[:, 4].astype(np.uint64) * np.uint64(len(SERVE_MODES))) >> np.uint64(32)).astype(np.int64)
    return arrival, sizes, modes
