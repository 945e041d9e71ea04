"""GPU parity: every kernel of the path through the C ABI against the CPU oracle.

Rounding, scaling and splitting are compared bit for bit; GEMMs element by
element within the FP32 accumulation bound and normwise within 1e-5 of the
oracle's result on the same rounded inputs.
"""
import time

import numpy as np
import pytest

import synth
from oracle import gemm as og
from oracle import numerics as nm
from tests.gpu_common import TOL_NORMWISE, dev, elementwise_ok, host, need_gpu, normwise_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    need_gpu()
    from paper_1803_04014_gb300 import binding
    binding.load()
    return binding


DT_NAME = {0: "f16", 1: "bf16", 2: "e4m3"}


def _quant_dev(b, dt, X, transpose=False):
    """Quantise FP32 numpy X on the GPU; returns (device tensor of codes, device scale word)."""
    rows, cols = X.shape
    xt = dev(X)
    tdt = {0: torch.float16, 1: torch.bfloat16, 2: torch.uint8}[dt]
    out = torch.empty((cols, rows) if transpose else (rows, cols), dtype=tdt, device="cuda")
    scale = torch.empty(1, dtype=torch.float32, device="cuda")
    ld = rows if transpose else cols
    b.tc_quantize(dt, rows, cols, xt, cols, out, ld, int(transpose), scale)
    return out, scale


def _codes_to_values(dt, t):
    if dt == 2:
        return nm.e4m3_value(host(t))
    return host(t.to(torch.float64))


# ------------------------------------------------------------------ rounding

@pytest.mark.parametrize("dt", [0, 1, 2])
@pytest.mark.parametrize("shape", [(64, 256), (37, 53), (1, 1), (130, 1000)])
@pytest.mark.parametrize("transpose", [False, True])
def test_quantize_bit_exact(b, dt, shape, transpose):
    X = synth.normal(shape, seed=synth.seed_for(1, 7)) * np.float32(30.0)
    q, scale = _quant_dev(b, dt, X, transpose)
    got = _codes_to_values(dt, q)
    if transpose:
        got = got.T
    want, s = nm.quantize(X, DT_NAME[dt])
    assert np.array_equal(got, want) and np.array_equal(np.signbit(got), np.signbit(want))
    if dt == 2:
        assert float(host(scale)[0]) == s


def test_quantize_special_values(b):
    X = np.float32([[0.0, -0.0, 65504.0, 65519.0, 65520.0, 1e30, -1e-30, 2.0 ** -25, 1.5 * 2.0 ** -25,
                     1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, np.inf, -np.inf, 5.96e-8, 3.0e-5, 7.0]])
    for dt in (0, 1):
        q, _ = _quant_dev(b, dt, X)
        got = _codes_to_values(dt, q)
        want = nm.round_to(X, DT_NAME[dt])
        assert np.array_equal(got, want) and np.array_equal(np.signbit(got), np.signbit(want))
    # E4M3: scale from the largest finite magnitude (no infinities here)
    Y = np.float32([[0.0, -0.0, 448.0, 1.0, -3.3, 1e-6, 2.0 ** -12, 0.017]])
    q, scale = _quant_dev(b, 2, Y)
    want, s = nm.quantize(Y, "e4m3")
    assert np.array_equal(_codes_to_values(2, q), want) and float(host(scale)[0]) == s


def test_quantize_e4m3_zero_matrix_scale_is_one(b):
    q, scale = _quant_dev(b, 2, np.zeros((8, 16), np.float32))
    assert float(host(scale)[0]) == 1.0 and not np.any(host(q))


@pytest.mark.parametrize("piece", [0, 1])
@pytest.mark.parametrize("shape,transpose", [((64, 128), False), ((33, 70), False), ((100, 48), True)])
def test_split_bit_exact(b, piece, shape, transpose):
    X = synth.log_uniform_pow2(shape, seed=synth.seed_for(3, 9))
    rows, cols = shape
    tdt = torch.float16 if piece == 0 else torch.bfloat16
    oshape = (cols, rows) if transpose else (rows, cols)
    hi = torch.empty(oshape, dtype=tdt, device="cuda")
    lo = torch.empty(oshape, dtype=tdt, device="cuda")
    b.tc_split(piece, rows, cols, dev(X), cols, int(transpose), hi, lo, oshape[1])
    h, l = host(hi.to(torch.float64)), host(lo.to(torch.float64))
    if transpose:
        h, l = h.T, l.T
    wh, wl = nm.split(X, DT_NAME[piece])
    assert np.array_equal(h, wh) and np.array_equal(l, wl)


# ------------------------------------------------------------------ mixed GEMM

def _run_mixed(b, dt, A, B, alpha=1.0, beta=0.0, C0=None):
    m, k = A.shape
    n = B.shape[1]
    aq, sa = _quant_dev(b, dt, A)
    bq, sb = _quant_dev(b, dt, B, transpose=True)   # K-major copy of B (n x k)
    C = dev(C0) if C0 is not None else torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    b.gemm_mixed(dt, m, n, k, alpha, aq, k, 0, bq, k, 1, beta, C, n,
                 sa if dt == 2 else None, sb if dt == 2 else None)
    b.tc_sync_status()
    return host(C)


def _mag(dt, A, B, alpha, beta, C0):
    Aq, sa = nm.quantize(A, DT_NAME[dt])
    Bq, sb = nm.quantize(B, DT_NAME[dt])
    mag = abs(alpha) * (np.abs(Aq) @ np.abs(Bq)) / (sa * sb)
    if beta != 0.0:
        mag = mag + abs(beta) * np.abs(C0.astype(np.float64))
    return mag


@pytest.mark.parametrize("dt", [0, 1, 2])
@pytest.mark.parametrize("mnk", [(256, 256, 256), (128, 256, 64), (300, 520, 136), (1, 1, 8), (129, 257, 1000),
                                 (640, 384, 2048)])
def test_gemm_mixed_parity(b, dt, mnk):
    m, n, k = mnk
    if dt == 2 and k % 16:
        k = (k + 15) // 16 * 16   # E4M3 rows must be 16-byte multiples
    A = synth.uniform((m, k), seed=synth.seed_for(0, 0))
    B = synth.uniform((k, n), seed=synth.seed_for(0, 1))
    C = _run_mixed(b, dt, A, B)
    ref = og.gemm_mixed(DT_NAME[dt], A, B)
    ok, info = elementwise_ok(C, ref, _mag(dt, A, B, 1.0, 0.0, None), k)
    assert ok, info
    assert normwise_dev(C, ref, A, B) <= TOL_NORMWISE


@pytest.mark.parametrize("dt", [0, 2])
def test_gemm_mixed_alpha_beta(b, dt):
    m, n, k = 200, 300, 512
    A = synth.normal((m, k), seed=11)
    B = synth.normal((k, n), seed=12)
    C0 = synth.uniform((m, n), seed=13)
    alpha, beta = 0.75, -1.5
    C = _run_mixed(b, dt, A, B, alpha, beta, C0)
    ref = og.gemm_mixed(DT_NAME[dt], A, B, alpha, beta, C0)
    ok, info = elementwise_ok(C, ref, _mag(dt, A, B, alpha, beta, C0), k)
    assert ok, info
    assert normwise_dev(C, ref, A, B, alpha, beta, C0) <= TOL_NORMWISE


def test_gemm_mixed_k_zero_scales_c(b):
    C0 = synth.uniform((10, 12), seed=3)
    C = dev(C0)
    a = torch.zeros(16, dtype=torch.float16, device="cuda")
    b.gemm_mixed(0, 10, 12, 0, 1.0, a, 8, 0, a, 8, 1, 0.5, C, 12)
    assert np.array_equal(host(C), (0.5 * C0.astype(np.float64)).astype(np.float32))


def test_gemm_mixed_rejects_unsupported_layouts(b):
    a = torch.zeros(64, dtype=torch.float16, device="cuda")
    a8 = torch.zeros(256, dtype=torch.uint8, device="cuda")
    s = torch.ones(1, dtype=torch.float32, device="cuda")
    c = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(b.TcError) as e:                     # column-major A
        b.gemm_mixed(0, 8, 8, 8, 1.0, a, 8, 1, a, 8, 1, 0.0, c, 8)
    assert e.value.status == b.TC_ERR_UNSUPPORTED
    with pytest.raises(b.TcError) as e:                     # row-major E4M3 B
        b.gemm_mixed(2, 8, 8, 16, 1.0, a8, 16, 0, a8, 16, 0, 0.0, c, 8, s, s)
    assert e.value.status == b.TC_ERR_UNSUPPORTED


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("mnk", [(300, 200, 160), (64, 256, 96), (520, 600, 1000), (2560, 2560, 128),
                                 (1000, 1032, 520)])
def test_gemm_mixed_row_major_b(b, dt, mnk):
    # B stored k x n (row-major) is read by the tensor cores as MN-major: no transposed copy
    m, n, k = mnk
    A = synth.uniform((m, k), seed=161)
    B = synth.uniform((k, n), seed=162)
    C0 = synth.uniform((m, n), seed=163)
    tdt = torch.float16 if dt == 0 else torch.bfloat16
    Aq = torch.empty((m, k), dtype=tdt, device="cuda")
    Bq = torch.empty((k, n), dtype=tdt, device="cuda")
    b.tc_quantize(dt, m, k, dev(A), k, Aq, k, 0)
    b.tc_quantize(dt, k, n, dev(B), n, Bq, n, 0)            # row-major, not transposed
    C = dev(C0)
    b.gemm_mixed(dt, m, n, k, 1.0, Aq, k, 0, Bq, n, 0, 0.5, C, n)
    b.tc_sync_status()
    ref = og.gemm_mixed(DT_NAME[dt], A, B, 1.0, 0.5, C0)
    ok, info = elementwise_ok(host(C), ref, _mag(dt, A, B, 1.0, 0.5, C0), k)
    assert ok, info


def test_gemm_mixed_is_deterministic(b):
    A = synth.uniform((384, 1024), seed=21)
    B = synth.uniform((1024, 512), seed=22)
    c1 = _run_mixed(b, 0, A, B)
    c2 = _run_mixed(b, 0, A, B)
    assert np.array_equal(c1, c2)


# ------------------------------------------------------------------ split GEMM (Eq. 1 / Eq. 2)

@pytest.mark.parametrize("piece", [0, 1])
@pytest.mark.parametrize("nprod", [2, 3, 4])
@pytest.mark.parametrize("layouts", [(0, 0), (1, 1), (0, 1)])
def test_gemm_split_parity(b, piece, nprod, layouts):
    m, n, k = 192, 320, 264
    la, lb = layouts
    A = synth.log_uniform_pow2((m, k), seed=synth.seed_for(2, 0))
    B = synth.log_uniform_pow2((k, n), seed=synth.seed_for(2, 1))
    Ad = dev(A if la == 0 else np.ascontiguousarray(A.T))
    Bd = dev(B if lb == 0 else np.ascontiguousarray(B.T))
    C0 = synth.uniform((m, n), seed=5)
    C = dev(C0)
    alpha, beta = 1.0, 0.5
    b.gemm_split(piece, nprod, m, n, k, alpha, Ad, k if la == 0 else m, la, Bd, n if lb == 0 else k, lb,
                 beta, C, n)
    b.tc_sync_status()
    got = host(C)
    ref = og.gemm_split(DT_NAME[piece], nprod, A, B, alpha, beta, C0)
    Ah, Al = nm.split(A, DT_NAME[piece])
    Bh, Bl = nm.split(B, DT_NAME[piece])
    mag = (np.abs(Ah) + np.abs(Al)) @ (np.abs(Bh) + np.abs(Bl)) + beta * np.abs(C0.astype(np.float64))
    ok, info = elementwise_ok(got, ref, mag, nprod * k)
    assert ok, info
    assert normwise_dev(got, ref, A, B, alpha, beta, C0) <= TOL_NORMWISE


def test_gemm_split_with_caller_workspace(b):
    m, n, k = 130, 70, 96
    A = synth.uniform((m, k), seed=31)
    B = synth.uniform((k, n), seed=32)
    nbytes = b.gemm_split_workspace_bytes(0, 3, m, n, k)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    b.gemm_split(0, 3, m, n, k, 1.0, dev(A), k, 0, dev(B), n, 0, 0.0, C, n, ws, nbytes)
    got = host(C)
    ref = og.gemm_split("f16", 3, A, B)
    assert normwise_dev(got, ref, A, B) <= TOL_NORMWISE


def test_split_of_half_inputs_matches_mixed(b):
    m, n, k = 128, 256, 192
    A = nm.round_to(synth.uniform((m, k), seed=41), "f16").astype(np.float32)
    B = nm.round_to(synth.uniform((k, n), seed=42), "f16").astype(np.float32)
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    b.gemm_split(0, 4, m, n, k, 1.0, dev(A), k, 0, dev(B), n, 0, 0.0, C, n)
    mixed = _run_mixed(b, 0, A, B)
    ref = og.gemm_mixed("f16", A, B)
    assert normwise_dev(host(C), ref, A, B) <= TOL_NORMWISE
    assert normwise_dev(mixed, ref, A, B) <= TOL_NORMWISE


# ------------------------------------------------------------------ SIMT FP32 GEMM

@pytest.mark.parametrize("layouts", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_sgemm_parity(b, layouts):
    m, n, k = 150, 260, 200
    la, lb = layouts
    A = synth.normal((m, k), seed=51)
    B = synth.normal((k, n), seed=52)
    C0 = synth.uniform((m, n), seed=53)
    C = dev(C0)
    b.gemm_sgemm(m, n, k, 1.25, dev(A if la == 0 else A.T), k if la == 0 else m, la,
                 dev(B if lb == 0 else B.T), n if lb == 0 else k, lb, 0.5, C, n)
    got = host(C)
    ref = og.gemm_truth(A, B, 1.25, 0.5, C0)
    mag = 1.25 * (np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))) + 0.5 * np.abs(C0)
    ok, info = elementwise_ok(got, ref, mag, k)
    assert ok, info


# ------------------------------------------------------------------ batched 16^3 (Listing 1's unit)

@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("lb", [0, 1])
@pytest.mark.parametrize("batch", [1, 31, 33, 1000])
def test_batched16_parity(b, dt, lb, batch):
    A = synth.uniform((batch, 16, 16), seed=61)
    B = synth.uniform((batch, 16, 16), seed=62)
    C0 = synth.uniform((batch, 16, 16), seed=63)
    tdt = torch.float16 if dt == 0 else torch.bfloat16
    Aq = dev(A, tdt)
    Bq = dev(B if lb == 0 else np.ascontiguousarray(B.transpose(0, 2, 1)), tdt)
    C = dev(C0)
    b.gemm_batched_strided(dt, batch, 16, 16, 16, 1.0, Aq, 256, 0, Bq, 256, lb, 0.25, C, 256)
    b.tc_sync_status()
    got = host(C)
    ref = og.gemm_batched(DT_NAME[dt], A, B, 1.0, 0.25, C0)
    assert np.max(np.abs(got - ref)) <= 16 * 2.0 ** -22 * 16


def test_batched16_padded_strides(b):
    batch = 50
    A = synth.uniform((batch, 16, 16), seed=64)
    B = synth.uniform((batch, 16, 16), seed=65)
    Ap = np.zeros((batch, 264), np.float32)
    Bp = np.zeros((batch, 272), np.float32)
    Ap[:, :256] = A.reshape(batch, 256)
    Bp[:, :256] = B.reshape(batch, 256)
    C = torch.zeros((batch, 260), dtype=torch.float32, device="cuda")
    b.gemm_batched_strided(0, batch, 16, 16, 16, 1.0, dev(Ap, torch.float16), 264, 0, dev(Bp, torch.float16), 272, 0,
                           0.0, C, 260)
    got = host(C)[:, :256].reshape(batch, 16, 16)
    ref = og.gemm_batched("f16", A, B)
    assert np.max(np.abs(got - ref)) <= 16 * 2.0 ** -22 * 16
    assert not np.any(host(C)[:, 256:])


# ------------------------------------------------------------------ grouped GEMM

def _grouped_case(count, seed, lb, ragged=False):
    # ragged: m, n, k each reduced by 0..8; "mk": only m and k, so every C_g row stays 16-byte aligned
    sizes = synth.group_sizes(count, seed)
    if ragged:
        sizes = sizes - (synth.words(sizes.size, seed=seed + 1).reshape(sizes.shape) % 9).astype(np.int64)
        if ragged == "mk":
            sizes[:, 1] = (sizes[:, 1] + 3) // 4 * 4
    rows, Ablocks, Bblocks = [], [], []
    oa = ob = oc = 0
    probs = []
    for g, (m, n, k) in enumerate(sizes):
        m, n, k = int(m), int(n), int(k)
        lda = (k + 7) // 8 * 8
        ldb = ((n if lb == 0 else k) + 7) // 8 * 8
        A = synth.uniform((m, k), seed=1000 + g)
        B = synth.uniform((k, n), seed=5000 + g)
        probs.append((m, n, k, oa, ob, oc, lda, ldb, n, A, B))
        oa += m * lda
        ob += (k if lb == 0 else n) * ldb
        oc += m * n
    abuf = np.zeros(oa, np.float32)
    bbuf = np.zeros(ob, np.float32)
    for (m, n, k, a0, b0, c0, lda, ldb, ldc, A, B) in probs:
        abuf[a0:a0 + m * lda].reshape(m, lda)[:, :k] = A
        if lb == 0:
            bbuf[b0:b0 + k * ldb].reshape(k, ldb)[:, :n] = B
        else:
            bbuf[b0:b0 + n * ldb].reshape(n, ldb)[:, :k] = B.T
    return probs, abuf, bbuf, oc


@pytest.mark.parametrize("lb", [0, 1])
@pytest.mark.parametrize("count,ragged", [(1, False), (7, False), (300, False), (50, True)])
def test_grouped_parity(b, lb, count, ragged):
    probs, abuf, bbuf, csize = _grouped_case(count, seed=70 + count, lb=lb, ragged=ragged)
    C = torch.zeros(csize, dtype=torch.float32, device="cuda")
    desc = [p[:9] for p in probs]
    b.gemm_grouped(0, desc, dev(abuf, torch.float16), 0, dev(bbuf, torch.float16), lb, C, 1.0, 0.0)
    got = host(C)
    for (m, n, k, a0, b0, c0, lda, ldb, ldc, A, B) in probs:
        ref = og.gemm_mixed("f16", A, B)
        g = got[c0:c0 + m * n].reshape(m, n)
        mag = np.abs(nm.round_to(A, "f16")) @ np.abs(nm.round_to(B, "f16"))
        ok, info = elementwise_ok(g, ref, mag, k)
        assert ok, (m, n, k, info)


def test_grouped_plan_graph_replay_and_beta(b):
    probs, abuf, bbuf, csize = _grouped_case(40, seed=90, lb=0)
    desc = [p[:9] for p in probs]
    plan = b.gemm_grouped_plan_create(0, desc, 0, 0)
    try:
        Ad, Bd = dev(abuf, torch.float16), dev(bbuf, torch.float16)
        C = torch.ones(csize, dtype=torch.float32, device="cuda")
        for _ in range(3):   # C <- A B + 0.5 C, three replays of the same graph
            b.gemm_grouped_plan_run(plan, Ad, Bd, C, 1.0, 0.5, use_graph=1)
        got = host(C)
    finally:
        b.gemm_grouped_plan_destroy(plan)
    for (m, n, k, a0, b0, c0, lda, ldb, ldc, A, B) in probs:
        p = og.gemm_mixed("f16", A, B)
        ref = p * (1 + 0.5 + 0.25) + 0.125
        g = got[c0:c0 + m * n].reshape(m, n)
        assert np.max(np.abs(g - ref)) <= 4 * k * 2.0 ** -22 * (np.max(np.abs(ref)) + 1)


# ------------------------------------------------------------------ FP64 error reduction

@pytest.mark.parametrize("m,n,k", [(333, 211, 97), (300, 1032, 96), (256, 512, 99), (2100, 4096, 8)])
def test_error_norm_matches_oracle(b, m, n, k):
    # 16-byte loads where every row is 16-byte aligned (n, k multiples of 4), scalar loads otherwise
    C = synth.uniform((m, n), seed=81)
    C64 = C.astype(np.float64) + synth.normal((m, n), seed=82).astype(np.float64) * 1e-3
    A = synth.uniform((m, k), seed=83)
    B = synth.uniform((k, n), seed=84)
    out = b.tc_error_norm(m, n, dev(C), n, dev(C64), n, 1, dev(A), m, k, k, dev(B), k, n, n)
    want = og.error_sums(C, C64, A, B)
    for g, w in zip(out, want):
        assert abs(g - w) <= 1e-12 * abs(w)
    # the FP32-reference form (the paper's e = C_half - C_single)
    out32 = b.tc_error_norm(m, n, dev(C), n, dev(C64.astype(np.float32)), n, 0)
    want32 = og.error_sums(C, C64.astype(np.float32), np.zeros(1), np.zeros(1))
    assert abs(out32[0] - want32[0]) <= 1e-12 * want32[0] and out32[3] == want32[3]
    # deterministic
    assert b.tc_error_norm(m, n, dev(C), n, dev(C64), n, 1, dev(A), m, k, k, dev(B), k, n, n) == out


@pytest.mark.parametrize("n", [64, 63])
def test_error_norm_special_values(b, n):
    # zeros of both signs, FP32 subnormals and the extremes of the normal range go through the
    # integer FP32 -> FP64 conversion and its fallback
    m, k = 40, 12
    specials = np.array([0.0, -0.0, 1e-40, -3e-39, 2.0 ** -126, -(2.0 ** -126), 3.4e38, -1.5, 2.0 ** -149],
                        dtype=np.float32)
    C = synth.uniform((m, n), seed=85)
    C.flat[: specials.size] = specials
    C64 = C.astype(np.float64)
    C64.flat[specials.size:] += synth.normal((m * n - specials.size,), seed=86).astype(np.float64) * 1e-6
    A = synth.uniform((m, k), seed=87)
    A.flat[: specials.size - 1] = specials[:-3].tolist() + [1e-45, -1e-44]
    B = synth.uniform((k, n), seed=88)
    out = b.tc_error_norm(m, n, dev(C), n, dev(C64), n, 1, dev(A), m, k, k, dev(B), k, n, n)
    want = og.error_sums(C, C64, A, B)
    for g, w in zip(out, want):
        assert abs(g - w) <= 1e-12 * abs(w)
    # only special values: C against its own exact FP64 copy gives exactly zero error, and the squares
    # of subnormals (~1e-80, normal in FP64) are summed exactly as the oracle sums them
    S = np.resize(specials, (2, 8)).astype(np.float32)
    sub = np.array([[1e-40, -3e-39, 2.0 ** -149, 1e-45, -(2.0 ** -127), 5e-39, 0.0, -0.0]], dtype=np.float32)
    out = b.tc_error_norm(2, 8, dev(S), 8, dev(S.astype(np.float64)), 8, 1, dev(sub), 1, 8, 8)
    want = og.error_sums(S, S.astype(np.float64), sub, np.zeros(1))
    assert out[0] == 0.0 and out[3] == 0.0
    assert abs(out[1] - want[1]) <= 1e-14 * want[1]


def test_error_norm_at_the_edges_of_the_float_float_range(b):
    # the squares are summed exactly as float-float groups only for 2^-50 <= |x| < 2^60 (values
    # outside take the FP64 path): put entries of A and B and differences C - C64 at and just past
    # both edges, mixed into the same groups of 4 and 8 as ordinary values
    edges = np.array([2.0 ** -50, -(2.0 ** -51), 1.99 * 2.0 ** 59, -(2.0 ** 60), 2.0 ** -49, -(2.0 ** 59)])
    m, n, k = 8, 24, 16
    A = synth.uniform((m, k), seed=89)
    B = synth.uniform((k, n), seed=90)
    for arr in (A, B):
        flat = arr.reshape(-1)
        for i, v in enumerate(edges):
            flat[3 * i + 1] = np.float32(v)   # spread over several groups, each beside ordinary values
    C = synth.uniform((m, n), seed=91)
    C64 = C.astype(np.float64) + synth.normal((m, n), seed=92).astype(np.float64) * 1e-4
    flatc, flat64 = C.reshape(-1), C64.reshape(-1)
    for i, v in enumerate(edges):
        j = 5 * i + 2
        flatc[j] = 0.0
        flat64[j] = -float(v)            # C - C64 = v exactly
    out = b.tc_error_norm(m, n, dev(C), n, dev(C64), n, 1, dev(A), m, k, k, dev(B), k, n, n)
    want = og.error_sums(C, C64, A, B)
    for g, w in zip(out, want):
        assert abs(g - w) <= 1e-12 * abs(w), (g, w)
    assert out[3] == want[3]


def test_error_norm_differences_taken_on_integers(b):
    # C - C64 is taken as an integer difference of aligned significands when both are normal with one
    # sign and exponents at most 1 apart, the result has at most 53 bits and lies in the float-float
    # range; everything else goes through the FP64 subtraction.  Pairs on both sides of each of those
    # lines, each in a group of 4 with ordinary values
    m, n = 8, 32
    C = synth.uniform((m, n), seed=97)
    C64 = C.astype(np.float64) + synth.normal((m, n), seed=98).astype(np.float64) * 1e-6
    pairs = [
        (1.0, 1.0 - 2.0 ** -30),          # exponents 1 apart
        (1.0, 1.0),                       # equal: difference 0
        (1.5, 0.75 + 2.0 ** -40),         # exponents 1 apart, 53 significant bits
        (1.75, 0.5 + 2.0 ** -53),         # exponents 1 apart, 54 significant bits: FP64 path
        (3.0, 0.7),                       # exponents 2 apart: FP64 path
        (1e-6, -1e-6),                    # opposite signs: FP64 path
        (1.0, 1.0 - 2.0 ** -50),          # difference 2^-50, the range's lower edge
        (1.0, 1.0 - 2.0 ** -52),          # difference 2^-52: FP64 path
        (-2.5, -2.5 + 2.0 ** -20),        # negative, same sign
        (2.0 ** 100, 2.0 ** 100 * (1 - 2.0 ** -45)),   # large values, difference 2^55
        (-(2.0 ** -100), -(2.0 ** -100) * (1 + 2.0 ** -20)),  # tiny values, difference 2^-120: FP64 path
    ]
    for i, (c, r) in enumerate(pairs):
        row, col = divmod(4 * i + 1 + (i % 3), n)
        C[row, col] = np.float32(c)
        C64[row, col] = r
    out = b.tc_error_norm(m, n, dev(C), n, dev(C64), n, 1)
    want = og.error_sums(C, C64, np.zeros(1), np.zeros(1))
    assert abs(out[0] - want[0]) <= 1e-12 * abs(want[0]), (out[0], want[0])
    assert out[3] == want[3]
    # the same against the FP64 path alone (rows of odd length: scalar loads, FP64 differences)
    Cs = np.zeros((m, n + 1), np.float32)
    Cs[:, :n] = C
    Rs = np.zeros((m, n + 1))
    Rs[:, :n] = C64
    outs = b.tc_error_norm(m, n + 1, dev(Cs), n + 1, dev(Rs), n + 1, 1)
    assert abs(outs[0] - want[0]) <= 1e-12 * abs(want[0]) and outs[3] == want[3]


def test_error_norm_dev_is_the_host_call_bit_for_bit(b):
    # the asynchronous form (device output, caller workspace) enqueues the same reduction
    m, n, k = 300, 260, 72
    C = synth.uniform((m, n), seed=93)
    C64 = C.astype(np.float64) + synth.normal((m, n), seed=94).astype(np.float64) * 1e-5
    A = synth.uniform((m, k), seed=95)
    B = synth.uniform((k, n), seed=96)
    args = (m, n, dev(C), n, dev(C64), n, 1, dev(A), m, k, k, dev(B), k, n, n)
    want = b.tc_error_norm(*args)
    ws_bytes = b.tc_error_norm_workspace_bytes()
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    b.tc_error_norm_dev(*args, out, ws, ws_bytes)
    got = tuple(host(out).tolist())
    assert got == want
    with pytest.raises(b.TcError) as e:
        b.tc_error_norm_dev(*args, out, ws, ws_bytes - 8)
    assert e.value.status == b.TC_ERR_INVALID


def test_binding_enqueues_on_torchs_current_stream(b):
    # entry points called without a stream go to torch's current stream, including inside a
    # stream context (the binding reads it through torch's raw-stream query when available)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        assert b._stream(None) == side.cuda_stream
    assert b._stream(None) == torch.cuda.current_stream().cuda_stream
    assert b._stream(side) == side.cuda_stream


# ------------------------------------------------------------------ both tile kernels (single CTA / CTA pair)

@pytest.mark.parametrize("tile", ["single", "pair"])
@pytest.mark.parametrize("dt", [0, 1, 2])
@pytest.mark.parametrize("mnk", [(64, 300, 96), (384, 640, 512), (1000, 260, 2048)])
def test_gemm_tile_kernels(b, monkeypatch, tile, dt, mnk):
    monkeypatch.setenv("TCGEMM_TILE", tile)
    m, n, k = mnk
    A = synth.uniform((m, k), seed=101)
    B = synth.uniform((k, n), seed=102)
    C0 = synth.uniform((m, n), seed=103)
    C = _run_mixed(b, dt, A, B, 1.0, 0.5, C0)
    ref = og.gemm_mixed(DT_NAME[dt], A, B, 1.0, 0.5, C0)
    ok, info = elementwise_ok(C, ref, _mag(dt, A, B, 1.0, 0.5, C0), k)
    assert ok, info
    assert normwise_dev(C, ref, A, B, 1.0, 0.5, C0) <= TOL_NORMWISE


@pytest.mark.parametrize("dt", [0, 1, 2])
@pytest.mark.parametrize("mnk", [(256, 256, 256), (1024, 1024, 1024), (1536, 1400, 208)])
def test_gemm_default_tiles_at_small_sizes(b, dt, mnk):
    # small sizes with the untuned tile choice: 8 and 128 single-CTA tiles of 128 x 64, and 132
    # of 128 x 128
    m, n, k = mnk
    A = synth.uniform((m, k), seed=151)
    B = synth.uniform((k, n), seed=152)
    C0 = synth.uniform((m, n), seed=153)
    C = _run_mixed(b, dt, A, B, 1.0, 0.5, C0)
    ref = og.gemm_mixed(DT_NAME[dt], A, B, 1.0, 0.5, C0)
    ok, info = elementwise_ok(C, ref, _mag(dt, A, B, 1.0, 0.5, C0), k)
    assert ok, info


@pytest.mark.parametrize("dt", [0, 1, 2])
@pytest.mark.parametrize("mnk", [(2560, 2560, 192), (2304, 2600, 320), (256, 2560, 128)])
def test_gemm_pair_full_and_half_width_units(b, monkeypatch, dt, mnk):
    # 100 and 99 tiles of 256 x 256 over 76 CTA pairs: the tiles of the partial last round run as
    # two units each after the full tiles; 10 tiles: every tile runs as two units.  K is short here,
    # so the units are 256 x 128 halves (parts of K from 48 k-blocks: test_gemm_pair_parts_of_k).
    monkeypatch.setenv("TCGEMM_TILE", "pair")
    m, n, k = mnk
    A = synth.uniform((m, k), seed=131)
    B = synth.uniform((k, n), seed=132)
    C0 = synth.uniform((m, n), seed=133)
    C = _run_mixed(b, dt, A, B, 1.0, -0.5, C0)
    ref = og.gemm_mixed(DT_NAME[dt], A, B, 1.0, -0.5, C0)
    ok, info = elementwise_ok(C, ref, _mag(dt, A, B, 1.0, -0.5, C0), k)
    assert ok, info
    assert np.array_equal(_run_mixed(b, dt, A, B, 1.0, -0.5, C0), C)
    # halves of N run the whole K chain of each element: the bits of whole tiles
    monkeypatch.setenv("TCGEMM_PAIR_TAIL", "halves")
    halves = _run_mixed(b, dt, A, B, 1.0, -0.5, C0)
    ok, info = elementwise_ok(halves, ref, _mag(dt, A, B, 1.0, -0.5, C0), k)
    assert ok, info
    monkeypatch.setenv("TCGEMM_PAIR_TAIL", "full")
    assert np.array_equal(_run_mixed(b, dt, A, B, 1.0, -0.5, C0), halves)


@pytest.mark.parametrize("epi", ["staged", "direct"])
@pytest.mark.parametrize("beta", [0.0, 0.75])
@pytest.mark.parametrize("case", ["f16", "e4m3", "f16_row_major_b"])
def test_gemm_pair_parts_of_k(b, monkeypatch, epi, beta, case):
    # parts of K on 24 cut tiles (100 tiles over 76 CTA pairs), K = 48 k-blocks (the first part 16,
    # 16 shorter than the second: the shortest K cut into parts); m and n ragged so that some
    # epilogue warps of cut tiles hold no rows of C and the last tiles hold a few columns; both
    # epilogues, beta 0 (the second part still reads what the first stored) and 0.75, E4M3 (k-blocks
    # of 128) with its scales and a row-major B read as MN-major.  The bits are the same every run.
    monkeypatch.setenv("TCGEMM_TILE", "pair")
    monkeypatch.setenv("TCGEMM_EPILOGUE", epi)
    dt = 2 if case == "e4m3" else 0
    m, n, k = 2500, 2520, 6144 if dt == 2 else 3072
    A = synth.uniform((m, k), seed=141)
    B = synth.uniform((k, n), seed=142)
    C0 = synth.uniform((m, n), seed=143)
    if case == "f16_row_major_b":
        Aq = torch.empty((m, k), dtype=torch.float16, device="cuda")
        Bq = torch.empty((k, n), dtype=torch.float16, device="cuda")
        b.tc_quantize(0, m, k, dev(A), k, Aq, k, 0)
        b.tc_quantize(0, k, n, dev(B), n, Bq, n, 0)
        C = dev(C0)
        b.gemm_mixed(0, m, n, k, 1.5, Aq, k, 0, Bq, n, 0, beta, C, n)
        b.tc_sync_status()
        got = host(C)
        C = dev(C0)
        b.gemm_mixed(0, m, n, k, 1.5, Aq, k, 0, Bq, n, 0, beta, C, n)
        b.tc_sync_status()
        again = host(C)
    else:
        got = _run_mixed(b, dt, A, B, 1.5, beta, C0)
        again = _run_mixed(b, dt, A, B, 1.5, beta, C0)
    ref = og.gemm_mixed(DT_NAME[dt], A, B, 1.5, beta, C0)
    ok, info = elementwise_ok(got, ref, _mag(dt, A, B, 1.5, beta, C0), k)
    assert ok, info
    assert np.array_equal(got, again)


def test_gemm_pair_parts_of_k_in_graphs_and_on_streams(b, monkeypatch):
    # parts of K signal through flags: an eager launch uses its stream's own flags and a token of its
    # own, a captured launch flags that the graph allocates and zeroes at each replay.  Eager launches
    # on three streams at once (one of them a graph replay) and repeated replays give the bits of one
    # launch alone.
    monkeypatch.setenv("TCGEMM_TILE", "pair")
    m, n, k = 2500, 2520, 3072
    A = synth.uniform((m, k), seed=181)
    B = synth.uniform((k, n), seed=182)
    C0 = dev(synth.uniform((m, n), seed=183))
    aq, _ = _quant_dev(b, 0, A)
    bq, _ = _quant_dev(b, 0, B, transpose=True)

    def launch(C, stream):
        b.gemm_mixed(0, m, n, k, 1.0, aq, k, 0, bq, k, 1, 0.5, C, n, stream=stream)

    main = torch.cuda.current_stream()
    alone = C0.clone()
    launch(alone, main)
    b.tc_sync_status()
    # a graph of one launch, replayed three times
    s_cap = torch.cuda.Stream()
    s_cap.wait_stream(main)
    Cg = C0.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s_cap):
        launch(Cg, s_cap)   # one eager launch first: set-up outside the capture
        torch.cuda.synchronize()
        Cg.copy_(C0)
        with torch.cuda.graph(g, stream=s_cap):
            launch(Cg, s_cap)
    main.wait_stream(s_cap)
    for _ in range(3):
        Cg.copy_(C0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        b.tc_sync_status()
        assert torch.equal(Cg, alone)
    # two eager streams and a replay at once
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    C1, C2 = C0.clone(), C0.clone()
    Cg.copy_(C0)
    torch.cuda.synchronize()
    for s_ in (s1, s2):
        s_.wait_stream(main)
    launch(C1, s1)
    launch(C2, s2)
    g.replay()
    torch.cuda.synchronize()
    b.tc_sync_status()
    assert torch.equal(C1, alone) and torch.equal(C2, alone) and torch.equal(Cg, alone)


@pytest.mark.parametrize("tile", ["single", "pair"])
@pytest.mark.parametrize("nprod", [2, 3, 4])
def test_split_tile_kernels(b, monkeypatch, tile, nprod):
    monkeypatch.setenv("TCGEMM_TILE", tile)
    m, n, k = 520, 264, 300
    A = synth.log_uniform_pow2((m, k), seed=111)
    B = synth.log_uniform_pow2((k, n), seed=112)
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    b.gemm_split(0, nprod, m, n, k, 1.0, dev(A), k, 0, dev(B), n, 0, 0.0, C, n)
    b.tc_sync_status()
    ref = og.gemm_split("f16", nprod, A, B)
    assert normwise_dev(host(C), ref, A, B) <= TOL_NORMWISE


# ------------------------------------------------------------------ accuracy gate of the refinement

@pytest.mark.parametrize("K", [1024, 4096])
def test_split3_error_within_2x_of_fp32_cuda_core_gemm(b, K):
    # inputs with full 24-bit significands over 16 binades; error vs the FP64 truth
    M = N = 256
    A = synth.log_uniform_pow2((M, K), seed=synth.seed_for(2, 0))
    B = synth.log_uniform_pow2((K, N), seed=synth.seed_for(2, 1))
    truth = og.gemm_truth(A, B)
    Ad, Bd = dev(A), dev(B)
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    b.gemm_split(0, 3, M, N, K, 1.0, Ad, K, 0, Bd, N, 0, 0.0, C, N)
    e_split = og.normwise_error(host(C), truth, A, B)
    b.gemm_sgemm(M, N, K, 1.0, Ad, K, 0, Bd, N, 0, 0.0, C, N)
    e_fp32 = og.normwise_error(host(C), truth, A, B)
    assert e_split <= 2.0 * e_fp32, (e_split, e_fp32)


@pytest.mark.parametrize("promote", ["0", "1", "2", "4"])
def test_split_promotion_settings_match_oracle(b, monkeypatch, promote):
    monkeypatch.setenv("TCGEMM_SPLIT_PROMOTE", promote)
    m, n, k = 384, 512, 1000
    A = synth.log_uniform_pow2((m, k), seed=121)
    B = synth.log_uniform_pow2((k, n), seed=122)
    C0 = synth.uniform((m, n), seed=123)
    C = dev(C0)
    b.gemm_split(0, 3, m, n, k, 1.5, dev(A), k, 0, dev(B), n, 0, -0.25, C, n)
    b.tc_sync_status()
    ref = og.gemm_split("f16", 3, A, B, 1.5, -0.25, C0)
    assert normwise_dev(host(C), ref, A, B, 1.5, -0.25, C0) <= TOL_NORMWISE


# ------------------------------------------------------------------ grouped GEMM: tensor-core and mma.sync kernels

@pytest.mark.parametrize("lb", [1, 0])
@pytest.mark.parametrize("impl", ["tc", "tc_direct", "mma"])
@pytest.mark.parametrize("count,ragged", [(1, False), (9, False), (400, False), (60, True), (60, "mk")])
def test_grouped_kmajor_parity(b, monkeypatch, lb, impl, count, ragged):
    # lb = 1: B_g K-major; lb = 0: B_g row-major (read by the tensor cores as MN-major).
    # tc: C chunks transposed through shared memory and stored as row segments (vector stores
    # where C_g rows are 16-byte aligned, ragged n is not); tc_direct: each lane stores its row.
    if impl == "mma":
        monkeypatch.setenv("TCGEMM_GROUPED", "mma")
    if impl == "tc_direct":
        monkeypatch.setenv("TCGEMM_GROUPED_EPI", "direct")
    probs, abuf, bbuf, csize = _grouped_case(count, seed=170 + count, lb=lb, ragged=ragged)
    C0 = synth.uniform((csize,), seed=77)
    C = dev(C0)
    desc = [p[:9] for p in probs]
    b.gemm_grouped(0, desc, dev(abuf, torch.float16), 0, dev(bbuf, torch.float16), lb, C, 0.75, -0.5)
    b.tc_sync_status()
    got = host(C)
    for (m, n, k, a0, b0, c0, lda, ldb, ldc, A, B) in probs:
        ref = og.gemm_mixed("f16", A, B, 0.75, -0.5, C0[c0:c0 + m * n].reshape(m, n))
        g = got[c0:c0 + m * n].reshape(m, n)
        mag = 0.75 * (np.abs(nm.round_to(A, "f16")) @ np.abs(nm.round_to(B, "f16"))) + 0.5 * np.abs(
            C0[c0:c0 + m * n].reshape(m, n))
        ok, info = elementwise_ok(g, ref, mag, k)
        assert ok, (m, n, k, info)


def test_grouped_tc_large_problems_and_new_bases(b):
    # problems above one 128 x 256 tile in both directions, and a second run on moved operands
    sizes = [(300, 520, 200), (129, 257, 72), (16, 16, 8), (256, 256, 256)]
    rows, a_parts, b_parts = [], [], []
    oa = ob = oc = 0
    data = []
    for i, (m, n, k) in enumerate(sizes):
        A = synth.uniform((m, k), seed=300 + i)
        B = synth.uniform((k, n), seed=400 + i)
        lda = (k + 7) // 8 * 8
        Ap = np.zeros((m, lda), np.float32); Ap[:, :k] = A
        Bp = np.zeros((n, lda), np.float32); Bp[:, :k] = B.T
        rows.append((m, n, k, oa, ob, oc, lda, lda, n))
        a_parts.append(Ap.ravel()); b_parts.append(Bp.ravel())
        data.append((m, n, k, oc, A, B))
        oa += Ap.size; ob += Bp.size; oc += m * n
    abuf = np.concatenate(a_parts); bbuf = np.concatenate(b_parts)
    plan = b.gemm_grouped_plan_create(0, rows, 0, 1)
    try:
        for shift in (0, 8):   # second run: same problems at other base addresses
            Ad = dev(np.concatenate([np.zeros(shift, np.float32), abuf]), torch.float16)[shift:]
            Bd = dev(np.concatenate([np.zeros(shift, np.float32), bbuf]), torch.float16)[shift:]
            C = torch.zeros(oc, dtype=torch.float32, device="cuda")
            b.gemm_grouped_plan_run(plan, Ad, Bd, C, 1.0, 0.0, use_graph=1)
            b.tc_sync_status()
            got = host(C)
            for (m, n, k, c0, A, B) in data:
                ref = og.gemm_mixed("f16", A, B)
                assert normwise_dev(got[c0:c0 + m * n].reshape(m, n), ref, A, B) <= TOL_NORMWISE, (m, n, k)
    finally:
        b.gemm_grouped_plan_destroy(plan)


@pytest.mark.parametrize("lb", [1, 0])
@pytest.mark.parametrize("epi", ["staged", "direct"])
@pytest.mark.parametrize("beta", [0.0, -0.75])
def test_grouped_transposed_problems(b, monkeypatch, lb, epi, beta):
    # m < n <= 256: the problem runs as C^T = B^T A^T (tall when m <= 128 < n) and its tiles are
    # stored to C transposed; with a row-major B, B^T is an MN-major A operand.  Against the oracle,
    # and against the untransposed run (TCGEMM_GROUPED_SWAP=0) within the same bound; odd m, n and
    # ldc (scalar stores), m = 1, m = n.
    monkeypatch.setenv("TCGEMM_GROUPED_EPI", epi)
    sizes = [(32, 256, 32), (16, 200, 96), (100, 240, 64), (129, 250, 40), (200, 256, 128), (1, 17, 16),
             (7, 9, 24), (64, 64, 64), (250, 256, 200), (120, 130, 8), (300, 100, 64), (48, 512, 32)]
    rows, a_parts, b_parts, data = [], [], [], []
    oa = ob = oc = 0
    for i, (m, n, k) in enumerate(sizes):
        A = synth.uniform((m, k), seed=800 + i)
        B = synth.uniform((k, n), seed=900 + i)
        lda = (k + 7) // 8 * 8
        Ap = np.zeros((m, lda), np.float32); Ap[:, :k] = A
        if lb == 1:
            ldb = lda
            Bp = np.zeros((n, ldb), np.float32); Bp[:, :k] = B.T
        else:
            ldb = (n + 7) // 8 * 8
            Bp = np.zeros((k, ldb), np.float32); Bp[:, :n] = B
        ldc = n + (i % 3)   # padded rows of C: 0, 1 or 2 extra floats
        rows.append((m, n, k, oa, ob, oc, lda, ldb, ldc))
        a_parts.append(Ap.ravel()); b_parts.append(Bp.ravel())
        data.append((m, n, k, oc, ldc, A, B))
        oa += Ap.size; ob += Bp.size; oc += m * ldc
    Ad = dev(np.concatenate(a_parts), torch.float16)
    Bd = dev(np.concatenate(b_parts), torch.float16)
    C0 = synth.uniform((oc,), seed=999)
    out = {}
    for swap in ("1", "0"):
        monkeypatch.setenv("TCGEMM_GROUPED_SWAP", swap)
        C = dev(C0)
        b.gemm_grouped(0, rows, Ad, 0, Bd, lb, C, 1.25, beta)
        b.tc_sync_status()
        out[swap] = host(C)
    # the same bits every run
    monkeypatch.setenv("TCGEMM_GROUPED_SWAP", "1")
    C = dev(C0)
    b.gemm_grouped(0, rows, Ad, 0, Bd, lb, C, 1.25, beta)
    b.tc_sync_status()
    assert np.array_equal(host(C), out["1"])
    for (m, n, k, c0, ldc, A, B) in data:
        Cg0 = C0[c0:c0 + m * ldc].reshape(m, ldc)
        ref = og.gemm_mixed("f16", A, B, 1.25, beta, Cg0[:, :n])
        mag = 1.25 * (np.abs(nm.round_to(A, "f16")) @ np.abs(nm.round_to(B, "f16"))) + abs(beta) * np.abs(Cg0[:, :n])
        for swap in ("1", "0"):
            g = out[swap][c0:c0 + m * ldc].reshape(m, ldc)
            ok, info = elementwise_ok(g[:, :n], ref, mag, k)
            assert ok, (swap, m, n, k, info)
            # the row padding is never written
            assert np.array_equal(g[:, n:], Cg0[:, n:]), (swap, m, n, k)


@pytest.mark.parametrize("lb", [1, 0])
@pytest.mark.parametrize("epi", ["staged", "direct"])
def test_grouped_tall_tiles_match_128_row_tiles(b, monkeypatch, lb, epi):
    # tall 256-row tiles (problems with n <= 128: M-blocks tm and tm + 1 share one B tile and one
    # accumulator buffer) against 128 x 256 tiles only: each element is the same MMA chain, so the
    # bits agree.  Problems with 1 to 5 M-blocks (an odd last block stays 128 rows), one row into the
    # second block, n at, below and past 128 (those stay 128-row tiles) and past 256.
    monkeypatch.setenv("TCGEMM_GROUPED_EPI", epi)
    sizes = [(129, 40, 64), (256, 256, 256), (300, 520, 200), (513, 100, 72), (640, 264, 136), (200, 16, 8),
             (96, 96, 96), (384, 250, 192), (257, 128, 64), (384, 112, 520)]
    rows, a_parts, b_parts = [], [], []
    oa = ob = oc = 0
    for i, (m, n, k) in enumerate(sizes):
        A = synth.uniform((m, k), seed=600 + i)
        B = synth.uniform((k, n), seed=700 + i)
        lda = (k + 7) // 8 * 8
        Ap = np.zeros((m, lda), np.float32); Ap[:, :k] = A
        if lb == 1:
            ldb = lda
            Bp = np.zeros((n, ldb), np.float32); Bp[:, :k] = B.T
        else:
            ldb = (n + 7) // 8 * 8
            Bp = np.zeros((k, ldb), np.float32); Bp[:, :n] = B
        rows.append((m, n, k, oa, ob, oc, lda, ldb, n))
        a_parts.append(Ap.ravel()); b_parts.append(Bp.ravel())
        oa += Ap.size; ob += Bp.size; oc += m * n
    Ad = dev(np.concatenate(a_parts), torch.float16)
    Bd = dev(np.concatenate(b_parts), torch.float16)
    C0 = dev(synth.uniform((oc,), seed=777))
    out = {}
    for tall in ("1", "0"):
        monkeypatch.setenv("TCGEMM_GROUPED_TALL", tall)
        C = C0.clone()
        b.gemm_grouped(0, rows, Ad, 0, Bd, lb, C, 1.25, 0.5)
        b.tc_sync_status()
        out[tall] = C
    assert torch.equal(out["1"], out["0"])


# ------------------------------------------------------------------ autotuner

@pytest.mark.parametrize("dt", [0, 2])
def test_autotuned_gemm_still_matches_oracle(b, dt):
    m, n, k = 640, 768, 512
    ms = b.tc_autotune_gemm(dt, m, n, k)
    assert 0.0 < ms < 100.0
    A = synth.uniform((m, k), seed=501)
    B = synth.uniform((k, n), seed=502)
    C = _run_mixed(b, dt, A, B)
    ref = og.gemm_mixed(DT_NAME[dt], A, B)
    assert normwise_dev(C, ref, A, B) <= TOL_NORMWISE


@pytest.mark.parametrize("dt", [0, 1, 2])
@pytest.mark.parametrize("mnk", [(512, 512, 512), (300, 770, 208), (1024, 1280, 1008), (2304, 2560, 640),
                                 (256, 256, 64)])
def test_gemm_on_clusters_of_four_sharing_a_by_multicast(b, monkeypatch, dt, mnk):
    # TCGEMM_CLUSTER=4: two CTA pairs per cluster take adjacent tiles of a row band and multicast
    # their A quarters to each other.  Shapes: one unit, ragged m/n/k with an odd number of tile
    # columns (the second pair of the last unit has no tile), several rounds of units (odd rounds
    # walk K downwards), a single tile.  Same tolerance as the pair kernel; with K walked upwards
    # everywhere and whole tiles, equal to the pair kernel bit for bit (the products of a tile are
    # issued in the same order)
    m, n, k = mnk
    A = synth.uniform((m, k), seed=521)
    B = synth.uniform((k, n), seed=522)
    C0 = synth.uniform((m, n), seed=523)
    monkeypatch.setenv("TCGEMM_CLUSTER", "4")
    got = _run_mixed(b, dt, A, B, beta=0.5, C0=C0)
    ref = og.gemm_mixed(DT_NAME[dt], A, B, 1.0, 0.5, C0)
    ok, info = elementwise_ok(got, ref, _mag(dt, A, B, 1.0, 0.5, C0), k)
    assert ok, info
    monkeypatch.setenv("TCGEMM_K_ORDER", "forward")
    quad_fwd = _run_mixed(b, dt, A, B, beta=0.5, C0=C0)
    monkeypatch.setenv("TCGEMM_CLUSTER", "2")
    monkeypatch.setenv("TCGEMM_PAIR_TAIL", "full")
    pair_fwd = _run_mixed(b, dt, A, B, beta=0.5, C0=C0)
    assert np.array_equal(quad_fwd, pair_fwd)


def test_autotuning_on_one_thread_leaves_another_threads_gemms_alone(b):
    # while one thread times candidate configurations of a shape class, another issues gemm_mixed on
    # the same class: each call resolves its configuration when it is issued, and every result is
    # the one of the configuration before the table was updated or the one after it (candidates are
    # passed explicitly, never through state other threads read)
    import threading
    m, n, k = 1024, 1536, 1536   # > 76 tiles of 256 x 256: candidates differ in K order and tail
    A = synth.uniform((m, k), seed=511)
    B = synth.uniform((k, n), seed=512)
    Ad, Bd = dev(A), dev(B)
    Aq = torch.empty((m, k), dtype=torch.float16, device="cuda")
    Bq = torch.empty((n, k), dtype=torch.float16, device="cuda")
    b.tc_quantize(0, m, k, Ad, k, Aq, k, 0)
    b.tc_quantize(0, k, n, Bd, n, Bq, k, 1)
    s_tune, s_call = torch.cuda.Stream(), torch.cuda.Stream()
    outs = [torch.zeros((m, n), dtype=torch.float32, device="cuda") for _ in range(65)]
    torch.cuda.synchronize()

    def call(C):
        with torch.cuda.stream(s_call):
            b.gemm_mixed(0, m, n, k, 1.0, Aq, k, 0, Bq, k, 1, 0.0, C, n)

    call(outs[0])                      # the configuration before tuning
    errors = []

    def tuner():
        try:
            b.tc_autotune_gemm(0, m, n, k, stream=s_tune.cuda_stream)
        except Exception as e:  # surfaced below
            errors.append(e)

    t = threading.Thread(target=tuner)
    t.start()
    issued_during = 0
    i = 1
    while i < len(outs) - 1 and t.is_alive():
        call(outs[i])
        issued_during += 1 if t.is_alive() else 0
        i += 1
        time.sleep(0.0005)
    t.join()
    call(outs[-1])                     # the configuration after tuning
    torch.cuda.synchronize()
    b.tc_sync_status()
    assert not errors, errors
    assert issued_during >= 1
    before, after = outs[0], outs[-1]
    for C in outs[1:i]:
        assert torch.equal(C, before) or torch.equal(C, after)
    ref = og.gemm_mixed("f16", A, B)
    assert normwise_dev(host(after), ref, A, B) <= TOL_NORMWISE


def test_autotuned_grouped_plan_still_matches_oracle(b):
    probs, abuf, bbuf, csize = _grouped_case(120, seed=503, lb=1)
    desc = [p[:9] for p in probs]
    Ad, Bd = dev(abuf, torch.float16), dev(bbuf, torch.float16)
    C = torch.zeros(csize, dtype=torch.float32, device="cuda")
    plan = b.gemm_grouped_plan_create(0, desc, 0, 1)
    try:
        ms = b.gemm_grouped_plan_autotune(plan, Ad, Bd, C)
        assert 0.0 < ms < 100.0
        C.zero_()
        b.gemm_grouped_plan_run(plan, Ad, Bd, C, 1.0, 0.0, use_graph=1)
        b.tc_sync_status()
        got = host(C)
    finally:
        b.gemm_grouped_plan_destroy(plan)
    for (m, n, k, a0, b0, c0, lda, ldb, ldc, A, B) in probs:
        ref = og.gemm_mixed("f16", A, B)
        assert normwise_dev(got[c0:c0 + m * n].reshape(m, n), ref, A, B) <= TOL_NORMWISE


# ------------------------------------------------------------------ padded leading dimensions

@pytest.mark.parametrize("tile", ["single", "pair"])
@pytest.mark.parametrize("dt", [0, 1, 2])
def test_gemm_mixed_padded_leading_dims(b, monkeypatch, tile, dt):
    # operands and C with row padding full of NaN: nothing may read or write the padding
    monkeypatch.setenv("TCGEMM_TILE", tile)
    m, n, k = 300, 200, 160
    pad = 16 if dt == 2 else 8
    lda, ldb, ldc = k + pad, k + 2 * pad, n + 3
    A = synth.uniform((m, k), seed=141)
    B = synth.uniform((k, n), seed=142)
    C0 = synth.uniform((m, n), seed=143)
    tdt = {0: torch.float16, 1: torch.bfloat16, 2: torch.uint8}[dt]
    if dt == 2:
        Aq = torch.full((m, lda), 0x7F, dtype=tdt, device="cuda")   # E4M3 NaN
        Bq = torch.full((n, ldb), 0x7F, dtype=tdt, device="cuda")
    else:
        Aq = torch.full((m, lda), float("nan"), dtype=tdt, device="cuda")
        Bq = torch.full((n, ldb), float("nan"), dtype=tdt, device="cuda")
    sc = torch.empty(2, dtype=torch.float32, device="cuda")
    b.tc_quantize(dt, m, k, dev(A), k, Aq, lda, 0, sc[0:1])
    b.tc_quantize(dt, k, n, dev(B), n, Bq, ldb, 1, sc[1:2])
    Cfull = torch.full((m, ldc), float("nan"), dtype=torch.float32, device="cuda")
    Cfull[:, :n] = dev(C0)
    b.gemm_mixed(dt, m, n, k, 1.0, Aq, lda, 0, Bq, ldb, 1, 0.5, Cfull, ldc,
                 sc[0:1] if dt == 2 else None, sc[1:2] if dt == 2 else None)
    b.tc_sync_status()
    got = host(Cfull)
    assert np.all(np.isnan(got[:, n:]))
    ref = og.gemm_mixed(DT_NAME[dt], A, B, 1.0, 0.5, C0)
    ok, info = elementwise_ok(got[:, :n], ref, _mag(dt, A, B, 1.0, 0.5, C0), k)
    assert ok, info


@pytest.mark.parametrize("layouts", [(0, 0), (1, 1)])
def test_gemm_split_padded_fp32_operands(b, layouts):
    # FP32 inputs with odd row pitches (the scalar split path) and C with padding
    la, lb = layouts
    m, n, k = 260, 136, 200
    A = synth.log_uniform_pow2((m, k), seed=151)
    B = synth.log_uniform_pow2((k, n), seed=152)
    if la == 0:
        lda = k + 3
        Ap = np.full((m, lda), np.nan, np.float32)
        Ap[:, :k] = A
    else:
        lda = m + 5
        Ap = np.full((k, lda), np.nan, np.float32)
        Ap[:, :m] = A.T
    if lb == 0:
        ldb = n + 1
        Bp = np.full((k, ldb), np.nan, np.float32)
        Bp[:, :n] = B
    else:
        ldb = k + 7
        Bp = np.full((n, ldb), np.nan, np.float32)
        Bp[:, :k] = B.T
    ldc = n + 5
    C = torch.full((m, ldc), float("nan"), dtype=torch.float32, device="cuda")
    b.gemm_split(0, 3, m, n, k, 1.0, dev(Ap), lda, la, dev(Bp), ldb, lb, 0.0, C, ldc)
    b.tc_sync_status()
    got = host(C)
    assert np.all(np.isnan(got[:, n:]))
    ref = og.gemm_split("f16", 3, A, B)
    assert normwise_dev(got[:, :n], ref, A, B) <= TOL_NORMWISE
