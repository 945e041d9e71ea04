"""GPU parity of the refinements beyond Eq. 1 / Eq. 2: the scaled-residual
split (Ootomo and Yokota, 2022) and the three-piece BF16 split (Henry, Tang
and Heinecke, 2019), each against the CPU oracle, plus their accuracy against
the FP64 truth next to the FP32 CUDA-core GEMM.
"""
import numpy as np
import pytest

import synth
from oracle import gemm as og
from oracle import numerics as nm
from tests.gpu_common import TOL_NORMWISE, dev, elementwise_ok, host, need_gpu, normwise_dev, torch

pytestmark = pytest.mark.gpu

DT_NAME = {0: "f16", 1: "bf16"}


@pytest.fixture(scope="module")
def b():
    need_gpu()
    from paper_1803_04014_gb300 import binding
    binding.load()
    return binding


def _bits_matrix(shape, seed, e_lo, e_hi):
    """FP32 values with full 24-bit significands, exponents uniform in [e_lo, e_hi)."""
    n = int(np.prod(shape))
    ints = (synth.words(n, seed=seed) & np.uint32((1 << 23) - 1)).astype(np.float64) + float(1 << 23)
    e = (synth.words(n, seed=seed + 1) % (e_hi - e_lo)).astype(np.float64) + e_lo
    sgn = np.where(synth.words(n, seed=seed + 2) & np.uint32(1), -1.0, 1.0)
    return (sgn * ints * 2.0 ** (e - 23)).astype(np.float32).reshape(shape)


# ------------------------------------------------------------------ piece formation, bit for bit

@pytest.mark.parametrize("piece", [0, 1])
@pytest.mark.parametrize("shape,transpose", [((64, 128), False), ((33, 70), False), ((100, 48), True)])
def test_split_scaled_bit_exact(b, piece, shape, transpose):
    X = _bits_matrix(shape, synth.seed_for(5, 0), -16, 8)
    rows, cols = shape
    tdt = torch.float16 if piece == 0 else torch.bfloat16
    oshape = (cols, rows) if transpose else (rows, cols)
    hi = torch.empty(oshape, dtype=tdt, device="cuda")
    lo = torch.empty(oshape, dtype=tdt, device="cuda")
    b.tc_split_scaled(piece, rows, cols, dev(X), cols, int(transpose), hi, lo, oshape[1])
    h, l = host(hi.to(torch.float64)), host(lo.to(torch.float64))
    if transpose:
        h, l = h.T, l.T
    wh, wl = nm.split_scaled(X, DT_NAME[piece])
    assert np.array_equal(h, wh) and np.array_equal(l, wl)


@pytest.mark.parametrize("shape,transpose", [((64, 128), False), ((33, 70), False), ((100, 48), True),
                                             ((257, 96), True)])
def test_split_bf16x3_bit_exact(b, shape, transpose):
    X = _bits_matrix(shape, synth.seed_for(5, 3), -60, 60)
    rows, cols = shape
    oshape = (cols, rows) if transpose else (rows, cols)
    ps = [torch.empty(oshape, dtype=torch.bfloat16, device="cuda") for _ in range(3)]
    b.tc_split_bf16x3(rows, cols, dev(X), cols, int(transpose), ps[0], ps[1], ps[2], oshape[1])
    got = [host(p.to(torch.float64)) for p in ps]
    if transpose:
        got = [g.T for g in got]
    want = nm.split_bf16x3(X)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    assert np.array_equal(got[0] + got[1] + got[2], X.astype(np.float64))


# ------------------------------------------------------------------ GEMM parity

@pytest.mark.parametrize("piece", [0, 1])
@pytest.mark.parametrize("nprod", [2, 3])
@pytest.mark.parametrize("layouts", [(0, 0), (1, 1), (0, 1)])
def test_gemm_split_scaled_parity(b, piece, nprod, layouts):
    m, n, k = 192, 320, 264
    la, lb = layouts
    A = synth.log_uniform_pow2((m, k), seed=synth.seed_for(5, 10))
    B = synth.log_uniform_pow2((k, n), seed=synth.seed_for(5, 11))
    Ad = dev(A if la == 0 else np.ascontiguousarray(A.T))
    Bd = dev(B if lb == 0 else np.ascontiguousarray(B.T))
    C0 = synth.uniform((m, n), seed=5)
    C = dev(C0)
    alpha, beta = 1.0, 0.5
    b.gemm_split_scaled(piece, nprod, m, n, k, alpha, Ad, k if la == 0 else m, la, Bd, n if lb == 0 else k, lb,
                        beta, C, n)
    b.tc_sync_status()
    got = host(C)
    ref = og.gemm_split_scaled(DT_NAME[piece], nprod, A, B, alpha, beta, C0)
    s = nm.SPLIT_SCALE_EXP[DT_NAME[piece]]
    Ah, Al = nm.split_scaled(A, DT_NAME[piece])
    Bh, Bl = nm.split_scaled(B, DT_NAME[piece])
    mag = (np.abs(Ah) + np.ldexp(np.abs(Al), -s)) @ (np.abs(Bh) + np.ldexp(np.abs(Bl), -s)) + \
        beta * np.abs(C0.astype(np.float64))
    ok, info = elementwise_ok(got, ref, mag, nprod * k)
    assert ok, info
    assert normwise_dev(got, ref, A, B, alpha, beta, C0) <= TOL_NORMWISE


@pytest.mark.parametrize("promote", ["2", "4"])
@pytest.mark.parametrize("mnk", [(520, 600, 1000), (256, 256, 64), (100, 40, 8), (300, 520, 2048)])
def test_gemm_split_scaled_shapes(b, monkeypatch, promote, mnk):
    # several tiles and chunks, ragged edges, k shorter than one promotion chunk; both chunk lengths
    monkeypatch.setenv("TCGEMM_SPLIT_PROMOTE", promote)
    m, n, k = mnk
    A = synth.uniform((m, k), seed=200)
    B = synth.uniform((k, n), seed=201)
    C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    b.gemm_split_scaled(0, 3, m, n, k, -1.25, dev(A), k, 0, dev(B), n, 0, 0.0, C, n)
    b.tc_sync_status()
    got = host(C)
    ref = og.gemm_split_scaled("f16", 3, A, B, -1.25)
    mag = 1.25 * np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    ok, info = elementwise_ok(got, ref, mag, 3 * k)
    assert ok, info


@pytest.mark.parametrize("layouts", [(0, 0), (1, 1), (0, 1), (1, 0)])
@pytest.mark.parametrize("mnk", [(192, 320, 264), (520, 300, 1000)])
def test_gemm_split_bf16x3_parity(b, layouts, mnk):
    _bf16x3_case(b, layouts, mnk)


@pytest.mark.parametrize("promote", ["2", "4"])
def test_gemm_split_bf16x3_chunk_lengths(b, monkeypatch, promote):
    monkeypatch.setenv("TCGEMM_SPLIT_PROMOTE", promote)
    _bf16x3_case(b, (0, 0), (300, 520, 1100))


def _bf16x3_case(b, layouts, mnk):
    m, n, k = mnk
    la, lb = layouts
    A = _bits_matrix((m, k), synth.seed_for(5, 20), -40, 40)
    B = _bits_matrix((k, n), synth.seed_for(5, 21), -40, 40)
    Ad = dev(A if la == 0 else np.ascontiguousarray(A.T))
    Bd = dev(B if lb == 0 else np.ascontiguousarray(B.T))
    C0 = synth.uniform((m, n), seed=7)
    C = dev(C0)
    alpha, beta = 0.75, -0.5
    b.gemm_split_bf16x3(m, n, k, alpha, Ad, k if la == 0 else m, la, Bd, n if lb == 0 else k, lb, beta, C, n)
    b.tc_sync_status()
    got = host(C)
    ref = og.gemm_split_bf16x3(A, B, alpha, beta, C0)
    mag = alpha * np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)) + abs(beta) * np.abs(C0.astype(np.float64))
    ok, info = elementwise_ok(got, ref, mag, 6 * k)
    assert ok, info
    assert normwise_dev(got, ref, A, B, alpha, beta, C0) <= TOL_NORMWISE


def test_gemm_split_bf16x3_caller_workspace_and_k0(b):
    m, n, k = 130, 70, 96
    A = synth.uniform((m, k), seed=31)
    B = synth.uniform((k, n), seed=32)
    nbytes = b.gemm_split_workspace_bytes(1, 6, m, n, k)
    assert nbytes >= 3 * (m + n) * k * 2
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    b.gemm_split_bf16x3(m, n, k, 1.0, dev(A), k, 0, dev(B), n, 0, 0.0, C, n, ws, nbytes)
    b.tc_sync_status()
    assert normwise_dev(host(C), og.gemm_split_bf16x3(A, B), A, B) <= TOL_NORMWISE
    with pytest.raises(b.TcError):
        b.gemm_split_bf16x3(m, n, k, 1.0, dev(A), k, 0, dev(B), n, 0, 0.0, C, n, ws, nbytes - 256)
    # k = 0: C = beta * C
    C0 = synth.uniform((m, n), seed=33)
    C = dev(C0)
    b.gemm_split_bf16x3(m, n, 0, 1.0, dev(A), k, 0, dev(B), n, 0, 2.0, C, n)
    assert np.array_equal(host(C), 2.0 * C0)
    with pytest.raises(b.TcError):
        b.gemm_split_scaled(0, 4, m, n, k, 1.0, dev(A), k, 0, dev(B), n, 0, 0.0, C, n)


# ------------------------------------------------------------------ accuracy against the FP64 truth

def test_scaled_split_recovers_small_magnitudes(b):
    # |x| in [2^-12, 2^-10): plain FP16 residuals are subnormal and lose bits, scaled ones stay normal
    M = N = 256
    K = 1024
    A = _bits_matrix((M, K), 300, -12, -10)
    B = _bits_matrix((K, N), 310, -12, -10)
    truth = og.gemm_truth(A, B)
    Ad, Bd = dev(A), dev(B)
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    b.gemm_split_scaled(0, 3, M, N, K, 1.0, Ad, K, 0, Bd, N, 0, 0.0, C, N)
    e_scaled = og.normwise_error(host(C), truth, A, B)
    b.gemm_split(0, 3, M, N, K, 1.0, Ad, K, 0, Bd, N, 0, 0.0, C, N)
    e_plain = og.normwise_error(host(C), truth, A, B)
    b.gemm_sgemm(M, N, K, 1.0, Ad, K, 0, Bd, N, 0, 0.0, C, N)
    e_fp32 = og.normwise_error(host(C), truth, A, B)
    assert e_scaled <= 2.0 * e_fp32, (e_scaled, e_fp32)
    assert e_plain > 10.0 * e_scaled, (e_plain, e_scaled)


def test_bf16x3_keeps_fp32_accuracy_over_a_wide_range(b):
    # exponents over 60 binades: FP16 pieces overflow and underflow, three BF16 pieces do not
    M = N = 256
    K = 1024
    A = _bits_matrix((M, K), 320, -30, 30)
    B = _bits_matrix((K, N), 330, -30, 30)
    truth = og.gemm_truth(A, B)
    Ad, Bd = dev(A), dev(B)
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    b.gemm_split_bf16x3(M, N, K, 1.0, Ad, K, 0, Bd, N, 0, 0.0, C, N)
    e_x3 = og.normwise_error(host(C), truth, A, B)
    b.gemm_split(1, 4, M, N, K, 1.0, Ad, K, 0, Bd, N, 0, 0.0, C, N)
    e_two = og.normwise_error(host(C), truth, A, B)
    b.gemm_sgemm(M, N, K, 1.0, Ad, K, 0, Bd, N, 0, 0.0, C, N)
    e_fp32 = og.normwise_error(host(C), truth, A, B)
    assert e_x3 <= 2.0 * e_fp32, (e_x3, e_fp32)
    assert e_two > 10.0 * e_x3, (e_two, e_x3)


# ------------------------------------------------------------------ two-phase refinement (pieces, then GEMM)

_ONE_CALL = {0: "gemm_split", 1: "gemm_split_scaled", 2: "gemm_split_bf16x3"}


def _one_call(b, scheme, piece, nprod, m, n, k, alpha, A, la, B, lb, beta, C):
    lda = k if la == 0 else m
    ldb = n if lb == 0 else k
    if scheme == 2:
        b.gemm_split_bf16x3(m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, n)
    else:
        getattr(b, _ONE_CALL[scheme])(piece, nprod, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, n)


@pytest.mark.parametrize("scheme,piece,nprod", [(0, 0, 2), (0, 0, 3), (0, 1, 4), (1, 0, 3), (1, 1, 2), (2, 1, 6)])
@pytest.mark.parametrize("la,lb", [(0, 0), (1, 1)])
def test_prepare_then_run_is_the_one_call_bit_for_bit(b, scheme, piece, nprod, la, lb):
    m, n, k = 300, 264, 520
    A = _bits_matrix((m, k) if la == 0 else (k, m), seed=701, e_lo=-6, e_hi=6)
    B = _bits_matrix((k, n) if lb == 0 else (n, k), seed=711, e_lo=-6, e_hi=6)
    C0 = synth.uniform((m, n), seed=721)
    Ad, Bd = dev(A), dev(B)
    want = dev(C0)
    _one_call(b, scheme, piece, nprod, m, n, k, 1.25, Ad, la, Bd, lb, -0.5, want)
    need = b.gemm_split_workspace_bytes(piece, nprod, m, n, k)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    got = dev(C0)
    b.gemm_split_prepare(scheme, piece, nprod, m, n, k, Ad, k if la == 0 else m, la, Bd, n if lb == 0 else k, lb,
                         ws, need)
    b.gemm_split_run(scheme, piece, nprod, m, n, k, 1.25, -0.5, got, n, ws, need)
    b.tc_sync_status()
    assert torch.equal(got, want)


def test_pipelined_prepare_and_run_on_two_streams(b):
    # the pieces of product i+1 formed on a side stream while product i runs on the main stream,
    # with two workspaces and events between the streams: every result as the one-call GEMM's
    m, n, k = 512, 384, 640
    count = 4
    ins = [(dev(_bits_matrix((m, k), seed=800 + 2 * i, e_lo=-4, e_hi=4)),
            dev(_bits_matrix((k, n), seed=801 + 2 * i, e_lo=-4, e_hi=4))) for i in range(count)]
    want = []
    for A, B in ins:
        C = torch.zeros((m, n), dtype=torch.float32, device="cuda")
        b.gemm_split(0, 3, m, n, k, 1.0, A, k, 0, B, n, 0, 0.0, C, n)
        want.append(C)
    need = b.gemm_split_workspace_bytes(0, 3, m, n, k)
    ws = [torch.empty(need, dtype=torch.uint8, device="cuda") for _ in range(2)]
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    ready = [torch.cuda.Event() for _ in range(2)]
    free = [torch.cuda.Event() for _ in range(2)]
    got = [torch.zeros((m, n), dtype=torch.float32, device="cuda") for _ in range(count)]
    side.wait_stream(main)
    b.gemm_split_prepare(0, 0, 3, m, n, k, ins[0][0], k, 0, ins[0][1], n, 0, ws[0], need, stream=side)
    ready[0].record(side)
    for i in range(count):
        if i + 1 < count:
            j = (i + 1) % 2
            if i >= 1:
                side.wait_event(free[j])
            b.gemm_split_prepare(0, 0, 3, m, n, k, ins[i + 1][0], k, 0, ins[i + 1][1], n, 0, ws[j], need,
                                 stream=side)
            ready[j].record(side)
        main.wait_event(ready[i % 2])
        b.gemm_split_run(0, 0, 3, m, n, k, 1.0, 0.0, got[i], n, ws[i % 2], need, stream=main)
        free[i % 2].record(main)
    torch.cuda.synchronize()
    b.tc_sync_status()
    for i in range(count):
        assert torch.equal(got[i], want[i]), i


# ------------------------------------------------------------------ the paper's precision claims, on the GPU

def test_paper_precision_claims_hold_on_the_gpu_path(b, golden_dir):
    # Sec. VII-B: with e = C_x - C_single (C_single the FP32 CUDA-core GEMM), the refinement with R_A
    # alone removes about 30 % of max |e|, and R_A with R_B at least the paper's factors (10x for
    # uniform [-1, 1] inputs, 35x for [-16, 16]); the same bounds as the oracle's pins of these claims
    import json
    import os
    with open(os.path.join(golden_dir, "paper_numbers.json")) as f:
        paper = json.load(f)
    n = 1024
    for scale, key in ((1.0, "refinement_uniform_pm1_n8192"), (16.0, "refinement_uniform_pm16_n4096")):
        A = dev(synth.uniform((n, n), seed=synth.seed_for(0, 0)) * np.float32(scale))
        B = dev(synth.uniform((n, n), seed=synth.seed_for(0, 1)) * np.float32(scale))
        Cs = torch.empty((n, n), dtype=torch.float32, device="cuda")
        Cx = torch.empty_like(Cs)
        b.gemm_sgemm(n, n, n, 1.0, A, n, 0, B, n, 0, 0.0, Cs, n)
        Aq = torch.empty((n, n), dtype=torch.float16, device="cuda")
        Bq = torch.empty((n, n), dtype=torch.float16, device="cuda")
        b.tc_quantize(0, n, n, A, n, Aq, n, 0)
        b.tc_quantize(0, n, n, B, n, Bq, n, 1)
        b.gemm_mixed(0, n, n, n, 1.0, Aq, n, 0, Bq, n, 1, 0.0, Cx, n)
        e0 = b.tc_error_norm(n, n, Cx, n, Cs, n, 0)[3]
        b.gemm_split(0, 2, n, n, n, 1.0, A, n, 0, B, n, 0, 0.0, Cx, n)
        e2 = b.tc_error_norm(n, n, Cx, n, Cs, n, 0)[3]
        b.gemm_split(0, 4, n, n, n, 1.0, A, n, 0, B, n, 0, 0.0, Cx, n)
        e4 = b.tc_error_norm(n, n, Cx, n, Cs, n, 0)[3]
        b.tc_sync_status()
        ref = paper[key]
        if scale == 1.0:
            assert abs((1.0 - e2 / e0) - ref["emax_reduction_RA_only_fraction"]) < 0.12, (e0, e2)
            assert e0 > ref["emax_reduction_RA_RB_factor"] * e4, (e0, e4)
        else:
            assert e0 > ref["reduction_factor"] * e4, (e0, e4)
