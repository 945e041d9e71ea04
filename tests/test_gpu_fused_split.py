"""The one-launch refined GEMM: pieces formed on chip from FP32 tiles.

gemm_split and gemm_split_scaled called without a workspace read FP32 A and B
and form the pieces of Sec. V (hi = RN(x), lo = RN(x - hi); the scaled
residual) inside the GEMM kernel when both operands are 16-byte aligned with
leading dimensions that are multiples of 4.  TCGEMM_SPLIT=fused / =twopass
force the one-launch path or the two-pass path (a split pass into a
workspace, then the promoted tensor-core GEMM on the pieces); gemm_split_bf16x3
always takes two passes.  Both must give the same C bit for bit: the pieces
are the same roundings and the products are issued in the same order into the
same accumulators.  Each result is also checked against the oracle (Eq. 1 /
Eq. 2 on the same pieces, in FP64).
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


def _call(b, scheme, piece, nprod, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc):
    if scheme == 0:
        b.gemm_split(piece, nprod, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc)
    elif scheme == 1:
        b.gemm_split_scaled(piece, nprod, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc)
    else:
        b.gemm_split_bf16x3(m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc)


def _oracle(scheme, piece, nprod, A, B, alpha, beta, C0):
    if scheme == 0:
        return og.gemm_split(DT_NAME[piece], nprod, A, B, alpha, beta, C0)
    if scheme == 1:
        return og.gemm_split_scaled(DT_NAME[piece], nprod, A, B, alpha, beta, C0)
    return og.gemm_split_bf16x3(A, B, alpha, beta, C0)


def _stored(X, layout):
    return np.ascontiguousarray(X if layout == 0 else X.T)


SCHEMES = [(0, 0, 2), (0, 0, 3), (0, 0, 4), (0, 1, 2), (0, 1, 3), (0, 1, 4),
           (1, 0, 2), (1, 0, 3), (1, 1, 2), (1, 1, 3), (2, 1, 6)]


@pytest.mark.parametrize("scheme,piece,nprod", SCHEMES)
@pytest.mark.parametrize("la,lb", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_one_launch_matches_two_pass_bit_for_bit(b, monkeypatch, scheme, piece, nprod, la, lb):
    # ragged in every dimension: m and n cross a 256-tile edge and a CTA's 128-row half, k ends
    # inside a k-block of 64 and inside a group of four
    m, n, k = 300, 264, 203
    A = synth.log_uniform_pow2((m, k), seed=synth.seed_for(2, 10))
    B = synth.log_uniform_pow2((k, n), seed=synth.seed_for(2, 11))
    C0 = synth.uniform((m, n), seed=synth.seed_for(2, 12))
    lda = k if la == 0 else m
    ldb = n if lb == 0 else k
    # leading dimensions must be multiples of 4 for the one-launch path: pad where needed
    lda4, ldb4 = (lda + 3) // 4 * 4, (ldb + 3) // 4 * 4
    As, Bs = _stored(A, la), _stored(B, lb)
    Ap = np.zeros((As.shape[0], lda4), np.float32)
    Ap[:, :As.shape[1]] = As
    Bp = np.zeros((Bs.shape[0], ldb4), np.float32)
    Bp[:, :Bs.shape[1]] = Bs
    Ad, Bd = dev(Ap), dev(Bp)
    monkeypatch.setenv("TCGEMM_SPLIT", "fused")
    fused = dev(C0)
    _call(b, scheme, piece, nprod, m, n, k, 1.25, Ad, lda4, la, Bd, ldb4, lb, -0.5, fused, n)
    monkeypatch.setenv("TCGEMM_SPLIT", "twopass")
    twopass = dev(C0)
    _call(b, scheme, piece, nprod, m, n, k, 1.25, Ad, lda4, la, Bd, ldb4, lb, -0.5, twopass, n)
    b.tc_sync_status()
    got = host(fused)
    assert torch.equal(fused, twopass), np.abs(got - host(twopass)).max()
    ref = _oracle(scheme, piece, nprod, A, B, 1.25, -0.5, C0)
    assert normwise_dev(got, ref, A, B, 1.25, -0.5, C0) <= TOL_NORMWISE


@pytest.mark.parametrize("scheme,nprod", [(0, 3), (1, 2)])
def test_one_launch_matches_two_pass_over_several_rounds_of_tiles(b, monkeypatch, scheme, nprod):
    # 11 x 10 tiles of 256 x 256: more tiles than CTA pairs, so pairs take a second round of tiles,
    # which walks K downwards (ragged K: the last k-block comes first there)
    m, n, k = 2816, 2560, 1000
    A = dev(synth.log_uniform_pow2((m, k), seed=191))
    B = dev(synth.log_uniform_pow2((k, n), seed=192))
    out = {}
    for path in ("fused", "twopass"):
        monkeypatch.setenv("TCGEMM_SPLIT", path)
        C = torch.zeros((m, n), dtype=torch.float32, device="cuda")
        _call(b, scheme, 0, nprod, m, n, k, 1.0, A, k, 0, B, n, 0, 0.0, C, n)
        out[path] = C
    b.tc_sync_status()
    assert torch.equal(out["fused"], out["twopass"])


@pytest.mark.parametrize("mnk", [(1, 1, 1), (100, 72, 40), (128, 256, 64), (257, 513, 129), (640, 384, 1030)])
def test_one_launch_shapes_against_the_oracle(b, monkeypatch, mnk):
    monkeypatch.setenv("TCGEMM_SPLIT", "fused")
    # single elements, m within one CTA's rows, exact tiles, one past the tile edges, many k-blocks
    m, n, k = mnk
    A = synth.log_uniform_pow2((m, k), seed=synth.seed_for(2, 20))
    B = synth.log_uniform_pow2((k, n), seed=synth.seed_for(2, 21))
    C0 = synth.uniform((m, n), seed=synth.seed_for(2, 22))
    ld4 = lambda v: (v + 3) // 4 * 4
    Ap = np.zeros((m, ld4(k)), np.float32)
    Ap[:, :k] = A
    Bp = np.zeros((k, ld4(n)), np.float32)
    Bp[:, :n] = B
    Ad, Bd = dev(Ap), dev(Bp)
    for scheme, piece, nprod in [(0, 0, 3), (1, 0, 3), (2, 1, 6)]:
        C = dev(C0)
        _call(b, scheme, piece, nprod, m, n, k, 1.0, Ad, ld4(k), 0, Bd, ld4(n), 0, 0.5, C, n)
        b.tc_sync_status()
        got = host(C)
        ref = _oracle(scheme, piece, nprod, A, B, 1.0, 0.5, C0)
        if scheme == 0:
            Ah, Al = nm.split(A, "f16")
            Bh, Bl = nm.split(B, "f16")
            mag = (np.abs(Ah) + np.abs(Al)) @ (np.abs(Bh) + np.abs(Bl)) + 0.5 * np.abs(C0.astype(np.float64))
            ok, info = elementwise_ok(got, ref, mag, nprod * k)
            assert ok, (scheme, info)
        assert normwise_dev(got, ref, A, B, 1.0, 0.5, C0) <= TOL_NORMWISE, scheme


@pytest.mark.parametrize("la,lb", [(0, 0), (1, 1)])
def test_one_launch_reads_nothing_past_the_matrix(b, monkeypatch, la, lb):
    monkeypatch.setenv("TCGEMM_SPLIT", "fused")
    # NaN in the padding of every row (leading dimensions multiples of 4, larger than the rows),
    # k and m not multiples of 4: a read past the matrix would put NaN into C
    m, n, k = 259, 140, 201
    A = synth.log_uniform_pow2((m, k), seed=161)
    B = synth.log_uniform_pow2((k, n), seed=162)
    As, Bs = _stored(A, la), _stored(B, lb)
    lda = (As.shape[1] + 3) // 4 * 4 + 4
    ldb = (Bs.shape[1] + 3) // 4 * 4 + 4
    Ap = np.full((As.shape[0], lda), np.nan, np.float32)
    Ap[:, :As.shape[1]] = As
    Bp = np.full((Bs.shape[0], ldb), np.nan, np.float32)
    Bp[:, :Bs.shape[1]] = Bs
    ldc = n + 5
    C = torch.full((m, ldc), float("nan"), dtype=torch.float32, device="cuda")
    b.gemm_split(0, 3, m, n, k, 1.0, dev(Ap), lda, la, dev(Bp), ldb, lb, 0.0, C, ldc)
    b.tc_sync_status()
    got = host(C)
    assert np.all(np.isnan(got[:, n:]))
    assert np.all(np.isfinite(got[:, :n]))
    ref = og.gemm_split("f16", 3, A, B)
    assert normwise_dev(got[:, :n], ref, A, B) <= TOL_NORMWISE


def test_one_launch_is_deterministic(b, monkeypatch):
    monkeypatch.setenv("TCGEMM_SPLIT", "fused")
    m, n, k = 512, 768, 1024
    A = dev(synth.log_uniform_pow2((m, k), seed=171))
    B = dev(synth.log_uniform_pow2((k, n), seed=172))
    outs = []
    for _ in range(2):
        C = torch.zeros((m, n), dtype=torch.float32, device="cuda")
        b.gemm_split(0, 3, m, n, k, 1.0, A, k, 0, B, n, 0, 0.0, C, n)
        outs.append(C)
    b.tc_sync_status()
    assert torch.equal(outs[0], outs[1])


def test_without_a_workspace_the_call_matches_the_call_with_one(b, monkeypatch):
    # no TCGEMM_SPLIT: a call without workspace runs the one-launch kernel, a call with one the two
    # passes (the launch lists under profiles/ show which kernels each runs); they agree bit for bit
    monkeypatch.delenv("TCGEMM_SPLIT", raising=False)
    m, n, k = 384, 512, 640
    A = dev(synth.log_uniform_pow2((m, k), seed=181))
    B = dev(synth.log_uniform_pow2((k, n), seed=182))
    ws_bytes = b.gemm_split_workspace_bytes(0, 3, m, n, k)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    c1 = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    c2 = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    b.gemm_split(0, 3, m, n, k, 1.0, A, k, 0, B, n, 0, 0.0, c1, n)
    b.gemm_split(0, 3, m, n, k, 1.0, A, k, 0, B, n, 0, 0.0, c2, n, ws, ws_bytes)
    b.tc_sync_status()
    assert torch.equal(c1, c2)
