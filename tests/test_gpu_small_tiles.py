"""Narrow single-CTA tiles and launches that overlap the kernel before them.

gemm_mixed runs problems that 128 x 64 (else 128 x 128) tiles spread over no
more SMs than the device has on single CTAs with those tiles; TCGEMM_TILE and
TCGEMM_BN force any width.  Each width is checked element by element against
the oracle (Sec. IV: C = alpha*A*B + beta*C on the rounded inputs, FP32
accumulation) on ragged shapes.

The GEMM kernels are launched with programmatic stream serialization: their
set-up may overlap the kernel before them in the stream, and they wait for it
before touching any operand.  A chain of kernels that each read what the one
before wrote must therefore give the same bits as the same chain with the host
synchronising between launches, eagerly and replayed from a CUDA graph.
"""
import numpy as np
import pytest

import synth
from oracle import gemm as og
from oracle import numerics as nm
from tests.gpu_common import TOL_NORMWISE, dev, elementwise_ok, host, need_gpu, normwise_dev, torch

pytestmark = pytest.mark.gpu

DT_NAME = {0: "f16", 1: "bf16", 2: "e4m3"}
TDT = {0: torch.float16, 1: torch.bfloat16, 2: torch.uint8}


@pytest.fixture(scope="module")
def b():
    need_gpu()
    from paper_1803_04014_gb300 import binding
    binding.load()
    return binding


def _rounded(b, dt, A, B):
    m, k = A.shape
    n = B.shape[1]
    aq = torch.empty((m, k), dtype=TDT[dt], device="cuda")
    bq = torch.empty((n, k), dtype=TDT[dt], device="cuda")
    sc = torch.empty(2, dtype=torch.float32, device="cuda")
    b.tc_quantize(dt, m, k, dev(A), k, aq, k, 0, sc[0:1])
    b.tc_quantize(dt, k, n, dev(B), n, bq, k, 1, sc[1:2])
    return aq, bq, sc


def _mag(dt, A, B, alpha, beta, C0):
    Aq, sa = nm.quantize(A, DT_NAME[dt])
    Bq, sb = nm.quantize(B, DT_NAME[dt])
    return abs(alpha) * (np.abs(Aq) @ np.abs(Bq)) / (sa * sb) + abs(beta) * np.abs(C0.astype(np.float64))


@pytest.mark.parametrize("bn", ["64", "128", "256"])
@pytest.mark.parametrize("dt", [0, 1, 2])
@pytest.mark.parametrize("mnk", [(300, 200, 160), (129, 1000, 96), (1, 65, 32), (640, 384, 1024)])
def test_single_cta_tile_widths(b, monkeypatch, bn, dt, mnk):
    # ragged m and n (one row past a 128-row tile, n ending inside a 64-, 128- or 256-wide tile),
    # several k-blocks and a deep ring
    monkeypatch.setenv("TCGEMM_TILE", "single")
    monkeypatch.setenv("TCGEMM_BN", bn)
    m, n, k = mnk
    A = synth.uniform((m, k), seed=201)
    B = synth.uniform((k, n), seed=202)
    C0 = synth.uniform((m, n), seed=203)
    aq, bq, sc = _rounded(b, dt, A, B)
    C = dev(C0)
    b.gemm_mixed(dt, m, n, k, 1.25, aq, k, 0, bq, k, 1, -0.5, C, n,
                 sc[0:1] if dt == 2 else None, sc[1:2] if dt == 2 else None)
    b.tc_sync_status()
    got = host(C)
    ref = og.gemm_mixed(DT_NAME[dt], A, B, 1.25, -0.5, C0)
    ok, info = elementwise_ok(got, ref, _mag(dt, A, B, 1.25, -0.5, C0), k)
    assert ok, info
    assert normwise_dev(got, ref, A, B, 1.25, -0.5, C0) <= TOL_NORMWISE


@pytest.mark.parametrize("dt", [0, 2])
@pytest.mark.parametrize("mn", [(256, 256), (1024, 1024), (1536, 1400), (128, 4096)])
def test_untuned_narrow_tiles_against_the_oracle(b, monkeypatch, dt, mn):
    # the untuned choice at these sizes: 128 x 64 tiles (8 and 128 of them), 128 x 128 (132), and
    # 128 x 64 for a 128-row problem (64 tiles)
    for var in ("TCGEMM_TILE", "TCGEMM_BN"):
        monkeypatch.delenv(var, raising=False)
    m, n = mn
    k = 192
    A = synth.uniform((m, k), seed=211)
    B = synth.uniform((k, n), seed=212)
    C0 = synth.uniform((m, n), seed=213)
    aq, bq, sc = _rounded(b, dt, A, B)
    C = dev(C0)
    b.gemm_mixed(dt, m, n, k, 1.0, aq, k, 0, bq, k, 1, 0.5, C, n,
                 sc[0:1] if dt == 2 else None, sc[1:2] if dt == 2 else None)
    b.tc_sync_status()
    got = host(C)
    ref = og.gemm_mixed(DT_NAME[dt], A, B, 1.0, 0.5, C0)
    ok, info = elementwise_ok(got, ref, _mag(dt, A, B, 1.0, 0.5, C0), k)
    assert ok, info


def _chain(b, X, Aq, Bq, C, m, n, k, steps, sync):
    # each step: torch scales X by 1.5, tc_quantize rounds it into Aq, gemm_mixed adds Aq B to C (beta = 1);
    # every kernel reads what the kernel before it wrote
    for _ in range(steps):
        X.mul_(1.5)
        b.tc_quantize(0, m, k, X, k, Aq, k, 0)
        if sync:
            torch.cuda.synchronize()
        b.gemm_mixed(0, m, n, k, 1.0, Aq, k, 0, Bq, k, 1, 1.0, C, n)
        if sync:
            torch.cuda.synchronize()


@pytest.mark.parametrize("mnk", [(256, 256, 256), (2048, 2048, 512)])
def test_overlapped_launches_give_the_synchronised_result(b, mnk):
    m, n, k = mnk
    X0 = dev(synth.uniform((m, k), seed=221) * np.float32(1e-3))
    B = synth.uniform((k, n), seed=222)
    Bq = torch.empty((n, k), dtype=torch.float16, device="cuda")
    b.tc_quantize(0, k, n, dev(B), n, Bq, k, 1)
    Aq = torch.empty((m, k), dtype=torch.float16, device="cuda")
    C0 = dev(synth.uniform((m, n), seed=223))
    out = {}
    for sync in (True, False):
        X, C = X0.clone(), C0.clone()
        torch.cuda.synchronize()
        _chain(b, X, Aq, Bq, C, m, n, k, 12, sync)
        torch.cuda.synchronize()
        out[sync] = C
    b.tc_sync_status()
    assert torch.equal(out[True], out[False])
    # the same chain replayed from a CUDA graph (one synchronised step first: per-kernel set-up
    # happens outside the capture)
    X, C = X0.clone(), C0.clone()
    _chain(b, X.clone(), Aq, Bq, C.clone(), m, n, k, 1, True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            _chain(b, X, Aq, Bq, C, m, n, k, 12, False)
    torch.cuda.current_stream().wait_stream(s)
    X.copy_(X0)
    C.copy_(C0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    b.tc_sync_status()
    assert torch.equal(C, out[True])
