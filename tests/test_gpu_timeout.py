"""Failure detection without a fault: a GEMM whose barrier is never completed.

tc_debug_stall_next_gemm makes the next tensor-core GEMM withhold one
k-block, so the MMA issuer waits on an mbarrier that nothing completes.  The
bounded wait must give up (2 s), record TC_ERR_TIMEOUT for tc_sync_status,
release TMEM and return; the context must stay usable for the next GEMM.
"""
import numpy as np
import pytest

import synth
from oracle import gemm as og
from tests.gpu_common import TOL_NORMWISE, dev, host, need_gpu, normwise_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    need_gpu()
    from paper_1803_04014_gb300 import binding
    binding.load()
    return binding


def _operands(b, m, n, k, seed):
    A = synth.uniform((m, k), seed=seed)
    B = synth.uniform((k, n), seed=seed + 1)
    Aq = torch.empty((m, k), dtype=torch.float16, device="cuda")
    Bq = torch.empty((n, k), dtype=torch.float16, device="cuda")
    b.tc_quantize(0, m, k, dev(A), k, Aq, k, 0)
    b.tc_quantize(0, k, n, dev(B), n, Bq, k, 1)
    return A, B, Aq, Bq


@pytest.mark.parametrize("tile,mnk", [("single", (128, 256, 512)), ("pair", (512, 512, 512)),
                                      ("quad", (512, 1024, 512))])
def test_stalled_gemm_times_out_and_the_context_survives(b, monkeypatch, tile, mnk):
    # "quad": clusters of four CTAs (two pairs sharing A by multicast)
    monkeypatch.setenv("TCGEMM_TILE", "pair" if tile == "quad" else tile)
    monkeypatch.setenv("TCGEMM_CLUSTER", "4" if tile == "quad" else "2")
    m, n, k = mnk
    A, B, Aq, Bq = _operands(b, m, n, k, seed=5)
    b.tc_sync_status()
    C = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    b.tc_debug_stall_next_gemm(2)
    b.gemm_mixed(0, m, n, k, 1.0, Aq, k, 0, Bq, k, 1, 0.0, C, n)
    with pytest.raises(b.TcError) as e:
        b.tc_sync_status()
    assert e.value.status == b.TC_ERR_TIMEOUT
    # the status was cleared and the next GEMM is correct
    b.gemm_mixed(0, m, n, k, 1.0, Aq, k, 0, Bq, k, 1, 0.0, C, n)
    b.tc_sync_status()
    ref = og.gemm_mixed("f16", A, B)
    assert normwise_dev(host(C), ref, A, B) <= TOL_NORMWISE


@pytest.mark.parametrize("scheme,path", [("eq2", "fused"), ("eq2", "twopass"), ("scaled", "fused"),
                                         ("scaled", "twopass"), ("bf16x3", "twopass")])
def test_stalled_refined_gemm_times_out_and_the_context_survives(b, monkeypatch, scheme, path):
    # "fused": the one-launch kernel (a piece warp of the first CTA pair withholds its arrival);
    # "twopass": the promoted GEMM on pieces from a split pass (the producer withholds a k-block)
    monkeypatch.setenv("TCGEMM_SPLIT", path)
    m, n, k = 512, 256, 640
    A = synth.log_uniform_pow2((m, k), seed=9)
    B = synth.log_uniform_pow2((k, n), seed=10)
    Ad, Bd = dev(A), dev(B)
    C = torch.zeros((m, n), dtype=torch.float32, device="cuda")

    def run():
        if scheme == "eq2":
            b.gemm_split(0, 3, m, n, k, 1.0, Ad, k, 0, Bd, n, 0, 0.0, C, n)
        elif scheme == "scaled":
            b.gemm_split_scaled(0, 3, m, n, k, 1.0, Ad, k, 0, Bd, n, 0, 0.0, C, n)
        else:
            b.gemm_split_bf16x3(m, n, k, 1.0, Ad, k, 0, Bd, n, 0, 0.0, C, n)

    b.tc_debug_stall_next_gemm(3)
    run()
    with pytest.raises(b.TcError) as e:
        b.tc_sync_status()
    assert e.value.status == b.TC_ERR_TIMEOUT
    run()
    b.tc_sync_status()
    ref = {"eq2": lambda: og.gemm_split("f16", 3, A, B),
           "scaled": lambda: og.gemm_split_scaled("f16", 3, A, B),
           "bf16x3": lambda: og.gemm_split_bf16x3(A, B)}[scheme]()
    assert normwise_dev(host(C), ref, A, B) <= TOL_NORMWISE


def test_a_cleared_request_does_not_stall(b):
    m = n = k = 256
    A, B, Aq, Bq = _operands(b, m, n, k, seed=11)
    C = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    b.tc_debug_stall_next_gemm(1)
    b.tc_debug_stall_next_gemm(-1)
    b.gemm_mixed(0, m, n, k, 1.0, Aq, k, 0, Bq, k, 1, 0.0, C, n)
    b.tc_sync_status()
    assert np.all(np.isfinite(host(C)))
