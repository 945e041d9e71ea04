"""Serving queue (serve_open / serve_submit / serve_poll): continuous batching on one GPU.

Each request's result is checked against the oracle for its mode, and is
bitwise the same when the request runs alone and when it runs in a mix of
other requests that overlap it on the GPU.  Admission by the HBM budget, the
queue bound, and ticket handling are checked too.
"""
import time

import numpy as np
import pytest

import synth
from oracle import gemm as og
from tests.gpu_common import TOL_NORMWISE, dev, host, need_gpu, normwise_dev, torch

pytestmark = pytest.mark.gpu

MODE_NAMES = {0: "f16", 1: "bf16", 2: "e4m3", 3: "split3"}


@pytest.fixture(scope="module")
def b():
    need_gpu()
    from paper_1803_04014_gb300 import binding
    binding.load()
    return binding


def _oracle(mode, A, B, alpha, beta, C0):
    if mode == 3:
        return og.gemm_split("f16", 3, A, B, alpha, beta, C0)
    return og.gemm_mixed(MODE_NAMES[mode], A, B, alpha, beta, C0)


def _wait(b, srv, ticket, timeout_s=60.0):
    t0 = time.time()
    while True:
        r = b.serve_poll(srv, ticket)
        if r is not None:
            return r
        if time.time() - t0 > timeout_s:
            raise TimeoutError("request did not finish")
        time.sleep(0.0005)


def _requests(count, seed, lo=32, hi=700):
    _, sizes, modes = synth.serve_stream(count, seed=seed, rate_per_s=1.0, lo=lo, hi=hi)
    out = []
    for i in range(count):
        m, n, k = (int(x) for x in sizes[i])
        A = synth.uniform((m, k), seed=seed * 1000 + 3 * i)
        B = synth.uniform((k, n), seed=seed * 1000 + 3 * i + 1)
        C0 = synth.uniform((m, n), seed=seed * 1000 + 3 * i + 2)
        out.append((int(modes[i]), A, B, C0))
    return out


def test_each_mode_matches_oracle(b):
    srv = b.serve_open(1 << 30, max_inflight=8, num_streams=4)
    try:
        for mode in range(4):
            m, n, k = 200, 136, 264
            A = synth.uniform((m, k), seed=10 + mode)
            B = synth.uniform((k, n), seed=20 + mode)
            C0 = synth.uniform((m, n), seed=30 + mode)
            Ad, Bd, Cd = dev(A), dev(B), dev(C0)
            t = b.serve_submit(srv, mode, m, n, k, Ad, k, Bd, n, Cd, n, 0.5, 2.0)
            r = _wait(b, srv, t)
            assert r["status"] == 0
            assert r["t_submit_us"] <= r["t_start_us"] <= r["t_done_us"]
            ref = _oracle(mode, A, B, 0.5, 2.0, C0)
            assert normwise_dev(host(Cd), ref, A, B, 0.5, 2.0, C0) <= TOL_NORMWISE
    finally:
        b.serve_close(srv)


def test_result_is_the_same_alone_and_in_a_mix(b):
    reqs = _requests(40, seed=5)
    target = 17
    srv = b.serve_open(1 << 30, max_inflight=12, num_streams=4)
    try:
        mode, A, B, C0 = reqs[target]
        m, k = A.shape
        n = B.shape[1]
        # alone
        Ad, Bd, Cd = dev(A), dev(B), dev(C0)
        _wait(b, srv, b.serve_submit(srv, mode, m, n, k, Ad, k, Bd, n, Cd, n, 1.0, 0.5))
        alone = host(Cd)
        # in a mix: every request submitted back to back, the target in the middle
        bufs, tickets = [], []
        for (md, Ai, Bi, Ci) in reqs:
            mi, ki = Ai.shape
            ni = Bi.shape[1]
            a_, b_, c_ = dev(Ai), dev(Bi), dev(Ci)
            bufs.append(c_)
            tickets.append(b.serve_submit(srv, md, mi, ni, ki, a_, ki, b_, ni, c_, ni, 1.0, 0.5))
            bufs.append((a_, b_))
        results = [_wait(b, srv, t) for t in tickets]
        assert all(r["status"] == 0 for r in results)
        mixed = host(bufs[2 * target])
        assert np.array_equal(alone, mixed)
        # and every request of the mix matches the oracle
        for i, (md, Ai, Bi, Ci) in enumerate(reqs):
            got = host(bufs[2 * i])
            ref = _oracle(md, Ai, Bi, 1.0, 0.5, Ci)
            assert normwise_dev(got, ref, Ai, Bi, 1.0, 0.5, Ci) <= TOL_NORMWISE, (i, md)
        st = b.serve_stats(srv)
        assert st["completed"] == st["submitted"] == 41
        assert st["peak_inflight"] >= 2   # requests overlapped on the GPU
    finally:
        b.serve_close(srv)


def test_admission_waits_for_budget(b):
    # a budget that holds one request's workspace at a time
    m = n = k = 512
    one = (m * k + n * k) * 2                   # FP16 copies of A and B: 1 MiB
    need = one + one // 2                       # room for one request at a time
    srv = b.serve_open(need, max_inflight=8, num_streams=4)
    try:
        A = synth.uniform((m, k), seed=41)
        B = synth.uniform((k, n), seed=42)
        Ad, Bd = dev(A), dev(B)
        outs = [torch.empty((m, n), dtype=torch.float32, device="cuda") for _ in range(6)]
        tickets = [b.serve_submit(srv, 0, m, n, k, Ad, k, Bd, n, c, n, 1.0, 0.0) for c in outs]
        res = [_wait(b, srv, t) for t in tickets]
        assert all(r["status"] == 0 for r in res)
        st = b.serve_stats(srv)
        assert st["peak_inflight"] == 1
        assert st["peak_bytes"] <= need
        ref = og.gemm_mixed("f16", A, B)
        for c in outs:
            assert normwise_dev(host(c), ref, A, B) <= TOL_NORMWISE
    finally:
        b.serve_close(srv)


def test_oversize_request_is_rejected(b):
    srv = b.serve_open(1 << 20, max_inflight=4, num_streams=2)
    try:
        a = torch.zeros(2048 * 2048, dtype=torch.float32, device="cuda")
        with pytest.raises(b.TcError) as e:
            b.serve_submit(srv, 3, 2048, 2048, 2048, a, 2048, a, 2048, a, 2048)
        assert e.value.status == b.TC_ERR_INVALID
        with pytest.raises(b.TcError):
            b.serve_submit(srv, 7, 16, 16, 16, a, 16, a, 16, a, 16)       # unknown mode
        with pytest.raises(b.TcError):
            b.serve_poll(srv, 12345)                                      # unknown ticket
    finally:
        b.serve_close(srv)


def test_full_queue_reports_busy_and_tickets_are_forgotten_after_poll(b):
    N = 8192
    A = torch.empty((N, N), dtype=torch.float32, device="cuda").uniform_(-1, 1)
    C = torch.empty((N, N), dtype=torch.float32, device="cuda")
    small = torch.empty((64, 64), dtype=torch.float32, device="cuda")
    srv = b.serve_open(4 << 30, max_inflight=1, num_streams=1, queue_capacity=2)
    try:
        first = b.serve_submit(srv, 3, N, N, N, A, N, A, N, C, N)   # a long request occupies the slot
        tickets, busy = [], 0
        for _ in range(6):
            t = b.serve_submit(srv, 0, 64, 64, 64, small, 64, small, 64, small, 64)
            if t is None:
                busy += 1
            else:
                tickets.append(t)
        assert busy >= 1
        for t in [first] + tickets:
            assert _wait(b, srv, t)["status"] == 0
        with pytest.raises(b.TcError):
            b.serve_poll(srv, first)          # already reported, forgotten
    finally:
        b.serve_close(srv)


def test_scheduler_timing_counters(b):
    # serve_timing reports where the scheduler thread spent its time; after a drained stream every
    # request is counted as completed and each phase took some time
    reqs = _requests(24, seed=synth.seed_for(4, 30))
    srv = b.serve_open(1 << 30, max_inflight=8, num_streams=4)
    keep = []
    try:
        tickets = []
        for (mode, A, B, C0) in reqs:
            (m, k), n = A.shape, B.shape[1]
            Ad, Bd, Cd = dev(A), dev(B), dev(C0)
            keep.append((Ad, Bd, Cd))
            t = None
            while t is None:
                t = b.serve_submit(srv, mode, m, n, k, Ad, k, Bd, n, Cd, n)
            tickets.append(t)
        b.serve_drain(srv, 60_000)
        for t in tickets:
            assert _wait(b, srv, t)["status"] == b.TC_OK
        tm = b.serve_timing(srv)
    finally:
        b.serve_close(srv)
    assert tm["completed"] == len(reqs)
    assert tm["launch_ns"] > 0 and tm["admit_ns"] > 0 and tm["retire_ns"] > 0
    assert 1 <= tm["launch_groups"] <= len(reqs)
