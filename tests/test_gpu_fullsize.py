"""Parity at the full sizes of the measured configurations, on sampled outputs.

Every configuration runs at its real size through the C ABI, in the launch
configuration the benchmark uses; the oracle then computes sampled rows and
columns of the result (FP64 dot products of the rounded inputs), or whole
sampled problems of a group or batch:

* the square sweep, N = 1024 ... 16384, FP16 / BF16 / E4M3, uniform and normal
  inputs, beta = 0.5 with C0 (tc_quantize + gemm_mixed);
* the refinement at N = 4096 and 8192 (Eq. 2 with 3 and 4 products, FP16 and
  BF16 pieces; the scaled split; three BF16 pieces), with the error against
  FP64 next to the FP32 CUDA-core GEMM's on the same samples;
* the 10 000-problem grouped GEMM (plan with CUDA-graph replay) and the
  10^6-problem 16^3 batch;
* a served stream of requests drawn like the benchmark's.
"""
import numpy as np
import pytest

import synth
from oracle import gemm as og
from oracle import numerics as nm
from tests.gpu_common import dev, elementwise_ok, host, need_gpu, torch

pytestmark = pytest.mark.gpu

DT_NAME = {0: "f16", 1: "bf16", 2: "e4m3"}


@pytest.fixture(scope="module")
def b():
    need_gpu()
    from paper_1803_04014_gb300 import binding
    binding.load()
    return binding


def _samples(N, count, mul, add):
    idx = (np.arange(count, dtype=np.int64) * mul + add) % N
    return np.unique(np.concatenate([idx, [0, N - 1]]))


def _sampled_normwise(got, ref, A_rows, B_cols):
    d = np.asarray(got, np.float64) - np.asarray(ref, np.float64)
    den = np.linalg.norm(np.asarray(A_rows, np.float64)) * np.linalg.norm(np.asarray(B_cols, np.float64))
    return float(np.linalg.norm(d) / den)


# ------------------------------------------------------------------ square sweep

@pytest.mark.parametrize("dist", ["uniform", "normal"])
@pytest.mark.parametrize("N", [1024, 2048, 4096, 8192, 16384])
def test_square_sweep_sampled(b, N, dist):
    gen = synth.uniform if dist == "uniform" else synth.normal
    off = 0 if dist == "uniform" else 3
    A = gen((N, N), seed=synth.seed_for(1, off + 0))
    B = gen((N, N), seed=synth.seed_for(1, off + 1))
    C0 = synth.uniform((N, N), seed=synth.seed_for(1, 2))
    rows = _samples(N, 16, 1237, 5)
    cols = _samples(N, 48, 3319, 11)
    Ad, Bd = dev(A), dev(B)
    C = torch.empty((N, N), dtype=torch.float32, device="cuda")
    C0d = dev(C0)
    # FP64 copies made once: the oracle's calls below take them without converting again
    A, B, C0 = A.astype(np.float64), B.astype(np.float64), C0.astype(np.float64)
    errs = {}
    for dt in (0, 1, 2):
        tdt = {0: torch.float16, 1: torch.bfloat16, 2: torch.uint8}[dt]
        Aq = torch.empty((N, N), dtype=tdt, device="cuda")
        Bq = torch.empty((N, N), dtype=tdt, device="cuda")
        sc = torch.empty(2, dtype=torch.float32, device="cuda")
        b.tc_quantize(dt, N, N, Ad, N, Aq, N, 0, sc[0:1])
        b.tc_quantize(dt, N, N, Bd, N, Bq, N, 1, sc[1:2])
        C.copy_(C0d)
        b.gemm_mixed(dt, N, N, N, 1.0, Aq, N, 0, Bq, N, 1, 0.5, C, N,
                     sc[0:1] if dt == 2 else None, sc[1:2] if dt == 2 else None)
        b.tc_sync_status()
        got = host(C[torch.from_numpy(rows).cuda()][:, torch.from_numpy(cols).cuda()])
        ref = og.gemm_mixed(DT_NAME[dt], A, B, 1.0, 0.5, C0, rows=rows, cols=cols)
        # elementwise FP32-accumulation bound on the sample
        amax_a = nm.absmax(A) if dt == 2 else None
        amax_b = nm.absmax(B) if dt == 2 else None
        Aq_s, sa = nm.quantize(A[rows], DT_NAME[dt], amax_a)
        Bq_s, sb = nm.quantize(B[:, cols], DT_NAME[dt], amax_b)
        mag = (np.abs(Aq_s) @ np.abs(Bq_s)) / (sa * sb) + 0.5 * np.abs(C0[rows][:, cols])
        ok, info = elementwise_ok(got, ref, mag, N)
        assert ok, (DT_NAME[dt], info)
        assert _sampled_normwise(got, ref, A[rows], B[:, cols]) <= 1e-5
        truth = og.gemm_truth(A, B, 1.0, 0.5, C0, rows=rows, cols=cols)
        errs[dt] = _sampled_normwise(got, truth, A[rows], B[:, cols])
        del Aq, Bq
    # error against FP64 grows as the format narrows
    assert errs[0] < errs[1] < errs[2], errs
    assert errs[0] < 1e-4 and errs[2] < 1e-2, errs


# ------------------------------------------------------------------ refinement

@pytest.mark.parametrize("N", [4096, 8192])
def test_refinement_sampled(b, N):
    A = synth.log_uniform_pow2((N, N), seed=synth.seed_for(2, 0))
    B = synth.log_uniform_pow2((N, N), seed=synth.seed_for(2, 1))
    rows = _samples(N, 12, 1531, 7)
    cols = _samples(N, 40, 2713, 3)
    rows_d, cols_d = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
    Ad, Bd = dev(A), dev(B)
    A, B = A.astype(np.float64), B.astype(np.float64)
    C = torch.empty((N, N), dtype=torch.float32, device="cuda")
    wsb = b.gemm_split_workspace_bytes(1, 6, N, N, N)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    truth = og.gemm_truth(A, B, rows=rows, cols=cols)
    A_r, B_c = A[rows], B[:, cols]

    def sample():
        b.tc_sync_status()
        return host(C[rows_d][:, cols_d])

    b.gemm_sgemm(N, N, N, 1.0, Ad, N, 0, Bd, N, 0, 0.0, C, N)
    e_fp32 = _sampled_normwise(sample(), truth, A_r, B_c)
    for piece in (0, 1):
        Ah, Al = nm.split(A_r, DT_NAME[piece])
        Bh, Bl = nm.split(B_c, DT_NAME[piece])
        mag = (np.abs(Ah) + np.abs(Al)) @ (np.abs(Bh) + np.abs(Bl))
        for nprod in (3, 4):
            b.gemm_split(piece, nprod, N, N, N, 1.0, Ad, N, 0, Bd, N, 0, 0.0, C, N, ws, wsb)
            got = sample()
            ref = og.gemm_split(DT_NAME[piece], nprod, A, B, rows=rows, cols=cols)
            ok, info = elementwise_ok(got, ref, mag, nprod * N)
            assert ok, (piece, nprod, info)
            if piece == 0:
                # the accuracy bar: within 2x of the FP32 CUDA-core GEMM's error
                assert _sampled_normwise(got, truth, A_r, B_c) <= 2.0 * e_fp32
            # the one-launch path (no workspace: pieces formed on chip) gives the same C bit for bit
            two_pass = C.clone()
            b.gemm_split(piece, nprod, N, N, N, 1.0, Ad, N, 0, Bd, N, 0, 0.0, C, N)
            b.tc_sync_status()
            assert torch.equal(C, two_pass), (piece, nprod)
    b.gemm_split_scaled(0, 3, N, N, N, 1.0, Ad, N, 0, Bd, N, 0, 0.0, C, N, ws, wsb)
    got = sample()
    two_pass = C.clone()
    b.gemm_split_scaled(0, 3, N, N, N, 1.0, Ad, N, 0, Bd, N, 0, 0.0, C, N)
    b.tc_sync_status()
    assert torch.equal(C, two_pass)
    ref = og.gemm_split_scaled("f16", 3, A, B, rows=rows, cols=cols)
    ok, info = elementwise_ok(got, ref, np.abs(A_r) @ np.abs(B_c), 3 * N)
    assert ok, info
    assert _sampled_normwise(got, truth, A_r, B_c) <= 2.0 * e_fp32
    b.gemm_split_bf16x3(N, N, N, 1.0, Ad, N, 0, Bd, N, 0, 0.0, C, N, ws, wsb)
    got = sample()
    ref = og.gemm_split_bf16x3(A, B, rows=rows, cols=cols)
    ok, info = elementwise_ok(got, ref, np.abs(A_r) @ np.abs(B_c), 6 * N)
    assert ok, info
    assert _sampled_normwise(got, truth, A_r, B_c) <= 2.0 * e_fp32


# ------------------------------------------------------------------ grouped and batched

def test_grouped_10000_sampled_problems(b):
    sizes = synth.group_sizes(10000, seed=synth.seed_for(3, 0))
    offa = np.zeros(len(sizes), np.int64)
    offb = np.zeros(len(sizes), np.int64)
    offc = np.zeros(len(sizes), np.int64)
    a = bb = c = 0
    for g, (m, n, k) in enumerate(sizes):
        offa[g], offb[g], offc[g] = a, bb, c
        a += m * k
        bb += n * k
        c += m * n
    # FP16 operands: the uniform draws converted to FP16 once (input preparation; the oracle's
    # rounding of an FP16 value is the identity)
    A16 = synth.uniform((a,), seed=synth.seed_for(3, 1)).astype(np.float16)
    B16 = synth.uniform((bb,), seed=synth.seed_for(3, 2)).astype(np.float16)
    C0 = synth.uniform((c,), seed=synth.seed_for(3, 3))
    desc = [(m, n, k, offa[g], offb[g], offc[g], k, k, n) for g, (m, n, k) in enumerate(sizes)]
    Ad, Bd, Cd = dev(A16), dev(B16), dev(C0)
    plan = b.gemm_grouped_plan_create(0, desc, 0, 1)   # B_g stored n x k (K-major)
    try:
        b.gemm_grouped_plan_run(plan, Ad, Bd, Cd, 1.0, 0.5, use_graph=1)
        b.tc_sync_status()
    finally:
        b.gemm_grouped_plan_destroy(plan)
    Cg = host(Cd)
    picks = np.unique(np.concatenate([(np.arange(300) * 33 + 1) % len(sizes), [0, len(sizes) - 1]]))
    for g in picks:
        m, n, k = (int(x) for x in sizes[g])
        Ag = A16[offa[g]:offa[g] + m * k].astype(np.float32).reshape(m, k)
        Bg = B16[offb[g]:offb[g] + n * k].astype(np.float32).reshape(n, k).T
        C0g = C0[offc[g]:offc[g] + m * n].reshape(m, n)
        ref = og.gemm_mixed("f16", Ag, Bg, 1.0, 0.5, C0g)
        got = Cg[offc[g]:offc[g] + m * n].reshape(m, n)
        mag = np.abs(Ag.astype(np.float64)) @ np.abs(Bg.astype(np.float64)) + 0.5 * np.abs(C0g.astype(np.float64))
        ok, info = elementwise_ok(got, ref, mag, k)
        assert ok, (g, (m, n, k), info)


def test_batched_1e6_sampled_problems(b):
    batch = 1_000_000
    A16 = synth.uniform((batch * 256,), seed=synth.seed_for(3, 4)).astype(np.float16)
    B16 = synth.uniform((batch * 256,), seed=synth.seed_for(3, 5)).astype(np.float16)
    Ad, Bd = dev(A16), dev(B16)
    Cd = torch.empty(batch * 256, dtype=torch.float32, device="cuda")
    b.gemm_batched_strided(0, batch, 16, 16, 16, 1.0, Ad, 256, 0, Bd, 256, 0, 0.0, Cd, 256)
    b.tc_sync_status()
    picks = np.unique(np.concatenate([(np.arange(2000) * 499 + 17) % batch, [0, batch - 1]]))
    idx = torch.from_numpy(picks).cuda()
    got = host(Cd.view(batch, 16, 16)[idx])
    Ap = A16.reshape(batch, 16, 16)[picks].astype(np.float32)
    Bp = B16.reshape(batch, 16, 16)[picks].astype(np.float32)
    ref = og.gemm_batched("f16", Ap, Bp)
    mag = np.abs(Ap.astype(np.float64)) @ np.abs(Bp.astype(np.float64))
    ok, info = elementwise_ok(got, ref, mag, 16)
    assert ok, info


# ------------------------------------------------------------------ served stream

def test_served_stream_sampled_requests(b):
    S = 4096
    Apool = synth.uniform((S, S), seed=synth.seed_for(4, 2))
    Bpool = synth.uniform((S, S), seed=synth.seed_for(4, 3))
    Ad, Bd = dev(Apool), dev(Bpool)
    _, sizes, modes = synth.serve_stream(96, seed=synth.seed_for(4, 0), rate_per_s=1.0)
    outs = [torch.full((int(m), int(n)), float("nan"), dtype=torch.float32, device="cuda") for (m, n, k) in sizes]
    srv = b.serve_open(40 << 30, max_inflight=32, num_streams=8)
    try:
        tickets = []
        for i, (m, n, k) in enumerate(sizes):
            t = None
            while t is None:
                t = b.serve_submit(srv, int(modes[i]), int(m), int(n), int(k), Ad, S, Bd, S, outs[i], int(n))
            tickets.append(t)
        b.serve_drain(srv, 120_000)
        for t in tickets:
            assert b.serve_poll(srv, t)["status"] == 0
    finally:
        b.serve_close(srv)
    for i, (m, n, k) in enumerate(sizes):
        m, n, k = int(m), int(n), int(k)
        rows = _samples(m, 8, 97, 1)
        cols = _samples(n, 16, 131, 2)
        A = Apool[:m, :k]
        B = Bpool[:k, :n]
        mode = synth.SERVE_MODES[int(modes[i])]
        got = host(outs[i])[rows][:, cols]
        if mode == "split3":
            ref = og.gemm_split("f16", 3, A, B, rows=rows, cols=cols)
            K = 3 * k
        else:
            ref = og.gemm_mixed(mode, A, B, rows=rows, cols=cols)
            K = k
        # |rounded| <= 1.25 |x| for every format here (E4M3 keeps 3 fraction bits)
        mag = 1.25 * np.abs(A[rows].astype(np.float64)) @ np.abs(B[:, cols].astype(np.float64))
        ok, info = elementwise_ok(got, ref, mag, K)
        assert ok, (i, mode, (m, n, k), info)
