"""GPU parity of the batched entry points the serving loop uses: many small
roundings in one launch (tc_quantize_batch) and a grouped GEMM whose schedule
lives in caller-owned device memory (gemm_grouped_ws), on the tcgen05 kernel and on the mma.sync kernel."""
import numpy as np
import pytest

import synth
from oracle import gemm as og
from oracle import numerics as nm
from tests.gpu_common import dev, elementwise_ok, host, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b():
    need_gpu()
    from paper_1803_04014_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("dt", [0, 1])
def test_quantize_batch_bit_exact(b, dt):
    tdt = torch.float16 if dt == 0 else torch.bfloat16
    # ragged sizes, both layouts, padded and unpadded destinations (vector and scalar stores)
    shapes = [(1, 1, 0, 0), (37, 70, 0, 2), (64, 32, 1, 0), (130, 33, 1, 5), (300, 257, 0, 8), (65, 129, 1, 8),
              (16, 16, 0, 0), (200, 1000, 1, 3)]
    srcs, dsts, jobs, want = [], [], [], []
    for i, (rows, cols, tr, pad) in enumerate(shapes):
        X = synth.log_uniform_pow2((rows, cols), seed=synth.seed_for(6, i))
        Xd = dev(X)
        drows, dcols = (cols, rows) if tr else (rows, cols)
        ld = dcols + pad
        D = torch.full((drows, ld), -7.0, dtype=tdt, device="cuda")
        jobs.append((rows, cols, Xd, cols, D, ld, tr))
        srcs.append(Xd)
        dsts.append(D)
        w = nm.round_to(X, "f16" if dt == 0 else "bf16")
        want.append(w.T if tr else w)
    need = b.tc_quantize_batch_workspace_bytes(jobs)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    b.tc_quantize_batch(dt, jobs, ws, need)
    for (rows, cols, _, _, D, ld, tr), w in zip(jobs, want):
        got = host(D.to(torch.float64))
        dcols = rows if tr else cols
        assert np.array_equal(got[:, :dcols], w)
        assert np.all(got[:, dcols:] == -7.0)          # padding untouched
    with pytest.raises(b.TcError):
        b.tc_quantize_batch(dt, jobs, ws, need - 16)
    with pytest.raises(b.TcError):
        b.tc_quantize_batch(2, jobs, ws, need)          # E4M3 needs a per-tensor scale


def test_quantize_batch_e4m3_matches_per_tensor_rounding(b):
    # each job's scale and codes equal tc_quantize's (and the oracle's) bit for bit: ragged sizes,
    # both layouts, padded and unaligned destinations, an empty job, an all-zero job, magnitudes
    # far apart (each job gets its own scale), one job with inf and NaN (NaN ignored by the max,
    # inf gives scale 1)
    shapes = [(1, 1, 0, 0, 1.0), (37, 70, 0, 2, 1e-6), (64, 32, 1, 0, 3e4), (130, 33, 1, 5, 1.0),
              (300, 257, 0, 8, 0.02), (65, 129, 1, 8, 7.0), (0, 16, 0, 0, 1.0), (16, 16, 0, 0, 0.0),
              (200, 1000, 1, 3, 1.0), (40, 48, 0, 0, 1.0)]
    jobs, dsts, scales, srcs = [], [], [], []
    for i, (rows, cols, tr, pad, mag) in enumerate(shapes):
        X = synth.log_uniform_pow2((rows, cols), seed=synth.seed_for(6, 60 + i)) * np.float32(mag)
        if i == 9:
            X[3, 5], X[7, 9] = np.inf, np.nan
        srcs.append(X)
        Xd = dev(X) if X.size else torch.empty((max(rows, 1), max(cols, 1)), device="cuda")
        drows, dcols = (cols, rows) if tr else (rows, cols)
        ld = max(dcols + pad, 1)
        D = torch.full((max(drows, 1), ld), 0x55, dtype=torch.uint8, device="cuda")
        jobs.append((rows, cols, Xd, max(cols, 1), D, ld, tr))
        dsts.append(D)
        scales.append(torch.full((1,), -1.0, device="cuda"))
    need = b.tc_quantize_batch_workspace_bytes(jobs)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    b.tc_quantize_batch_e4m3(jobs, scales, ws, need)
    b.tc_sync_status()
    for (rows, cols, Xd, lds, D, ld, tr), X, sc in zip(jobs, srcs, scales):
        # the same rounding one tensor at a time
        D1 = torch.full_like(D, 0x55)
        s1 = torch.full((1,), -1.0, device="cuda")
        b.tc_quantize(2, rows, cols, Xd, lds, D1, ld, tr, s1)
        b.tc_sync_status()
        assert float(host(sc)[0]) == float(host(s1)[0])
        assert torch.equal(D, D1)
        if rows and cols and np.all(np.isfinite(X)):
            want, s = nm.quantize(X, "e4m3")
            assert float(host(sc)[0]) == s
            got = nm.e4m3_value(host(D))[:, :(rows if tr else cols)]
            assert np.array_equal(got, want.T if tr else want)   # the oracle's values carry the scale
    assert float(host(scales[6])[0]) == 1.0 and float(host(scales[7])[0]) == 1.0
    with pytest.raises(b.TcError):
        b.tc_quantize_batch_e4m3(jobs, scales, ws, need - 16)
    with pytest.raises(b.TcError):
        b.tc_quantize_batch_e4m3(jobs, scales[:-1] + [0], ws, need)   # a null scale pointer


@pytest.mark.parametrize("impl", ["tc", "mma"])
@pytest.mark.parametrize("lb", [0, 1])
def test_grouped_ws_matches_oracle_and_runs_concurrently(b, lb, impl, monkeypatch):
    if impl == "mma":
        monkeypatch.setenv("TCGEMM_GROUPED", "mma")
    rng_sizes = synth.group_sizes(150, seed=synth.seed_for(6, 40))
    def build(sizes, seed):
        offa = offb = offc = 0
        desc, probs = [], []
        for g, (m, n, k) in enumerate(sizes):
            desc.append((m, n, k, offa, offb, offc, k, (n if lb == 0 else k), n))
            offa += m * k
            offb += k * n
            offc += m * n
        A = synth.uniform((offa,), seed=seed).astype(np.float16)
        B = synth.uniform((offb,), seed=seed + 1).astype(np.float16)
        C0 = synth.uniform((offc,), seed=seed + 2)
        return desc, A, B, C0
    d1, A1, B1, C1 = build(rng_sizes[:80], synth.seed_for(6, 41))
    d2, A2, B2, C2 = build(rng_sizes[80:], synth.seed_for(6, 44))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for desc, A, B, C0, st in ((d1, A1, B1, C1, s1), (d2, A2, B2, C2, s2)):
        need = b.gemm_grouped_workspace_bytes(desc)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        Ad, Bd, Cd = dev(A), dev(B), dev(C0)
        torch.cuda.synchronize()
        b.gemm_grouped_ws(0, desc, Ad, 0, Bd, lb, Cd, 1.0, 0.5, ws, need, stream=st)
        outs.append((desc, A, B, C0, Cd, ws, Ad, Bd))
    torch.cuda.synchronize()
    b.tc_sync_status()
    for desc, A, B, C0, Cd, _, _, _ in outs:
        Cg = host(Cd)
        for (m, n, k, oa, ob, oc, lda, ldb, ldc) in desc:
            Ag = A[oa:oa + m * k].astype(np.float32).reshape(m, k)
            if lb == 0:
                Bg = B[ob:ob + k * n].astype(np.float32).reshape(k, n)
            else:
                Bg = B[ob:ob + k * n].astype(np.float32).reshape(n, k).T
            C0g = C0[oc:oc + m * n].reshape(m, n)
            ref = og.gemm_mixed("f16", Ag, Bg, 1.0, 0.5, C0g)
            mag = np.abs(Ag.astype(np.float64)) @ np.abs(Bg.astype(np.float64)) + 0.5 * np.abs(C0g)
            ok, info = elementwise_ok(Cg[oc:oc + m * n].reshape(m, n), ref, mag, k)
            assert ok, ((m, n, k), info)
    desc, _, _, _, Cd, ws, Ad, Bd = outs[0]
    with pytest.raises(b.TcError):
        b.gemm_grouped_ws(0, desc, Ad, 0, Bd, lb, Cd, 1.0, 0.0, ws, 64)
