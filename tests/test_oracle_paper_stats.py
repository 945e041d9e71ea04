"""Statistical pins against the numbers the paper prints (Sec. VII-B).

The paper's figures are seed-dependent maxima, so these tests check order of
magnitude and ratios, on a row/column sample of C (the maximum over fewer
entries is slightly smaller; the bounds below allow a factor of two).
The paper measures against an FP32 GEMM; the oracle measures against the
FP64 truth, which removes the FP32 accumulation error from both sides, so the
refined errors here are smaller than the paper's and the pins on refinement
are one-sided (at least the paper's improvement).
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import gemm as og


@pytest.fixture(scope="module")
def paper(golden_dir):
    with open(os.path.join(golden_dir, "paper_numbers.json")) as f:
        return json.load(f)


def _sample(n, count, seed):
    return np.sort(synth.words(count, seed=seed).astype(np.int64) % n)


@pytest.mark.slow
def test_pm16_n4096_errors(paper):
    ref = paper["refinement_uniform_pm16_n4096"]
    N = 4096
    A = synth.uniform((N, N), seed=synth.seed_for(2, 0), lo=-16.0, hi=16.0)
    B = synth.uniform((N, N), seed=synth.seed_for(2, 1), lo=-16.0, hi=16.0)
    rows = _sample(N, 512, 1)
    cols = _sample(N, 1024, 2)
    truth = og.gemm_truth(A, B, rows=rows, cols=cols)
    e0 = og.max_error(og.gemm_mixed("f16", A, B, rows=rows, cols=cols), truth)
    e4 = og.max_error(og.gemm_split("f16", 4, A, B, rows=rows, cols=cols), truth)
    assert ref["emax_no_refinement"] / 2 < e0 < ref["emax_no_refinement"] * 2
    # inputs on the 2^-19 grid split exactly into two FP16 pieces, so Eq. 2 in
    # exact arithmetic leaves only FP64 rounding: far below the paper's 0.24
    assert e4 < ref["emax_refined_RA_RB"]
    assert e0 > ref["reduction_factor"] * e4


@pytest.mark.slow
def test_pm1_n8192_refinement_ratios(paper):
    ref = paper["refinement_uniform_pm1_n8192"]
    N = 8192
    A = synth.uniform((N, N), seed=synth.seed_for(2, 0))
    B = synth.uniform((N, N), seed=synth.seed_for(2, 1))
    rows = _sample(N, 256, 3)
    cols = _sample(N, 512, 4)
    A = A[rows]
    B = B[:, cols]
    truth = og.gemm_truth(A, B)
    e0 = og.max_error(og.gemm_mixed("f16", A, B), truth)
    e2 = og.max_error(og.gemm_split("f16", 2, A, B), truth)
    e4 = og.max_error(og.gemm_split("f16", 4, A, B), truth)
    # Eq. 1 removes one of two equal-norm error sources: about 30 % (1 - 1/sqrt 2)
    drop = 1.0 - e2 / e0
    assert abs(drop - ref["emax_reduction_RA_only_fraction"]) < 0.12
    # Eq. 2: at least the paper's factor of ten
    assert e0 > ref["emax_reduction_RA_RB_factor"] * e4


@pytest.mark.slow
def test_log_uniform_split_is_inexact_but_close():
    # full 24-bit significands: the two FP16 pieces cannot hold every value, so
    # Eq. 2 leaves a residual error, still far below the unrefined one
    N = 2048
    A = synth.log_uniform_pow2((128, N), seed=synth.seed_for(3, 0))
    B = synth.log_uniform_pow2((N, 128), seed=synth.seed_for(3, 1))
    truth = og.gemm_truth(A, B)
    e0 = og.normwise_error(og.gemm_mixed("f16", A, B), truth, A, B)
    e3 = og.normwise_error(og.gemm_split("f16", 3, A, B), truth, A, B)
    e4 = og.normwise_error(og.gemm_split("f16", 4, A, B), truth, A, B)
    assert e4 > 0 and e3 >= e4
    assert e0 > 100 * e3
    # FP16 pieces hold 22 of 24 bits: relative error of a piece pair about 2^-22
    assert e4 < 2.0 ** -20


def test_error_grows_with_n_like_sqrt_n():
    # Sec. VII-B: the error grows with N.  With independent rounding errors the
    # typical entry error grows like sqrt(K); check the fitted slope lies well
    # below the linear and quadratic readings.
    errs = []
    Ns = [256, 1024, 4096]
    for N in Ns:
        A = synth.uniform((64, N), seed=50 + N)
        B = synth.uniform((N, 64), seed=60 + N)
        d = og.gemm_mixed("f16", A, B) - og.gemm_truth(A, B)
        errs.append(float(np.sqrt(np.mean(d * d))))
    slope = np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert 0.35 < slope < 0.65
