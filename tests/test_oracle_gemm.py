"""Pins of the oracle GEMM definitions.

Closed forms (identity, permutation, rank-1), integer-valued products checked
in exact integer arithmetic, the paper's 4x4 tensor-core operation by brute
force over exact rationals, the FP64 summation error against correctly rounded
dot products, and the algebra of Eq. 1 / Eq. 2 on inputs whose split is exact.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import gemm as og
from oracle import numerics as nm


def test_identity_returns_rounded_operand():
    B = synth.uniform((64, 48), seed=1)
    I = np.eye(64, dtype=np.float32)
    for dt in ("f16", "bf16"):
        assert np.array_equal(og.gemm_mixed(dt, I, B), nm.round_to(B, dt))
    C = og.gemm_mixed("f16", B.T, np.eye(64, dtype=np.float32))
    assert np.array_equal(C, nm.round_to(B.T, "f16"))


def test_permutation_is_exact_row_shuffle():
    B = synth.uniform((32, 40), seed=2)
    perm = (synth.words(32, seed=3).astype(np.int64)).argsort()
    P = np.zeros((32, 32), dtype=np.float32)
    P[np.arange(32), perm] = 1.0
    assert np.array_equal(og.gemm_mixed("f16", P, B), nm.round_to(B, "f16")[perm])


def test_integer_valued_products_are_exact():
    # |a|,|b| <= 16, K = 1024: every partial sum < 2^20, exact in FP16 inputs and FP64
    A = synth.integers((48, 1024), seed=4, lo=-16, hi=16)
    B = synth.integers((1024, 40), seed=5, lo=-16, hi=16)
    ref = A.astype(np.int64) @ B.astype(np.int64)
    for dt in ("f16", "bf16"):
        assert np.array_equal(og.gemm_mixed(dt, A, B), ref.astype(np.float64))
    # E4M3: integers up to 16 are exact after the power-of-two scale (16 * 16 = 256 <= 448)
    A8 = synth.integers((16, 256), seed=6, lo=-8, hi=8)
    B8 = synth.integers((256, 24), seed=7, lo=-8, hi=8)
    ref8 = (A8.astype(np.int64) @ B8.astype(np.int64)).astype(np.float64)
    assert np.array_equal(og.gemm_mixed("e4m3", A8, B8), ref8)


def test_rank_one_closed_form():
    K = 96
    u = synth.uniform((20,), seed=8)
    w = synth.uniform((30,), seed=9)
    u16 = nm.round_to(u, "f16").astype(np.float32)
    w16 = nm.round_to(w, "f16").astype(np.float32)
    A = np.repeat(u16[:, None], K, axis=1)
    B = np.repeat(w16[None, :], K, axis=0)
    want = K * np.outer(u16.astype(np.float64), w16.astype(np.float64))
    assert np.array_equal(og.gemm_mixed("f16", A, B), want)


def _exact_dot(a_row, b_col):
    return sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a_row, b_col))


def test_tensor_core_4x4_brute_force():
    # the paper's hardware operation: D = A*B + C on 4x4 matrices, FP16 A, B; FP32 C
    rng_bits = synth.words(3 * 16 * 200, seed=10).reshape(200, 3, 16)
    for t in range(200):
        a16 = (rng_bits[t, 0] & np.uint32(0xFFFF)).astype(np.uint16).view(np.float16)
        b16 = (rng_bits[t, 1] & np.uint32(0xFFFF)).astype(np.uint16).view(np.float16)
        # keep finite values (inf/nan patterns replaced by 1)
        a16 = np.where(np.isfinite(a16), a16, np.float16(1.0)).astype(np.float64).reshape(4, 4)
        b16 = np.where(np.isfinite(b16), b16, np.float16(1.0)).astype(np.float64).reshape(4, 4)
        c0 = synth.uniform((4, 4), seed=1000 + t)
        got = og.gemm_mixed("f16", a16, b16, alpha=1.0, beta=1.0, C0=c0)
        for i in range(4):
            for j in range(4):
                exact = _exact_dot(a16[i], b16[:, j]) + Fraction(float(c0[i, j]))
                mag = sum(abs(a16[i, k] * b16[k, j]) for k in range(4)) + abs(float(c0[i, j]))
                assert abs(Fraction(got[i, j]) - exact) <= Fraction(5 * mag) * Fraction(2) ** -53


def test_wmma_unit_16x16x16_brute_force():
    # Listing 1's unit of work: one 16x16x16 product of half inputs, FP32 output
    A = synth.uniform((16, 16), seed=11)
    B = synth.uniform((16, 16), seed=12)
    Ah = nm.round_to(A, "f16")
    Bh = nm.round_to(B, "f16")
    got = og.gemm_mixed("f16", A, B)
    for i in range(16):
        for j in range(16):
            # inputs in [-1,1]: all products are multiples of 2^-48 below 1, sums below 16 -> exact
            assert Fraction(got[i, j]) == _exact_dot(Ah[i], Bh[:, j])


def test_fp64_summation_error_is_bounded():
    A = synth.normal((24, 512), seed=13)
    B = synth.normal((512, 20), seed=14)
    Ah = nm.round_to(A, "f16")
    Bh = nm.round_to(B, "f16")
    got = og.gemm_mixed("f16", A, B)
    K = 512
    for i in range(24):
        for j in range(20):
            prods = Ah[i] * Bh[:, j]           # exact in FP64
            exact = math.fsum(prods)          # correctly rounded sum
            assert abs(got[i, j] - exact) <= K * 2.0 ** -53 * float(np.sum(np.abs(prods)))


def test_alpha_beta_epilogue():
    A = synth.uniform((16, 32), seed=15)
    B = synth.uniform((32, 8), seed=16)
    C0 = synth.uniform((16, 8), seed=17)
    base = og.gemm_mixed("f16", A, B)
    got = og.gemm_mixed("f16", A, B, alpha=2.5, beta=-0.5, C0=C0)
    assert np.allclose(got, 2.5 * base - 0.5 * C0.astype(np.float64), rtol=0, atol=1e-13)
    zero = og.gemm_mixed("f16", np.zeros_like(A), B, alpha=1.0, beta=0.75, C0=C0)
    assert np.array_equal(zero, 0.75 * C0.astype(np.float64))
    # beta = 0 never reads C0 (NaN in C0 does not propagate)
    nanC = np.full_like(C0, np.nan)
    assert np.all(np.isfinite(og.gemm_mixed("f16", A, B, beta=0.0, C0=nanC)))


def test_e4m3_descale():
    A = synth.uniform((8, 64), seed=18, lo=-4.0, hi=4.0)
    B = synth.uniform((64, 8), seed=19, lo=-0.5, hi=0.5)
    sa = nm.e4m3_scale(nm.absmax(A))
    sb = nm.e4m3_scale(nm.absmax(B))
    qa = nm.round_to(A.astype(np.float64) * sa, "e4m3")
    qb = nm.round_to(B.astype(np.float64) * sb, "e4m3")
    assert np.array_equal(og.gemm_mixed("e4m3", A, B), (qa @ qb) / (sa * sb))
    # operands exactly representable after scaling -> exact product
    A2 = nm.round_to(A.astype(np.float64) * sa, "e4m3") / sa
    B2 = nm.round_to(B.astype(np.float64) * sb, "e4m3") / sb
    assert np.allclose(og.gemm_mixed("e4m3", A2, B2), A2 @ B2, rtol=0, atol=1e-12)


def test_row_and_column_sampling_matches_full():
    A = synth.uniform((64, 96), seed=20)
    B = synth.uniform((96, 80), seed=21)
    C0 = synth.uniform((64, 80), seed=22)
    rows = np.array([0, 5, 63])
    cols = np.array([1, 79])
    for dt in ("f16", "bf16", "e4m3"):
        full = og.gemm_mixed(dt, A, B, 1.0, 0.5, C0)
        assert np.array_equal(og.gemm_mixed(dt, A, B, 1.0, 0.5, C0, rows=rows, cols=cols), full[rows][:, cols])
    for p in (2, 3, 4):
        full = og.gemm_split("f16", p, A, B, 1.0, 0.5, C0)
        assert np.array_equal(og.gemm_split("f16", p, A, B, 1.0, 0.5, C0, rows=rows, cols=cols), full[rows][:, cols])


# ---- Eq. 1 / Eq. 2 -------------------------------------------------------------

def _22bit_matrix(shape, seed):
    n = int(np.prod(shape))
    ints = (synth.words(n, seed=seed) & np.uint32((1 << 22) - 1)).astype(np.float64) + float(1 << 21)
    sgn = np.where(synth.words(n, seed=seed + 1) & np.uint32(1), -1.0, 1.0)
    return (sgn * ints * 2.0 ** -22).astype(np.float32).reshape(shape)   # |x| in [0.5, 1.5)


def test_eq2_four_products_recover_fp32_product():
    A = _22bit_matrix((24, 128), 30)
    B = _22bit_matrix((128, 16), 32)
    got = og.gemm_split("f16", 4, A, B)
    want = og.gemm_truth(A, B)
    assert np.allclose(got, want, rtol=0, atol=128 * 2.0 ** -50)


def test_eq1_two_products_equal_single_times_half():
    A = _22bit_matrix((24, 128), 34)
    B = _22bit_matrix((128, 16), 36)
    got = og.gemm_split("f16", 2, A, B)
    want = A.astype(np.float64) @ nm.round_to(B, "f16")
    assert np.allclose(got, want, rtol=0, atol=128 * 2.0 ** -50)


def test_three_products_drop_only_lo_lo():
    A = synth.log_uniform_pow2((16, 64), seed=38)
    B = synth.log_uniform_pow2((64, 12), seed=39)
    Ah, Al = nm.split(A, "f16")
    Bh, Bl = nm.split(B, "f16")
    diff = og.gemm_split("f16", 4, A, B) - og.gemm_split("f16", 3, A, B)
    # each sum is rounded in FP64: bound by K * 2^-52 times the sum of |terms|
    mag = (np.abs(Ah) + np.abs(Al)) @ (np.abs(Bh) + np.abs(Bl))
    assert np.all(np.abs(diff - Al @ Bl) <= 2 * 64 * 2.0 ** -52 * mag)
    assert np.max(np.abs(Al @ Bl)) > 1e3 * np.max(2 * 64 * 2.0 ** -52 * mag)


def test_split_of_half_inputs_equals_mixed():
    A = nm.round_to(synth.uniform((32, 64), seed=40), "f16").astype(np.float32)
    B = nm.round_to(synth.uniform((64, 24), seed=41), "f16").astype(np.float32)
    for p in (2, 3, 4):
        assert np.array_equal(og.gemm_split("f16", p, A, B), og.gemm_mixed("f16", A, B))


def test_split_beta_added_once():
    A = synth.uniform((8, 32), seed=42)
    B = synth.uniform((32, 8), seed=43)
    C0 = synth.uniform((8, 8), seed=44)
    no_c = og.gemm_split("f16", 4, A, B, alpha=2.0)
    with_c = og.gemm_split("f16", 4, A, B, alpha=2.0, beta=0.5, C0=C0)
    assert np.allclose(with_c - no_c, 0.5 * C0.astype(np.float64), rtol=0, atol=1e-14)


# ---- grouped / batched ----------------------------------------------------------

def test_grouped_and_batched_are_independent_problems():
    sizes = synth.group_sizes(6, seed=45)
    probs = []
    for g, (m, n, k) in enumerate(sizes):
        probs.append((synth.uniform((m, k), seed=100 + g), synth.uniform((k, n), seed=200 + g), None))
    outs = og.gemm_grouped("f16", probs)
    for (A, B, _), C in zip(probs, outs):
        assert np.array_equal(C, nm.round_to(A, "f16") @ nm.round_to(B, "f16"))
    A = synth.uniform((5, 16, 16), seed=46)
    B = synth.uniform((5, 16, 16), seed=47)
    Cb = og.gemm_batched("f16", A, B)
    for i in range(5):
        assert np.array_equal(Cb[i], og.gemm_mixed("f16", A[i], B[i]))


# ---- error norms -------------------------------------------------------------------

def test_error_norm_closed_forms():
    A = np.full((3, 4), 2.0)
    B = np.full((4, 5), 3.0)
    C_ref = np.zeros((3, 5))
    C = np.zeros((3, 5))
    C[1, 2] = -0.5
    C[2, 4] = 0.25
    assert og.max_error(C, C_ref) == 0.5
    want = math.sqrt(0.25 + 0.0625) / (math.sqrt(12 * 4.0) * math.sqrt(20 * 9.0))
    assert abs(og.normwise_error(C, C_ref, A, B) - want) < 1e-16
    s = og.error_sums(C, C_ref, A, B)
    assert s == (0.3125, 48.0, 180.0, 0.5)


def test_scaled_split_recovers_where_plain_split_cannot():
    # inputs with 22 significant bits and |x| in [2^-10, 2^-8): every plain FP16 residual is
    # subnormal and loses bits, the scaled residuals are normal and exact, so the scaled
    # Eq. 2 without R_A R_B differs from the FP32 product only by that dropped term
    def m22(shape, seed):
        n = int(np.prod(shape))
        ints = (synth.words(n, seed=seed) & np.uint32((1 << 22) - 1)).astype(np.float64) + float(1 << 21)
        e = (synth.words(n, seed=seed + 1) % 2).astype(np.float64) - 10.0
        sgn = np.where(synth.words(n, seed=seed + 2) & np.uint32(1), -1.0, 1.0)
        return (sgn * ints * 2.0 ** (e - 21)).astype(np.float32).reshape(shape)
    A = m22((20, 96), 60)
    B = m22((96, 12), 63)
    truth = og.gemm_truth(A, B)
    Ah, Al = nm.split_scaled(A, "f16")
    Bh, Bl = nm.split_scaled(B, "f16")
    want = truth - np.ldexp(Al @ Bl, -22)
    got = og.gemm_split_scaled("f16", 3, A, B)
    assert np.allclose(got, want, rtol=0, atol=96 * 2.0 ** -52 * np.max(np.abs(truth)))
    plain = og.gemm_split("f16", 3, A, B)
    assert og.normwise_error(plain, truth, A, B) > 10 * og.normwise_error(got, truth, A, B)
    # nprod = 2 is Eq. 1: A_single B_half
    got2 = og.gemm_split_scaled("f16", 2, A, B)
    assert np.allclose(got2, A.astype(np.float64) @ Bh, rtol=0, atol=96 * 2.0 ** -50 * np.max(np.abs(truth)))


def test_scaled_split_beta_alpha():
    A = synth.uniform((8, 32), seed=70)
    B = synth.uniform((32, 8), seed=71)
    C0 = synth.uniform((8, 8), seed=72)
    a = og.gemm_split_scaled("bf16", 3, A, B, alpha=2.0)
    b_ = og.gemm_split_scaled("bf16", 3, A, B, alpha=2.0, beta=-1.0, C0=C0)
    assert np.allclose(b_ - a, -C0.astype(np.float64), rtol=0, atol=1e-14)
    with pytest.raises(ValueError):
        og.gemm_split_scaled("f16", 4, A, B)


def _bits_matrix(shape, bits, seed, e_span=40):
    """FP32 values with exactly `bits` significant bits and exponents over e_span binades."""
    n = int(np.prod(shape))
    ints = (synth.words(n, seed=seed) & np.uint32((1 << (bits - 1)) - 1)).astype(np.float64) + float(1 << (bits - 1))
    e = (synth.words(n, seed=seed + 1) % e_span).astype(np.float64) - e_span // 2
    sgn = np.where(synth.words(n, seed=seed + 2) & np.uint32(1), -1.0, 1.0)
    return (sgn * ints * 2.0 ** (e - (bits - 1))).astype(np.float32).reshape(shape)


@pytest.mark.parametrize("bits_a,bits_b", [(16, 16), (24, 8), (8, 24)])
def test_bf16x3_products_are_exact_when_the_dropped_pieces_vanish(bits_a, bits_b):
    # the kept products are (0,0) (1,0) (0,1) (2,0) (1,1) (0,2): with 16-bit operands the third
    # pieces are zero, with 8-bit B its second and third pieces are, so every one of these cases
    # needs exactly the products that are kept and the result is the FP32 inputs' product
    K = 96
    A = _bits_matrix((20, K), bits_a, 80)
    B = _bits_matrix((K, 12), bits_b, 90)
    truth = og.gemm_truth(A, B)
    mag = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    got = og.gemm_split_bf16x3(A, B)
    assert np.all(np.abs(got - truth) <= 6 * K * 2.0 ** -52 * mag)


def test_bf16x3_error_is_below_fp32_roundoff():
    # dropped terms A1 B2 + A2 B1 + A2 B2 are at most (2^-24 + 2^-24 + 2^-32) |a||b| each
    K = 64
    A = _bits_matrix((24, K), 24, 100)
    B = _bits_matrix((K, 16), 24, 110)
    truth = og.gemm_truth(A, B)
    mag = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    got = og.gemm_split_bf16x3(A, B)
    assert np.all(np.abs(got - truth) <= (2.0 ** -23 + 2.0 ** -31 + 6 * K * 2.0 ** -52) * mag)
    # the two-piece BF16 refinement is far less accurate on the same inputs
    two = og.gemm_split("bf16", 4, A, B)
    assert og.normwise_error(two, truth, A, B) > 100 * og.normwise_error(got, truth, A, B)


def test_bf16x3_alpha_beta():
    A = synth.uniform((8, 32), seed=120)
    B = synth.uniform((32, 8), seed=121)
    C0 = synth.uniform((8, 8), seed=122)
    a = og.gemm_split_bf16x3(A, B, alpha=-2.0)
    b_ = og.gemm_split_bf16x3(A, B, alpha=-2.0, beta=0.5, C0=C0)
    assert np.allclose(b_ - a, 0.5 * C0.astype(np.float64), rtol=0, atol=1e-14)
    assert np.array_equal(og.gemm_split_bf16x3(A, B, rows=[3, 1], cols=[0, 7]),
                          og.gemm_split_bf16x3(A, B)[[3, 1]][:, [0, 7]])


def _int_codes(q, step_exp):
    """q (FP64 values on a grid of 2^step_exp) -> Python ints q * 2^-step_exp."""
    scaled = np.asarray(q, np.float64) * 2.0 ** (-step_exp)
    ints = np.rint(scaled)
    assert np.array_equal(ints, scaled)       # every value lies on the grid
    return ints.astype(np.int64).astype(object)


@pytest.mark.parametrize("K", [256, 512])
def test_exact_integer_sums_pin_the_fp64_product_fp16(K):
    # at the depths of the GPU parity tests: every FP16 value is an integer multiple of 2^-24, so the
    # exact dot products are integers times 2^-48, summed here in Python integers.  With inputs in
    # [2^-6, 1) every partial sum needs at most 48 - 32 + 9 + 1 < 53 bits: the FP64 product is exact.
    # With the tests' uniform[-1,1] inputs it is within the FP64 summation bound K * 2^-53 * sum|ab|.
    M = N = 12
    mag = synth.uniform((M, K), seed=20, lo=0.0, hi=1.0) * 0.984375 + 0.015625
    sgn = np.where(synth.uniform((M, K), seed=21) < 0, -1.0, 1.0)
    A_narrow = (mag * sgn).astype(np.float32)
    B_narrow = (synth.uniform((K, N), seed=22, lo=0.0, hi=1.0) * 0.984375 + 0.015625).astype(np.float32)
    for A, B, exact_expected in ((A_narrow, B_narrow, True),
                                 (synth.uniform((M, K), seed=23), synth.uniform((K, N), seed=24), False)):
        got = og.gemm_mixed("f16", A, B)
        ia = _int_codes(nm.round_to(A, "f16"), -24)
        ib = _int_codes(nm.round_to(B, "f16"), -24)
        S = ia.dot(ib)                                   # exact, Python integers
        absS = np.abs(ia).dot(np.abs(ib))
        for i in range(M):
            for j in range(N):
                exact = Fraction(int(S[i, j]), 2 ** 48)
                if exact_expected:
                    assert Fraction(got[i, j]) == exact
                else:
                    bound = Fraction(K, 2 ** 53) * Fraction(int(absS[i, j]), 2 ** 48)
                    assert abs(Fraction(got[i, j]) - exact) <= bound


@pytest.mark.parametrize("K", [256, 512])
def test_exact_integer_sums_pin_the_fp64_product_e4m3(K):
    # E4M3 codes (after the power-of-two scale) are multiples of 2^-9 below 448, so every partial sum
    # of K <= 2^20 products is an integer times 2^-18 below 2^38: the FP64 product is exact, and so
    # is the descale by the power-of-two scales
    M, N = 10, 14
    A = synth.uniform((M, K), seed=25) * 3.0
    B = synth.uniform((K, N), seed=26) * 0.25
    got = og.gemm_mixed("e4m3", A, B)
    qa, sa = nm.quantize(A, "e4m3")
    qb, sb = nm.quantize(B, "e4m3")
    ia = _int_codes(qa, -9)
    ib = _int_codes(qb, -9)
    S = ia.dot(ib)
    descale = Fraction(1) / (Fraction(float(sa)) * Fraction(float(sb)))
    for i in range(M):
        for j in range(N):
            assert Fraction(got[i, j]) == Fraction(int(S[i, j]), 2 ** 18) * descale
