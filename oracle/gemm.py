"""GEMM definitions of the method, evaluated in FP64 on the CPU.

Oracle code (test infrastructure only; see the package header).

Matrices are given in their mathematical shape: A is (M, K), B is (K, N),
C0 is (M, N).  Storage layouts are the concern of the code under test, not of
the definitions here.  The one library primitive used is the FP64 matrix
product (numpy ``@``); every FP16/BF16/E4M3 value and every product of two of
them is exact in FP64, so the only rounding inside a product is the FP64
summation, which the pins bound.

* ``gemm_mixed``  -- Sec. IV: C = alpha*A*B + beta*C, with A and B first
  rounded to the input format (Sec. VI: "the values of A and B are first
  rounded to half precision"); for E4M3 each operand carries a per-tensor
  power-of-two scale and C = alpha/(s_A s_B) * (A s_A)_q (B s_B)_q + beta*C0.
* ``gemm_split``  -- precision refinement, Eq. 1 (2 products: R_A B_half +
  A_half B_half) and Eq. 2 (4 products: R_A R_B + A_half R_B + R_A B_half +
  A_half B_half); 3 products drops R_A R_B.  All products are summed into one
  result, alpha multiplies the sum, beta*C0 is added once (reading of the
  paper's chained beta=0,1,1,1 pipeline, Sec. VI).
* ``gemm_split_scaled`` -- the same refinement with residuals scaled by 2^s
  before rounding (Ootomo and Yokota, 2022) and the correction products
  summed apart and multiplied by 2^-s.
* ``gemm_split_bf16x3`` -- three BF16 pieces per operand and the six
  products whose piece orders add up to at most 2 (Henry et al., 2019).
* ``gemm_truth``  -- alpha*A*B + beta*C0 on the unrounded FP32 inputs.
* ``gemm_grouped`` / ``gemm_batched`` -- Sec. IV-B: independent problems.
* ``normwise_error`` / ``max_error`` -- ||C - C_ref||_F / (||A||_F ||B||_F)
  and the paper's max norm ||e||_max = max |e_ij| (Sec. VI).
"""
from __future__ import annotations

import numpy as np

from . import numerics

# (A piece, B piece) index pairs; 0 = hi (the rounded matrix), 1 = lo (the residual)
PRODUCTS = {
    2: ((0, 0), (1, 0)),                  # Eq. 1: A_half B_half + R_A B_half
    3: ((0, 0), (1, 0), (0, 1)),          # Eq. 2 without R_A R_B
    4: ((0, 0), (1, 0), (0, 1), (1, 1)),  # Eq. 2
}


# three-piece BF16 split: (A piece, B piece) with piece order sum <= 2, largest first
PRODUCTS_BF16X3 = ((0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2))


def _f64(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float64)


def _epilogue(acc, alpha, beta, C0):
    C = float(alpha) * acc
    if beta != 0.0:
        C = C + float(beta) * _f64(C0)
    return C


def gemm_mixed(dt: str, A, B, alpha: float = 1.0, beta: float = 0.0, C0=None,
               rows=None, cols=None) -> np.ndarray:
    """C = alpha*descale*(q(A) q(B)) + beta*C0 with q the rounding to ``dt``.

    ``rows``/``cols`` restrict the result to a sample of C (the E4M3 scales are
    still taken over the whole of A and B).
    """
    A = _f64(A)
    B = _f64(B)
    amax_a = numerics.absmax(A) if dt == "e4m3" else None
    amax_b = numerics.absmax(B) if dt == "e4m3" else None
    As = A if rows is None else A[rows]
    Bs = B if cols is None else B[:, cols]
    Aq, sa = numerics.quantize(As, dt, amax_a)
    Bq, sb = numerics.quantize(Bs, dt, amax_b)
    acc = (Aq @ Bq) * (1.0 / (sa * sb))
    if C0 is not None and beta != 0.0:
        C0 = _f64(C0)
        if rows is not None:
            C0 = C0[rows]
        if cols is not None:
            C0 = C0[:, cols]
    return _epilogue(acc, alpha, beta, C0)


def gemm_split(piece: str, nprod: int, A, B, alpha: float = 1.0, beta: float = 0.0, C0=None,
               rows=None, cols=None) -> np.ndarray:
    """Precision refinement: alpha * sum over the products of Eq. 1/2 + beta*C0."""
    if nprod not in PRODUCTS:
        raise ValueError("nprod must be 2, 3 or 4")
    A = _f64(A)
    B = _f64(B)
    if rows is not None:
        A = A[rows]
    if cols is not None:
        B = B[:, cols]
    Ap = numerics.split(A, piece)
    Bp = numerics.split(B, piece)
    acc = np.zeros((A.shape[0], B.shape[1]), dtype=np.float64)
    for pa, pb in PRODUCTS[nprod]:
        acc += Ap[pa] @ Bp[pb]
    if C0 is not None and beta != 0.0:
        C0 = _f64(C0)
        if rows is not None:
            C0 = C0[rows]
        if cols is not None:
            C0 = C0[:, cols]
    return _epilogue(acc, alpha, beta, C0)


def gemm_split_scaled(piece: str, nprod: int, A, B, alpha: float = 1.0, beta: float = 0.0, C0=None,
                      rows=None, cols=None) -> np.ndarray:
    """Refinement with scaled residuals (Ootomo and Yokota, 2022):

    C = alpha * (A_hi B_hi + 2^-s (A_lo' B_hi [+ A_hi B_lo'])) + beta*C0,
    lo' = round((x - hi) * 2^s); nprod = 2 keeps Eq. 1's product pair, nprod = 3
    Eq. 2 without the residual-residual product (about 2^-2s of the result).
    """
    if nprod not in (2, 3):
        raise ValueError("the scaled split takes nprod 2 or 3")
    A = _f64(A)
    B = _f64(B)
    if rows is not None:
        A = A[rows]
    if cols is not None:
        B = B[:, cols]
    Ah, Al = numerics.split_scaled(A, piece)
    Bh, Bl = numerics.split_scaled(B, piece)
    corr = Al @ Bh
    if nprod == 3:
        corr = corr + Ah @ Bl
    acc = Ah @ Bh + np.ldexp(corr, -numerics.SPLIT_SCALE_EXP[piece])
    if C0 is not None and beta != 0.0:
        C0 = _f64(C0)
        if rows is not None:
            C0 = C0[rows]
        if cols is not None:
            C0 = C0[:, cols]
    return _epilogue(acc, alpha, beta, C0)


def gemm_split_bf16x3(A, B, alpha: float = 1.0, beta: float = 0.0, C0=None,
                      rows=None, cols=None) -> np.ndarray:
    """C = alpha * sum_{i+j<=2} A_i B_j + beta*C0 over the BF16 triples of A and B.

    The dropped products A_1 B_2, A_2 B_1 and A_2 B_2 are each below 2^-24 of
    |a||b|, the unit roundoff of FP32.
    """
    A = _f64(A)
    B = _f64(B)
    if rows is not None:
        A = A[rows]
    if cols is not None:
        B = B[:, cols]
    Ap = numerics.split_bf16x3(A)
    Bp = numerics.split_bf16x3(B)
    acc = np.zeros((A.shape[0], B.shape[1]), dtype=np.float64)
    for pa, pb in PRODUCTS_BF16X3:
        acc += Ap[pa] @ Bp[pb]
    if C0 is not None and beta != 0.0:
        C0 = _f64(C0)
        if rows is not None:
            C0 = C0[rows]
        if cols is not None:
            C0 = C0[:, cols]
    return _epilogue(acc, alpha, beta, C0)


def gemm_truth(A, B, alpha: float = 1.0, beta: float = 0.0, C0=None, rows=None, cols=None) -> np.ndarray:
    """FP64 result on the unrounded FP32 inputs (the accuracy reference)."""
    A = _f64(A)
    B = _f64(B)
    if rows is not None:
        A = A[rows]
    if cols is not None:
        B = B[:, cols]
    if C0 is not None and beta != 0.0:
        C0 = _f64(C0)
        if rows is not None:
            C0 = C0[rows]
        if cols is not None:
            C0 = C0[:, cols]
    return _epilogue(A @ B, alpha, beta, C0)


def gemm_grouped(dt: str, problems, alpha: float = 1.0, beta: float = 0.0):
    """Independent problems [(A_g, B_g, C0_g or None), ...] -> [C_g, ...]."""
    return [gemm_mixed(dt, A, B, alpha, beta, C0) for (A, B, C0) in problems]


def gemm_batched(dt: str, A, B, alpha: float = 1.0, beta: float = 0.0, C0=None) -> np.ndarray:
    """Strided batch: A (b, m, k), B (b, k, n) -> C (b, m, n), one problem at a time."""
    A = _f64(A)
    B = _f64(B)
    out = np.empty((A.shape[0], A.shape[1], B.shape[2]), dtype=np.float64)
    for i in range(A.shape[0]):
        c0 = None if C0 is None else C0[i]
        out[i] = gemm_mixed(dt, A[i], B[i], alpha, beta, c0)
    return out


def frobenius(x) -> float:
    x = _f64(x)
    return float(np.sqrt(np.sum(x * x)))


def normwise_error(C, C_ref, A, B) -> float:
    """||C - C_ref||_F / (||A||_F ||B||_F)."""
    d = _f64(C) - _f64(C_ref)
    den = frobenius(A) * frobenius(B)
    return float(np.sqrt(np.sum(d * d)) / den) if den > 0 else float(np.sqrt(np.sum(d * d)))


def max_error(C, C_ref) -> float:
    """||C - C_ref||_max = max |C_ij - C_ref_ij| (Sec. VI)."""
    d = _f64(C) - _f64(C_ref)
    return float(np.max(np.abs(d))) if d.size else 0.0


def error_sums(C, C64, A, B):
    """The four sums the device error reduction returns, in FP64:
    (sum (C - C64)^2, sum A^2, sum B^2, max |C - C64|)."""
    d = _f64(C) - _f64(C64)
    a = _f64(A)
    b = _f64(B)
    return (float(np.sum(d * d)), float(np.sum(a * a)), float(np.sum(b * b)),
            float(np.max(np.abs(d))) if d.size else 0.0)
