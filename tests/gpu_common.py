"""Shared helpers of the GPU parity tests (device transfers, tolerances)."""
import numpy as np
import pytest

try:
    import torch
except Exception:  # pragma: no cover
    torch = None

TOL_NORMWISE = 1e-5   # fp32-accumulate deviation from the same-rounded-input oracle


def need_gpu():
    if torch is None or not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def normwise_dev(C, C_ref, A, B, alpha=1.0, beta=0.0, C0=None):
    """||C - C_ref||_F / (|alpha| ||A||_F ||B||_F + |beta| ||C0||_F)."""
    d = np.asarray(C, np.float64) - np.asarray(C_ref, np.float64)
    den = abs(alpha) * np.linalg.norm(np.asarray(A, np.float64)) * np.linalg.norm(np.asarray(B, np.float64))
    if beta != 0.0 and C0 is not None:
        den += abs(beta) * np.linalg.norm(np.asarray(C0, np.float64))
    return float(np.linalg.norm(d) / den)


def elementwise_ok(C, C_ref, mag, K):
    """|C - C_ref| <= K * 2^-22 * mag + tiny, mag = |alpha| |A||B| + |beta| |C0| (FP32 accumulation bound)."""
    d = np.abs(np.asarray(C, np.float64) - np.asarray(C_ref, np.float64))
    bound = max(K, 1) * 2.0 ** -22 * np.asarray(mag, np.float64) + 1e-30
    bad = d > bound
    return (not np.any(bad)), (np.argwhere(bad)[:5].tolist(), float(d.max()) if d.size else 0.0)
