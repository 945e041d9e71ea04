"""CPU oracle for the tensor-core GEMM path: plain, slow, obviously correct.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, calls or links it, and this package imports nothing from the product.

What it computes (all in FP64 unless a step is a rounding to a narrow format):

* ``numerics``: rounding of FP32 values to FP16, BF16 and FP8-E4M3 with IEEE
  round-to-nearest-even (Sec. V: "rounded" single -> half, range +-65504,
  epsilon 2^-10, gradual underflow), the per-tensor power-of-two E4M3 scale,
  and the hi/lo split that defines the residual matrices (Sec. V, the
  definition of R_A and Eq. 1 / Eq. 2).
* ``gemm``: C = alpha*A*B + beta*C (Sec. IV) on rounded inputs, the precision
  refinement with 2, 3 or 4 products (Eq. 1, Eq. 2), grouped and batched
  GEMM (Sec. IV-B), the FP64 truth on unrounded inputs, and the error norms
  (Sec. VI max norm; normwise ||C - C64||_F / (||A||_F ||B||_F)).

Every function's pins live in ``tests/test_oracle_*.py``.  No function here is
"parity unpinned".
"""
from . import numerics, gemm  # noqa: F401
