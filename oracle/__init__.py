"""CPU oracle for strong recursive skeletonization (RS-S).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never calls it and shares no code
with it; the only thing the two sides share is the seeded input generator in
``workloads``.

The oracle is a plain, slow, step-by-step restatement of the method of
"An O(N) distributed-memory parallel direct solver for planar integral
equations" (Liang, Chen, Martinsson, Biros), Algorithm 1 and Section 2.5, in
float64 / complex128 numpy.

Pins (tests under ``tests/test_oracle_*.py``, run with ``-m "not gpu"``):
  * kernel entries against textbook values and scipy's Bessel functions;
  * the column-pivoted QR ID against LAPACK's geqp3 pivots and the ID
    definition (Definition 1, Section 2.2);
  * the LU against scipy's getrf;
  * the FFT matvec against the dense matvec;
  * the whole factor/solve against a dense solve, and, with a kernel whose
    far field is exactly low rank, against the dense solve to rounding level
    (pins sparsification, elimination, merge and solve bookkeeping).

Parity unpinned: the exact per-level skeleton ranks.  The paper prints them
only as a figure (Fig. "Numerical ranks"), with no numbers in the text.
"""
from .rss import (KernelSpec, cpqr_id, lu_factor_pp, lu_solve_pp, factor, solve,
                  Factorization)
from .dense import dense_matrix, dense_matvec, fft_matvec, relres

__all__ = ["KernelSpec", "cpqr_id", "lu_factor_pp", "lu_solve_pp", "factor", "solve",
           "Factorization", "dense_matrix", "dense_matvec", "fft_matvec", "relres"]
