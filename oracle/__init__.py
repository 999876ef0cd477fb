"""CPU oracle for fast SVT matrix completion (Feng, Yu & Li, arXiv 1810.06860).

TEST INFRASTRUCTURE ONLY.  Plain, slow float64 restatements of the paper's
algorithms used to check the GPU library.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it; the library itself never does, and this package
imports nothing from the library.

Contents
  philox   -- Philox4x32-10 counter RNG and the Box-Muller Gaussian Omega
  rsvd     -- eigSVD (Alg. 3), lu basis (Lemma 3), orth, basic rSVD (Alg. 1),
              rSVD-PI (Alg. 4), rSVD-BKI (Alg. 5), recycling (Sec. IV.B)
  svt      -- SVT with exact SVD (Alg. 2), fast SVT (Alg. 6), ||P_Phi M||_2
  metrics  -- completion error on Phi, held-out RMSE/MAE (eq. (10)),
              singular-value error, principal angles

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, textbook routines or brute force.  The
paper's printed tables (Sec. V) use datasets that are not available, so the
oracle is not pinned to those numbers.
"""
from . import metrics, philox, rsvd, svt  # noqa: F401
