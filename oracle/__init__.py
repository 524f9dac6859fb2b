"""FP64 CPU oracle for the pass-efficient randomized low-rank SVD (Bjarkason 2018).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the
bench's CPU-baseline leg may import this package.  The GPU library never calls
it, links it or falls back to it, and this package imports nothing from the
GPU library (it shares only the seeded input generators).

Contents
  linalg      plain FP64 primitives written out from their definitions:
              Householder thin QR (diag R >= 0), Cholesky, triangular solves,
              one-sided Jacobi SVD, truncated SVD (Section 2 notation: qr,
              orth, tsvd, chol).  Matrix products use numpy's matmul.
  algorithms  the paper's algorithms step by step in its order: Alg. 1, Alg. 2
              (generalized subspace iteration), Alg. 7 (single pass, Tropp
              variant with l_c), Alg. 9 (generalized block Krylov), the
              row-streamed one-pass QB of Section 6.8 and the row-streamed
              block Krylov method of Section 7.3, plus the error measures of
              Section 8.2 and the bounds of Theorems 3.1 and 4.1.
  grad        reverse-mode derivatives of Alg. 2's outputs with respect to A
              (the sum of the top-k estimated singular values, and any loss
              on U, S and V; not in the paper).
  normal      the TEVD of a normal matrix J^T J from views of a matrix-free
              J (Section 4.2.3: Algs. 3, 4 and 5).
  extended    the other single-view methods of Section 6: Woolfe's variant
              (Alg. 8) and the extended SRFT sketch (Section 6.7).
  sharded     Alg. 2 on a matrix whose rows are split over several ranks
              (summed Grams and co-range partials).

Every function is pinned by tests that do not reuse it (closed forms, exact
recovery, brute force on tiny inputs, library routines, the paper's algebraic
equivalences and theorems).
"""
from . import linalg, algorithms, grad, normal, extended, sharded  # noqa: F401
