"""Reverse-mode derivative of the top-k singular-value sum of Alg. 2 (FP64).

Test infrastructure only (see the package docstring).  The paper has no
derivatives; this is the standard matrix calculus of the same FP64 steps:

  view j (odd):  B_j = A Q_r,    [Q_c, R_c] = qr(B_j)
  view j (even): B_j = A^T Q_c,  [Q_r, R_r] = qr(B_j)
  loss L = sum_{i<=k} sigma_i(R) with R = R_r (v even) or R_c (v odd).

Rules used (the random Omega is a constant):
  * sigma-sum of a square R = W S Z^T: dL/dR = W_k Z_k^T (distinct sigma_k,
    sigma_{k+1}), since d sigma_i = w_i^T dR z_i.
  * thin QR Y = Q R (full column rank), given Qb = dL/dQ, Rb = dL/dR:
    M = R Rb^T - Qb^T Q, Yb = (Qb + Q copyltu(M)) R^{-T}, with
    copyltu(M) = tril(M) + tril(M, -1)^T.  This follows from
    Q^T dY R^{-1} = C + dR R^{-1}, C = Q^T dQ skew-symmetric, dR R^{-1}
    upper triangular.
  * B = A X: dA += Bb X^T, Xb = A^T Bb;  B = A^T X: dA += X Bb^T, Xb = A Bb.
"""
from __future__ import annotations

import numpy as np

from .linalg import householder_qr, jacobi_svd, solve_upper

__all__ = ["qr_backward", "topk_sigma_sum", "grad_topk_sigma_sum"]


def qr_backward(q, r, qbar, rbar):
    """Yb for Y = Q R given Qb, Rb (either may be None for zero)."""
    n = r.shape[0]
    qbar = np.zeros_like(q) if qbar is None else qbar
    rbar = np.zeros((n, n)) if rbar is None else rbar
    mm = r @ rbar.T - qbar.T @ q
    sym = np.tril(mm) + np.tril(mm, -1).T
    rhs = qbar + q @ sym
    # Yb = rhs R^{-T}  <=>  R Yb^T = rhs^T (back substitution).
    return solve_upper(r, rhs.T).T


def _forward(a, omega, v):
    qr_ = np.asarray(omega, dtype=np.float64)
    qc = None
    tape = []
    for j in range(1, v + 1):
        if j % 2 == 1:
            x = qr_
            qc, rc = householder_qr(a @ x)
            tape.append((j, x, qc, rc))
        else:
            x = qc
            qr_, rr = householder_qr(a.T @ x)
            tape.append((j, x, qr_, rr))
    return tape


def topk_sigma_sum(a, omega, k, v):
    """L(A) = sum of the k largest singular values estimated by Alg. 2."""
    a = np.asarray(a, dtype=np.float64)
    tape = _forward(a, omega, v)
    r = tape[-1][3]
    return float(np.sum(jacobi_svd(r)[1][:k]))


def grad_topk_sigma_sum(a, omega, k, v):
    """dL/dA for L = topk_sigma_sum(A, Omega, k, v), by the reverse pass."""
    a = np.asarray(a, dtype=np.float64)
    tape = _forward(a, omega, v)
    r_last = tape[-1][3]
    w, _, z = jacobi_svd(r_last)
    rbar = w[:, :k] @ z[:, :k].T
    qbar = None
    da = np.zeros_like(a)
    for j, x, q, r in reversed(tape):
        bbar = qr_backward(q, r, qbar, rbar)
        if j % 2 == 1:            # B = A X
            da += bbar @ x.T
            qbar = a.T @ bbar
        else:                     # B = A^T X
            da += x @ bbar.T
            qbar = a @ bbar
        rbar = None
    return da
