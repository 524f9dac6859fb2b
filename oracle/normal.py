"""Truncated eigendecomposition of a normal matrix J^T J from views of J alone,
FP64 (Bjarkason 2018, Section 4.2.3: Algs. 3, 4 and 5).

Test infrastructure only (see the package docstring).  J is matrix-free: it
enters as two callables, apply(X) = J X and apply_t(W) = J^T W, so the same
code serves a Jacobian applied by direct and adjoint methods.  The random
start is an input, never drawn here.  Letters as in the rest of the oracle:
k = the paper's target rank p, ell = k + p (the paper's p + l).

Every function returns (V, lam2): V (n_c x k) with orthonormal columns and
lam2 (k,) the approximate leading eigenvalues of J^T J, descending; the sign
of each column of V is fixed so that its largest-magnitude entry is positive.
"""
from __future__ import annotations

import numpy as np

from .linalg import cholesky_upper, householder_qr, orth, solve_upper_right, tsvd

__all__ = ["MatrixOperator", "qrqc", "nystrom_tevd", "pinched_tevd"]


class MatrixOperator:
    """J given as an explicit matrix (n_r x n_c): apply = J X, apply_t = J^T W."""

    def __init__(self, j):
        self.j = np.asarray(j, dtype=np.float64)
        self.rows, self.cols = self.j.shape

    def apply(self, x):
        return self.j @ x

    def apply_t(self, w):
        return self.j.T @ w

    def transpose(self):
        return MatrixOperator(self.j.T)


class _Transposed:
    """J^T as an operator, from J's two callables."""

    def __init__(self, op):
        self.op = op
        self.rows, self.cols = op.cols, op.rows

    def apply(self, x):
        return self.op.apply_t(x)

    def apply_t(self, w):
        return self.op.apply(w)


def _transpose(op):
    return op.op if isinstance(op, _Transposed) else _Transposed(op)


def _sign_cols(v):
    idx = np.argmax(np.abs(v), axis=0)
    sgn = np.sign(v[idx, np.arange(v.shape[1])])
    sgn[sgn == 0] = 1.0
    return v * sgn[None, :]


def qrqc(op, omega, v):
    """Alg. 3: an approximate basis of the column space (v odd) or the row
    space (v even) of J after v views, starting from Q_r = Omega (n_c x ell):
    odd j -> Q_c = qr(J Q_r), even j -> Q_r = qr(J^T Q_c).  v = 0 returns
    Omega as it is."""
    qr_ = np.asarray(omega, dtype=np.float64)
    qc = None
    for j in range(1, v + 1):
        if j % 2 == 1:
            qc, _ = householder_qr(op.apply(qr_))
        else:
            qr_, _ = householder_qr(op.apply_t(qc))
    return qr_ if v % 2 == 0 else qc


def nystrom_tevd(op, omega, k, v, eps=2.2e-16, norm="2"):
    """Alg. 4: the Nystrom (prolonged) TEVD of J^T J with v >= 2 views of J.

    Q_r: orth(Omega) for v = 2; qrqc(J, Omega, v - 2) for even v (Omega
    n_c x ell); qrqc(J^T, Omega, v - 2) for odd v (Omega n_r x ell).  Then
    Y_r = J^T (J Q_r), nu = eps ||Y_r||_2, Y_r <- Y_r + nu Q_r,
    B = Q_r^T Y_r, C_L = chol((B + B^T) / 2) (lower), F = C_L^{-1} Y_r^T,
    [~, Lam^, V] = tsvd(F, k), lam2 = max(Lam^^2 - nu, 0).
    eps is the paper's unit-roundoff constant (2.2e-16 for FP64) and norm its
    ||.|| (the 2-norm); the GPU library shifts by 2^-23 ||Y_r||_F in FP32,
    which a parity test passes here as eps = 2**-23, norm = "fro"."""
    if v < 2:
        raise ValueError("Alg. 4 needs v >= 2")
    if v == 2:
        qr_ = orth(np.asarray(omega, dtype=np.float64))
    elif v % 2 == 0:
        qr_ = qrqc(op, omega, v - 2)
    else:
        qr_ = qrqc(_transpose(op), omega, v - 2)
    yr = op.apply_t(op.apply(qr_))
    nu = eps * np.linalg.norm(yr, 2 if norm == "2" else "fro")
    yr = yr + nu * qr_
    b = qr_.T @ yr
    cu = cholesky_upper(0.5 * (b + b.T))   # C_L = cu^T
    ft = solve_upper_right(yr, cu)         # F^T = Y_r C_L^{-T} = Y_r cu^{-1}
    vk, lam, _ = tsvd(ft, k)               # right singular vectors of F = left ones of F^T
    lam2 = np.maximum(lam ** 2 - nu, 0.0)
    return _sign_cols(vk), lam2


def pinched_tevd(op, omega, k, v):
    """Alg. 5: the pinched TEVD of J^T J with v >= 2 views of J.

    Q_r = qrqc(J^T, Omega, v - 1) for even v (Omega n_r x ell), qrqc(J,
    Omega, v - 1) for odd v (Omega n_c x ell); B_c = J Q_r;
    [lam2, V^] = tevd(B_c^T B_c, k); V = Q_r V^."""
    if v < 2:
        raise ValueError("Alg. 5 needs v >= 2")
    if v % 2 == 0:
        qr_ = qrqc(_transpose(op), omega, v - 1)
    else:
        qr_ = qrqc(op, omega, v - 1)
    bc = op.apply(qr_)
    # tevd of B_c^T B_c through the SVD of B_c's triangular factor:
    # B_c = Q R, R = U^ S W^T  =>  B_c^T B_c = W^ S^2 W^^T
    _, r = householder_qr(bc)
    _, s, w = tsvd(r, k)
    return _sign_cols(qr_ @ w), s ** 2
