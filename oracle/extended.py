"""The other single-view methods of Section 6, FP64: the Woolfe variant
(Alg. 8, Sec. 6.5) and the extended sketching scheme with SRFT test matrices
(Sec. 6.7, the approximation bwz2).

Test infrastructure only (see the package docstring).  Letters as in
oracle/algorithms.py (k = the paper's p; Omega = the paper's Omega_r,
n x ell1; Psi = the paper's Omega_c, m x ell2).  Random inputs -- the
Gaussian test matrices, the Rademacher signs and the sampled DCT columns of
an SRFT -- are arguments, never drawn here.
"""
from __future__ import annotations

import numpy as np

from .linalg import fix_signs, householder_qr, solve_upper, tsvd

__all__ = ["dct_matrix", "srft", "woolfe_single_pass", "extended_single_pass"]


def dct_matrix(n):
    """The orthonormal DCT-II matrix F (n x n) whose columns are the cosine
    basis vectors: F[j, k] = c_k sqrt(2 / n) cos(pi (2 j + 1) k / (2 n)),
    c_0 = 1 / sqrt(2), c_k = 1 otherwise, so a row vector times F is its
    DCT-II."""
    j = np.arange(n)[:, None]
    k = np.arange(n)[None, :]
    f = np.sqrt(2.0 / n) * np.cos(np.pi * (2 * j + 1) * k / (2.0 * n))
    f[:, 0] /= np.sqrt(2.0)
    return f


def srft(n, signs, cols):
    """Phi = D F P (n x s): D = diag(signs) (Rademacher, +-1), F the DCT-II
    matrix of dct_matrix, P the s columns `cols` (distinct, in [0, n)) of
    the identity: Phi[j, t] = signs[j] F[j, cols[t]]."""
    signs = np.asarray(signs, dtype=np.float64)
    cols = np.asarray(cols)
    return signs[:, None] * dct_matrix(n)[:, cols]


def woolfe_single_pass(a, omega, psi, k, l_c=None):
    """Alg. 8: Y_c = A Omega, Y_r = A^T Psi; [Q_c, R_c] = qr(Y_c),
    [Q_r, R_r] = qr(Y_r); Q^_c, Q^_r the leading k + l_c left singular
    vectors of R_c, R_r; Q_c = Q_c Q^_c, Q_r = Q_r Q^_r; X^ the least-squares
    solution of (Psi^T Q_c) X^ = Y_r^T Q_r; [U^, L, V^] = tsvd(X^, k);
    U = Q_c U^, V = Q_r V^.  l_c = None means l_c = l_1 (ell1 - k)."""
    a = np.asarray(a, dtype=np.float64)
    ell1 = omega.shape[1]
    lc = ell1 - k if l_c is None else int(l_c)
    kc = k + lc
    yc = a @ omega
    yr = a.T @ psi
    qc, rc = householder_qr(yc)
    qr_, rr = householder_qr(yr)
    qc = qc @ tsvd(rc, kc)[0]
    qr_ = qr_ @ tsvd(rr, kc)[0]
    qh, rh = householder_qr(psi.T @ qc)          # least squares through the QR of Psi^T Q_c
    x = solve_upper(rh, qh.T @ (yr.T @ qr_))
    uh, s, vh = tsvd(x, k)
    u, v = fix_signs(qc @ uh, qr_ @ vh)
    return u, s, v


def extended_single_pass(a, omega, psi, phi_c, phi_r, k):
    """Sec. 6.7, the approximation bwz2: Y_c = A Omega, Y_r = A^T Psi,
    Z = Phi_r^T A Phi_c; Q_c R_c = Y_c, Q_r R_r = Y_r; U_c T_c = Phi_r^T Q_c,
    U_r T_r = Phi_c^T Q_r; C = T_c^+ U_c^T Z U_r (T_r^T)^+ (T_c, T_r are
    square and invertible for full-rank sketches, s >= ell);
    [U^, L, V^] = tsvd(C, k); U = Q_c U^, V = Q_r V^."""
    a = np.asarray(a, dtype=np.float64)
    yc = a @ omega
    yr = a.T @ psi
    z = phi_r.T @ (a @ phi_c)
    qc, _ = householder_qr(yc)
    qr_, _ = householder_qr(yr)
    uc, tc = householder_qr(phi_r.T @ qc)
    ur, tr = householder_qr(phi_c.T @ qr_)
    core = uc.T @ z @ ur                          # T_c C T_r^T
    core = solve_upper(tc, core)                  # T_c^{-1} (.)
    core = solve_upper(tr, core.T).T              # (.) T_r^{-T} = (T_r^{-1} (.)^T)^T
    uh, s, vh = tsvd(core, k)
    u, v = fix_signs(qc @ uh, qr_ @ vh)
    return u, s, v
