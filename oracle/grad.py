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
  * square SVD R = W S Z^T with distinct singular values, given Wb, Sb, Zb
    (zero beyond the k kept columns): Rb = W [ (F o (W^T Wb - Wb^T W)) S
    + diag(Sb) + S (F o (Z^T Zb - Zb^T Z)) ] Z^T, F_ij = 1 / (s_j^2 - s_i^2)
    (i != j), F_ii = 0 -- the kept pairs couple to every other pair.
  * the lifts U = Q_c U^_k, V = Q_r V^_k: Qb_c += Ub U^_k^T, U^b = Q_c^T Ub,
    and likewise for V; the sign fix flips a pair (u_i, v_i) by a constant,
    so its gradients flip with it.
"""
from __future__ import annotations

import numpy as np

from .linalg import householder_qr, jacobi_svd, solve_upper

__all__ = ["qr_backward", "svd_backward", "topk_sigma_sum", "grad_topk_sigma_sum", "lowrank_outputs",
           "grad_lowrank"]


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


def svd_backward(w, s, z, wbar, sbar, zbar):
    """Rb for a square R = W diag(s) Z^T (full SVD, distinct s) given Wb, Sb,
    Zb (any of them None for zero)."""
    n = s.shape[0]
    wbar = np.zeros((n, n)) if wbar is None else wbar
    zbar = np.zeros((n, n)) if zbar is None else zbar
    sbar = np.zeros(n) if sbar is None else sbar
    s2 = s * s
    diff = s2[None, :] - s2[:, None]          # s_j^2 - s_i^2
    f = np.zeros((n, n))
    off = ~np.eye(n, dtype=bool)
    f[off] = 1.0 / diff[off]
    jw = f * (w.T @ wbar - wbar.T @ w)
    jz = f * (z.T @ zbar - zbar.T @ z)
    inner = jw * s[None, :] + np.diag(sbar) + s[:, None] * jz
    return w @ inner @ z.T


def lowrank_outputs(a, omega, k, v):
    """(U, S, V) of Alg. 2 (sign-fixed), the function the reverse pass differentiates."""
    from .algorithms import gen_subspace_iteration
    return gen_subspace_iteration(np.asarray(a, dtype=np.float64), omega, k, v)


def grad_lowrank(a, omega, k, v, ubar=None, sbar=None, vbar=None):
    """dL/dA for L = <Ub, U> + <Sb, S> + <Vb, V> with (U, S, V) = Alg. 2's
    output (lowrank_outputs), by the reverse pass of the same steps."""
    a = np.asarray(a, dtype=np.float64)
    m, n = a.shape
    tape = _forward(a, omega, v)
    q_last, r_last = tape[-1][2], tape[-1][3]
    q_prev = tape[-2][2]
    w, sv, z = jacobi_svd(r_last)
    ell = sv.shape[0]
    # the outputs before the sign fix: v odd R_c = U^ L V^^T; v even R_r = V^ L U^^T
    if v % 2 == 1:
        qc, qr_, uh, vh = q_last, q_prev, w[:, :k], z[:, :k]
    else:
        qc, qr_, uh, vh = q_prev, q_last, z[:, :k], w[:, :k]
    u_raw = qc @ uh
    idx = np.argmax(np.abs(u_raw), axis=0)
    d = np.sign(u_raw[idx, np.arange(k)])
    d[d == 0] = 1.0
    ub = np.zeros((m, k)) if ubar is None else ubar * d[None, :]
    vb = np.zeros((n, k)) if vbar is None else vbar * d[None, :]
    sb = np.zeros(k) if sbar is None else np.asarray(sbar, dtype=np.float64)
    # lifts
    qb_c, uhb = ub @ uh.T, qc.T @ ub
    qb_r, vhb = vb @ vh.T, qr_.T @ vb
    pad = lambda x: np.hstack([x, np.zeros((ell, ell - k))])  # noqa: E731
    sbar_full = np.concatenate([sb, np.zeros(ell - k)])
    if v % 2 == 1:
        rbar = svd_backward(w, sv, z, pad(uhb), sbar_full, pad(vhb))
        qbar_last, qbar_prev = qb_c, qb_r
    else:
        rbar = svd_backward(w, sv, z, pad(vhb), sbar_full, pad(uhb))
        qbar_last, qbar_prev = qb_r, qb_c
    qbar = qbar_last
    da = np.zeros_like(a)
    for t, (j, x, q, r) in enumerate(reversed(tape)):
        bbar = qr_backward(q, r, qbar, rbar)
        if j % 2 == 1:            # B = A X
            da += bbar @ x.T
            qbar = a.T @ bbar
        else:                     # B = A^T X
            da += x @ bbar.T
            qbar = a @ bbar
        if t == 0:                # Q of view v - 1 also feeds a lift
            qbar = qbar + qbar_prev
        rbar = None
    return da
