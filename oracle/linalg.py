"""Plain FP64 dense primitives (Section 2 of Bjarkason 2018).

Test infrastructure only (see the package docstring).  Each routine is the
textbook definition written out; numpy supplies array storage, elementwise
arithmetic and matrix products, nothing else.

Section 2 defines
  [Q, R] = qr(A):  A = QR, Q with orthonormal columns, R upper triangular
                   (thin QR).  The sign of R is not fixed by the paper; here
                   diag(R) >= 0, which makes the thin QR of a full-column-rank
                   matrix unique.
  Q = orth(A):     orthonormal basis of range(A) (Q of qr for full rank).
  [U, L, V] = tsvd(A, p):  the SVD of the best rank-p approximation.
  C = chol(A, LOWER):      A = C C^*.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "householder_qr", "orth", "cholesky_upper", "solve_upper", "solve_upper_right",
    "jacobi_svd", "tsvd", "fix_signs",
]


def householder_qr(y: np.ndarray):
    """Thin QR of y (m x n, m >= n) by Householder reflections, diag(R) >= 0.

    Column j: the reflector H_j = I - 2 w w^T with w = (x + sign(x_0)|x| e_1)
    / norm maps the trailing part x of column j onto a multiple of e_1 and is
    applied to the trailing columns.  Q is H_1 ... H_n applied to the first
    n columns of the identity.  Rank-deficient columns give a zero reflector
    (x = 0) and a zero diagonal in R, so the routine never divides by zero.
    """
    a = np.array(y, dtype=np.float64, copy=True)
    m, n = a.shape
    if m < n:
        raise ValueError("householder_qr needs rows >= cols")
    ws = []
    for j in range(n):
        x = a[j:, j]
        nx = np.sqrt(np.dot(x, x))
        w = x.copy()
        if nx == 0.0:
            ws.append(None)
            continue
        s = 1.0 if x[0] >= 0.0 else -1.0
        w[0] += s * nx
        nw = np.sqrt(np.dot(w, w))
        w /= nw
        ws.append(w)
        # a[j:, j:] <- (I - 2 w w^T) a[j:, j:]
        a[j:, j:] -= 2.0 * np.outer(w, w @ a[j:, j:])
    r = np.triu(a[:n, :n])
    q = np.zeros((m, n))
    q[np.arange(n), np.arange(n)] = 1.0
    for j in range(n - 1, -1, -1):
        w = ws[j]
        if w is None:
            continue
        q[j:, :] -= 2.0 * np.outer(w, w @ q[j:, :])
    d = np.where(np.diag(r) < 0.0, -1.0, 1.0)
    return q * d[None, :], r * d[:, None]


def orth(y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(y) for full-column-rank y (Q of qr)."""
    return householder_qr(y)[0]


def cholesky_upper(g: np.ndarray) -> np.ndarray:
    """Upper-triangular R with g = R^T R (g symmetric positive definite).

    Row j of R: r_jj = sqrt(g_jj - sum_i<j r_ij^2), and for l > j
    r_jl = (g_jl - sum_i<j r_ij r_il) / r_jj.  Raises on a pivot <= 0.
    """
    g = np.asarray(g, dtype=np.float64)
    n = g.shape[0]
    r = np.zeros((n, n))
    for j in range(n):
        d = g[j, j] - np.dot(r[:j, j], r[:j, j])
        if not d > 0.0:
            raise np.linalg.LinAlgError(f"non-positive pivot {d} at {j}")
        r[j, j] = np.sqrt(d)
        if j + 1 < n:
            r[j, j + 1:] = (g[j, j + 1:] - r[:j, j] @ r[:j, j + 1:]) / r[j, j]
    return r


def solve_upper(r: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x with r x = b (r upper triangular) by back substitution."""
    r = np.asarray(r, dtype=np.float64)
    b = np.array(b, dtype=np.float64, copy=True)
    vec = b.ndim == 1
    if vec:
        b = b[:, None]
    n = r.shape[0]
    x = np.zeros_like(b)
    for i in range(n - 1, -1, -1):
        x[i] = (b[i] - r[i, i + 1:] @ x[i + 1:]) / r[i, i]
    return x[:, 0] if vec else x


def solve_upper_right(b: np.ndarray, r: np.ndarray) -> np.ndarray:
    """x with x r = b (r upper triangular): x = b r^{-1}, column by column."""
    r = np.asarray(r, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = r.shape[0]
    x = np.zeros_like(b)
    for j in range(n):
        x[:, j] = (b[:, j] - x[:, :j] @ r[:j, j]) / r[j, j]
    return x


def _round_robin(n: int):
    """Rounds of disjoint index pairs covering every pair once (circle method)."""
    idx = list(range(n)) + ([None] if n % 2 else [])
    k = len(idx)
    rounds = []
    for _ in range(k - 1):
        pairs = [(idx[i], idx[k - 1 - i]) for i in range(k // 2)]
        rounds.append([(min(a, b), max(a, b)) for a, b in pairs if a is not None and b is not None])
        idx = [idx[0]] + [idx[-1]] + idx[1:-1]
    return rounds


def jacobi_svd(a: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """SVD a = U diag(s) V^T by one-sided (Hestenes) Jacobi, s descending.

    Works on the columns of a (rows >= cols; a wide matrix is handled through
    its transpose).  Each rotation makes one column pair orthogonal:
    alpha = |w_p|^2, beta = |w_q|^2, gamma = w_p . w_q,
    zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
    c = 1 / sqrt(1 + t^2), s = c t, and [w_p, w_q] <- [c w_p - s w_q, s w_p + c w_q].
    The same rotations applied to the identity give V.  Disjoint pairs of one
    round-robin round are rotated together.  Sweeps stop when every pair has
    |gamma| <= tol sqrt(alpha beta).  Then s_i = |w_i| and u_i = w_i / s_i
    (u_i = 0 for s_i = 0).  Returns U (rows x cols), s, V (cols x cols).
    """
    a = np.asarray(a, dtype=np.float64)
    if a.shape[0] < a.shape[1]:
        u, s, v = jacobi_svd(a.T, tol, max_sweeps)
        return v, s, u
    w = a.copy()
    n = w.shape[1]
    v = np.eye(n)
    rounds = [np.array(r, dtype=np.int64).reshape(-1, 2) for r in _round_robin(n)]
    for _ in range(max_sweeps):
        rotated = False
        for pr in rounds:
            if pr.size == 0:
                continue
            p, q = pr[:, 0], pr[:, 1]
            wp, wq = w[:, p], w[:, q]
            alpha = np.einsum("ij,ij->j", wp, wp)
            beta = np.einsum("ij,ij->j", wq, wq)
            gamma = np.einsum("ij,ij->j", wp, wq)
            act = np.abs(gamma) > tol * np.sqrt(alpha * beta)
            if not act.any():
                continue
            rotated = True
            g = np.where(act, gamma, 1.0)
            zeta = (beta - alpha) / (2.0 * g)
            t = np.where(zeta >= 0.0, 1.0, -1.0) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
            c = 1.0 / np.sqrt(1.0 + t * t)
            s = c * t
            c = np.where(act, c, 1.0)
            s = np.where(act, s, 0.0)
            w[:, p], w[:, q] = c * wp - s * wq, s * wp + c * wq
            vp, vq = v[:, p], v[:, q]
            v[:, p], v[:, q] = c * vp - s * vq, s * vp + c * vq
        if not rotated:
            break
    sv = np.sqrt(np.einsum("ij,ij->j", w, w))
    order = np.argsort(-sv, kind="stable")
    sv = sv[order]
    w = w[:, order]
    v = v[:, order]
    u = np.where(sv[None, :] > 0.0, w / np.where(sv > 0.0, sv, 1.0)[None, :], 0.0)
    return u, sv, v


def tsvd(a: np.ndarray, p: int):
    """[U_p, s_p, V_p] = tsvd(a, p): leading p singular triplets of a."""
    u, s, v = jacobi_svd(a)
    return u[:, :p], s[:p], v[:, :p]


def fix_signs(u: np.ndarray, v: np.ndarray):
    """Flip each pair (u_i, v_i) so the largest-magnitude entry of u_i is positive."""
    idx = np.argmax(np.abs(u), axis=0)
    sg = np.sign(u[idx, np.arange(u.shape[1])])
    sg[sg == 0] = 1.0
    return u * sg[None, :], v * sg[None, :]
