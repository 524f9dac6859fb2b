"""The paper's algorithms, step by step, in FP64 (Bjarkason 2018).

Test infrastructure only (see the package docstring).  Notation follows the
paper except for three letters (the library's API uses the same mapping):
  paper target rank p       -> k
  paper oversampling l      -> p     (sketch width ell = k + p, paper's k)
  paper Omega_r / Omega_c   -> Omega (n x ell) / Psi (m x ell2)
The random test matrices are inputs, never drawn here, so the GPU library can
be given the same arrays.  Every function returns U (m x k), s (k,), V (n x k)
with the sign of each pair (u_i, v_i) fixed so that the largest-magnitude
entry of u_i is positive.
"""
from __future__ import annotations

import math

import numpy as np

from .linalg import fix_signs, householder_qr, jacobi_svd, solve_upper, solve_upper_right, tsvd

__all__ = [
    "subspace_iteration", "gen_subspace_iteration", "single_pass", "block_krylov",
    "rowwise_qb_svd", "rowwise_block_krylov", "rel_frob_error", "rel_spec_error",
    "frob_error", "thm31_bound", "thm41_bound", "view_count_block_krylov",
    "oversampling_flat", "oversampling_decay", "oversampling_rapid", "lc_fixed_ratio",
    "minvar_spectra", "minvar_lc", "single_pass_minvar",
]


def _out(u, s, v):
    u, v = fix_signs(u, v)
    return u, s, v


def subspace_iteration(a, omega, k, q):
    """Alg. 1 (Section 3): standard subspace iteration with 2(q+1) views.

    Q_c = qr(A Omega); q times {Q_r = qr(A^T Q_c), Q_c = qr(A Q_r)};
    [Q_r, R_r] = qr(A^T Q_c); [V^, L, U^] = tsvd(R_r, k); U = Q_c U^, V = Q_r V^.
    """
    a = np.asarray(a, dtype=np.float64)
    qc, _ = householder_qr(a @ omega)
    for _ in range(q):
        qr_, _ = householder_qr(a.T @ qc)
        qc, _ = householder_qr(a @ qr_)
    qr_, rr = householder_qr(a.T @ qc)
    vh, s, uh = tsvd(rr, k)              # R_r = V^ L U^T
    return _out(qc @ uh, s, qr_ @ vh)


def gen_subspace_iteration(a, omega, k, v, return_state=False):
    """Alg. 2 (Section 4): generalized subspace iteration, any v >= 2 views.

    Q_r = Omega; for j = 1..v: odd j -> [Q_c, R_c] = qr(A Q_r);
    even j -> [Q_r, R_r] = qr(A^T Q_c).  v even: [V^, L, U^] = tsvd(R_r, k);
    v odd: [U^, L, V^] = tsvd(R_c, k).  U = Q_c U^, V = Q_r V^.
    """
    if v < 2:
        raise ValueError("Alg. 2 needs v >= 2")
    a = np.asarray(a, dtype=np.float64)
    qr_ = np.asarray(omega, dtype=np.float64)
    qc = rc = rr = None
    for j in range(1, v + 1):
        if j % 2 == 1:
            qc, rc = householder_qr(a @ qr_)
        else:
            qr_, rr = householder_qr(a.T @ qc)
    if v % 2 == 0:
        vh, s, uh = tsvd(rr, k)
    else:
        uh, s, vh = tsvd(rc, k)
    out = _out(qc @ uh, s, qr_ @ vh)
    if return_state:
        return out, dict(qc=qc, qr=qr_, rc=rc, rr=rr)
    return out


def single_pass(a, omega, psi, k, l_c=None, return_state=False):
    """Alg. 7 (Section 6.5): 1-view TSVD, Tropp variant with truncation l_c.

    omega: n x (k + l_1), psi: m x (k + l_2), l_2 >= l_1 >= l_c >= 0.
    Y_c = A Omega and Y_r = A^T Psi (one view); if l_c < l_1:
    [Q_c, R_c] = qr(Y_c), Q^_c = leading k + l_c left singular vectors of R_c,
    Q_c = Q_c Q^_c; else Q_c = qr(Y_c).  [Q^, R^] = qr(Psi^T Q_c),
    X = R^{-1} Q^T Y_r^T, [U^, L, V] = tsvd(X, k), U = Q_c U^.
    l_c = None means l_c = l_1 (the baseline method of Tropp et al.).
    """
    a = np.asarray(a, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    ell1 = omega.shape[1]
    l1 = ell1 - k
    if l_c is None:
        l_c = l1
    if not (psi.shape[1] >= ell1 and 0 <= l_c <= l1):
        raise ValueError("need l_2 >= l_1 >= l_c >= 0")
    yc = a @ omega
    yr = a.T @ psi
    qc, rc = householder_qr(yc)
    if l_c < l1:
        qhat, _, _ = tsvd(rc, k + l_c)
        qc = qc @ qhat
    qh, rh = householder_qr(psi.T @ qc)
    x = solve_upper(rh, qh.T @ yr.T)
    uh, s, vv = tsvd(x, k)
    out = _out(qc @ uh, s, vv)
    if return_state:
        return out, dict(yc=yc, yr=yr, qc=qc, x=x)
    return out


def block_krylov(a, omega, k, v, return_state=False):
    """Alg. 9 (Section 7.2): generalized block Krylov, any v >= 2 views.

    Q_r^0 = Omega.  For j = 1..v-1: odd j -> Q_c^j = qr(A Q_r^{j-1}) (raw
    A Q_r^{j-1} when j = v-1); even j -> Q_r^j = qr(A^T Q_c^{j-1}) (raw when
    j = v-1).  v even: K_c = [Q_c^1 Q_c^3 .. Q_c^{v-1}], Q_c = qr(K_c),
    [Q_r, R_r] = qr(A^T Q_c), [V^, L, U^] = tsvd(R_r, k).  v odd:
    K_r = [Q_r^2 .. Q_r^{v-1}], Q_r = qr(K_r), [Q_c, R_c] = qr(A Q_r),
    [U^, L, V^] = tsvd(R_c, k).  U = Q_c U^, V = Q_r V^.
    """
    if v < 2:
        raise ValueError("Alg. 9 needs v >= 2")
    a = np.asarray(a, dtype=np.float64)
    qprev = np.asarray(omega, dtype=np.float64)
    blocks = []
    for j in range(1, v):
        last = j == v - 1
        b = a @ qprev if j % 2 == 1 else a.T @ qprev
        qj = b if last else householder_qr(b)[0]
        if (j % 2 == 1) == (v % 2 == 0):
            blocks.append(qj)       # Q_c^j for even v, Q_r^j for odd v
        qprev = qj
    kk = np.concatenate(blocks, axis=1)
    if v % 2 == 0:
        qc, _ = householder_qr(kk)
        qr_, rr = householder_qr(a.T @ qc)
        vh, s, uh = tsvd(rr, k)
    else:
        qr_, _ = householder_qr(kk)
        qc, rc = householder_qr(a @ qr_)
        uh, s, vh = tsvd(rc, k)
    out = _out(qc @ uh, s, qr_ @ vh)
    if return_state:
        return out, dict(qc=qc, qr=qr_, k=kk)
    return out


def _rowwise_pass(a, x, rows_per_block=256):
    """One pass over the rows of A: Y[i,:] = A[i,:] X and Z = sum_i A[i,:]^T Y[i,:].

    This is the row-streamed evaluation of Section 6.8: each block of rows is
    used for its slice of Y and, while it is at hand, for its contribution to
    A^T Y.  The result equals (A X, A^T A X).
    """
    m = a.shape[0]
    y = np.zeros((m, x.shape[1]))
    z = np.zeros((a.shape[1], x.shape[1]))
    for i0 in range(0, m, rows_per_block):
        ai = a[i0:i0 + rows_per_block]
        y[i0:i0 + rows_per_block] = ai @ x
        z += ai.T @ y[i0:i0 + rows_per_block]
    return y, z


def rowwise_qb_svd(a, omega, k):
    """Section 6.8: one row-streamed pass giving the 2-view QB factorisation.

    Y_c = A Omega and Y^_r = A^T Y_c from one pass; [Q_c, R_c] = qr(Y_c);
    B solves B^T R_c = Y^_r (B^T = Y^_r R_c^{-1} = A^T Q_c for invertible
    R_c); then the TSVD of B: B^T = Q_b R_b, [V^, L, U^] = tsvd(R_b, k),
    U = Q_c U^, V = Q_b V^.
    """
    a = np.asarray(a, dtype=np.float64)
    yc, yr = _rowwise_pass(a, np.asarray(omega, dtype=np.float64))
    qc, rc = householder_qr(yc)
    bt = solve_upper_right(yr, rc)
    qb, rb = householder_qr(bt)
    vh, s, uh = tsvd(rb, k)
    return _out(qc @ uh, s, qb @ vh)


def rowwise_block_krylov(a, omega, k, v, return_state=False):
    """Section 7.3: block Krylov for row-streamed A, v views (v >= 2).

    Each of views 1..v-1 is one row-streamed pass giving Y = A X and
    Z = A^T Y (Section 6.8); with [Q_c, R_c] = qr(Y), A^T Q_c = Z R_c^{-1}
    is the next co-range block: orthonormalised (X = qr(Z R_c^{-1})) except
    after view v-1, where it is kept raw.  The co-range Krylov space
    K_r = [A^T Q_c^1 .. A^T Q_c^{v-1}] thus holds v-1 blocks from v-1 views
    (Alg. 9 needs 2v-3 views for it).  Q_r = qr(K_r); the last view is
    [Q_c, R_c] = qr(A Q_r); [U^, L, V^] = tsvd(R_c, k).  In exact arithmetic
    this equals Alg. 9 with 2v-1 views.
    """
    if v < 2:
        raise ValueError("needs v >= 2")
    a = np.asarray(a, dtype=np.float64)
    x = np.asarray(omega, dtype=np.float64)
    blocks = []
    for i in range(1, v):
        y, z = _rowwise_pass(a, x)
        _, rc = householder_qr(y)
        w = solve_upper_right(z, rc)          # A^T Q_c = Z R_c^{-1}
        x = w if i == v - 1 else householder_qr(w)[0]
        blocks.append(x)
    qr_, _ = householder_qr(np.concatenate(blocks, axis=1))
    qc, rc = householder_qr(a @ qr_)
    uh, s, vh = tsvd(rc, k)
    out = _out(qc @ uh, s, qr_ @ vh)
    if return_state:
        return out, dict(qc=qc, qr=qr_)
    return out


def view_count_block_krylov(v, ell):
    """Matrix-vector products of Alg. 9: (v + floor(v/2) - 1) ell (Section 7.2)."""
    return (v + v // 2 - 1) * ell


# ------------------------------------------------------------- Section 8.2
def frob_error(a, u, s, v):
    """|A - U diag(s) V^T|_F in FP64."""
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - (u * s[None, :]) @ v.T))


def rel_frob_error(a, u, s, v, tail_frob):
    """Relative Frobenius error: |A - A_out|_F / |A - [[A]]_k|_F - 1 (eq. relfroberr)."""
    return frob_error(a, u, s, v) / tail_frob - 1.0


def _spec_norm(m, iters=200, seed=0):
    """Largest singular value by power iteration on m^T m (FP64)."""
    g = np.random.Generator(np.random.PCG64(seed))
    x = g.standard_normal(m.shape[1])
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = m.T @ (m @ x)
        lam = np.linalg.norm(y)
        if lam == 0.0:
            return 0.0
        x = y / lam
    return math.sqrt(lam)


def rel_spec_error(a, u, s, v, tail_spec):
    """Relative spectral error: |A - A_out| / |A - [[A]]_k| - 1 (eq. relspecerr)."""
    r = np.asarray(a, dtype=np.float64) - (u * s[None, :]) @ v.T
    return _spec_norm(r) / tail_spec - 1.0


# ------------------------------------------------------ Theorems 3.1, 4.1
def thm31_bound(lam, p, l, q):
    """Theorem 3.1 bound on E|A - Q_c Q_c^* A| for Y_c = (A A^*)^q A Omega.

    p = target rank (paper), l = oversampling, lam = singular values.
    [(1 + sqrt(p/(l-1))) lam_{p+1}^{2q+1} + e sqrt(p+l)/l (sum_{j>p}
    lam_j^{2(2q+1)})^{1/2}]^{1/(2q+1)}.
    """
    lam = np.asarray(lam, dtype=np.float64)
    e = 2 * q + 1
    t1 = (1.0 + math.sqrt(p / (l - 1.0))) * lam[p] ** e
    t2 = math.e * math.sqrt(p + l) / l * math.sqrt(np.sum(lam[p:] ** (2 * e)))
    return (t1 + t2) ** (1.0 / e)


def thm41_bound(lam, p, l, q):
    """Theorem 4.1 bound on E|A - A Q_r Q_r^*| for Y_r = (A^* A)^q Omega, q >= 1.

    [(1 + sqrt(p/(l-1))) lam_{p+1}^{2q} + e sqrt(p+l)/l (sum_{j>p}
    lam_j^{4q})^{1/2}]^{1/(2q)}.
    """
    lam = np.asarray(lam, dtype=np.float64)
    e = 2 * q
    t1 = (1.0 + math.sqrt(p / (l - 1.0))) * lam[p] ** e
    t2 = math.e * math.sqrt(p + l) / l * math.sqrt(np.sum(lam[p:] ** (2 * e)))
    return (t1 + t2) ** (1.0 / e)


# ------------------------------- Section 6.3 (FLAT/DECAY/RAPID) and 6.6 (l_c) parameters
def oversampling_flat(T, p):
    """(l_1, l_2) for a flat spectrum: l_1 = max{2, floor((T - 1) (sqrt(p (T - p - 2)
    (1 - 2 / (T - 1))) - (p - 1)) / (T - 2p - 1)) - p}, l_2 = T - 2p - l_1."""
    q = (T - 1) * (math.sqrt(p * (T - p - 2) * (1 - 2 / (T - 1))) - (p - 1)) / (T - 2 * p - 1)
    l1 = max(2, int(math.floor(q)) - p)
    return l1, T - 2 * p - l1


def oversampling_decay(T, p):
    """(l_1, l_2) for a moderately decaying spectrum: l_1 = max{2, floor((T - 1) / 3) - p}."""
    l1 = max(2, int(math.floor((T - 1) / 3)) - p)
    return l1, T - 2 * p - l1


def oversampling_rapid(T, p):
    """(l_1, l_2) for a rapidly decaying spectrum: l_1 = floor((T - 2) / 2) - p."""
    l1 = int(math.floor((T - 2) / 2)) - p
    return l1, T - 2 * p - l1


def lc_fixed_ratio(l1, alpha):
    """l_c = floor(alpha l_1)."""
    return int(math.floor(alpha * l1))


def minvar_spectra(a, omega, psi, k):
    """Leading k singular values of X(l_c) for l_c = 0 .. l_1 (rows of the result).

    Alg. 7 with each trial l_c: Q_c holds the leading k + l_c left singular
    vectors of Y_c = A Omega, [Q^, R^] = qr(Psi^T Q_c), X = R^{-1} Q^T Y_r^T
    with Y_r = A^T Psi.
    """
    a = np.asarray(a, dtype=np.float64)
    yc = a @ omega
    yr = a.T @ psi
    ell1 = omega.shape[1]
    q, r = householder_qr(yc)
    w, _, _ = jacobi_svd(r)
    qfull = q @ w                      # left singular vectors of Y_c
    out = []
    for lc in range(0, ell1 - k + 1):
        qc = qfull[:, :k + lc]
        qh, rh = householder_qr(psi.T @ qc)
        x = solve_upper(rh, qh.T @ yr.T)
        _, s, _ = tsvd(x, k)
        out.append(s)
    return np.array(out)


def minvar_lc(spectra):
    """The minimum-variance l_c (Section 6.6) from the trial spectra lam[l_c, i]:
    s(l_c) = [lam(l_c - 1) / lam(l_c), lam(l_c) / lam(l_c), lam(l_c + 1) / lam(l_c)]
    (the first block absent for l_c = 0), argmin over 0 <= l_c < l_1 of the
    variance of s(l_c) (population variance; ties go to the smaller l_c)."""
    lam = np.asarray(spectra, dtype=np.float64)
    l1 = lam.shape[0] - 1
    best, arg = np.inf, 0
    for lc in range(0, l1):
        parts = [] if lc == 0 else [lam[lc - 1] / lam[lc]]
        parts += [lam[lc] / lam[lc], lam[lc + 1] / lam[lc]]
        v = float(np.var(np.concatenate(parts)))
        if v < best:
            best, arg = v, lc
    return arg


def single_pass_minvar(a, omega, psi, k):
    """Alg. 7 with l_c chosen by the minimum-variance rule; returns (out, l_c)."""
    lc = minvar_lc(minvar_spectra(a, omega, psi, k))
    return single_pass(a, omega, psi, k, l_c=lc), lc
