"""Alg. 2 on a matrix whose rows are split over G ranks, FP64.

Test infrastructure only (see the package docstring).  Rank g holds A_g, its
block of rows of A (the blocks in rank order make A), and the common random
start Omega (an input, never drawn here).  `allreduce(x)` returns the sum of
the array x over the ranks; the same function runs every rank's steps, either
in one process (ranks simulated in turn, see `simulate`) or in G processes
whose allreduce is a collective.

The views of Alg. 2 split by rows as follows:
  * A Q_r: rank g forms its rows A_g Q_r; nothing is exchanged;
  * A^T Q_c = sum_g A_g^T Q_c,g: one sum of an n x ell array;
  * qr of the row-split Y: the Gram Y^T Y = sum_g Y_g^T Y_g (one sum of an
    ell x ell array), its Cholesky factor R (Y^T Y = R^T R), Q_g = Y_g R^-1;
    taken twice (CholeskyQR2), R = R_2 R_1;
  * the core SVD and the n-side factors are the same on every rank;
  * the sign of each pair (u_i, v_i) follows the largest-magnitude entry of
    u_i over all rows of U (the lowest row on ties): the rule of
    linalg.fix_signs applied to the U that the blocks make.
"""
from __future__ import annotations

import numpy as np

from .linalg import cholesky_upper, householder_qr, solve_upper_right, tsvd

__all__ = ["chol_qr2", "subspace_iteration", "simulate"]


def chol_qr2(y_g, allreduce):
    """Thin QR of the row-split Y (this rank's rows y_g): (Q_g, R), R upper
    triangular with a positive diagonal, the same on every rank."""
    q = np.asarray(y_g, dtype=np.float64)
    r = np.eye(q.shape[1])
    for _ in range(2):
        rp = cholesky_upper(allreduce(q.T @ q))
        q = solve_upper_right(q, rp)
        r = rp @ r
    return q, r


def _peak_signs(u_g, rank, world, allreduce):
    """+-1 per column: the sign of the largest-magnitude entry of u_i over
    all ranks (lowest rank, then lowest row within it, on ties)."""
    k = u_g.shape[1]
    peaks = np.zeros((world, k))
    if u_g.shape[0] > 0:
        idx = np.argmax(np.abs(u_g), axis=0)
        peaks[rank] = u_g[idx, np.arange(k)]
    peaks = allreduce(peaks)
    pick = np.argmax(np.abs(peaks), axis=0)        # first maximum: the lowest rank
    sg = np.sign(peaks[pick, np.arange(k)])
    sg[sg == 0] = 1.0
    return sg


def subspace_iteration(a_g, omega, k, v, rank, world, allreduce):
    """Alg. 2 with v >= 2 views on the row-split A: (U_g, s, V), U_g this
    rank's rows of U.  Odd j: [Q_c, R_c] = qr(A Q_r); even j: [Q_r, R_r] =
    qr(A^T Q_c); v even: [V^, L, U^] = tsvd(R_r, k); v odd: [U^, L, V^] =
    tsvd(R_c, k); U = Q_c U^, V = Q_r V^."""
    if v < 2:
        raise ValueError("Alg. 2 needs v >= 2")
    a_g = np.asarray(a_g, dtype=np.float64)
    qr_ = np.asarray(omega, dtype=np.float64)
    qc = rc = rr = None
    for j in range(1, v + 1):
        if j % 2 == 1:
            qc, rc = chol_qr2(a_g @ qr_, allreduce)
        else:
            qr_, rr = householder_qr(allreduce(a_g.T @ qc))
    if v % 2 == 0:
        vh, s, uh = tsvd(rr, k)
    else:
        uh, s, vh = tsvd(rc, k)
    u_g, vv = qc @ uh, qr_ @ vh
    sg = _peak_signs(u_g, rank, world, allreduce)
    return u_g * sg[None, :], s, vv * sg[None, :]


def simulate(blocks, omega, k, v):
    """Every rank of subspace_iteration in one process: the ranks run in
    lock step (one thread each) and each allreduce returns the sum of the
    ranks' arrays.  Returns [(U_g, s, V) for each rank]."""
    import threading

    world = len(blocks)
    barrier = threading.Barrier(world)
    slots = [None] * world
    results = [None] * world
    errors = []

    def run(g):
        def allreduce(x):
            slots[g] = np.array(x, dtype=np.float64)
            barrier.wait()
            total = sum(slots[h] for h in range(world))
            barrier.wait()
            return total
        try:
            results[g] = subspace_iteration(blocks[g], omega, k, v, g, world, allreduce)
        except Exception as e:  # pragma: no cover - surfaced below
            errors.append(e)
            barrier.abort()

    threads = [threading.Thread(target=run, args=(g,)) for g in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return results
