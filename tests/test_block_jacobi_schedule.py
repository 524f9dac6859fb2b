"""Host model of the column-block cluster Jacobi's schedule (csrc/jacobi_block.cu).

The kernel splits the columns into 2P blocks of b, two per CTA, and runs a
sweep as 2P - 1 block rounds in circle-method order; the first block round
pairs all 2b local columns (2b - 1 local rounds), the others pair only across
the two blocks (b local rounds), and between block rounds every block moves
to its next holder.  These tests restate that schedule in Python, with the
kernel's index formulas, and check what its correctness rests on:
  * every pair of columns is rotated exactly once per sweep;
  * the rounds' pairs are disjoint (they run concurrently);
  * the hand-off between block rounds is a bijection of (CTA, slot)
    positions, and each CTA receives exactly the bytes its mbarrier expects;
  * the schedule, with the kernel's rotation formula and the V <- V J update
    per block round, converges to the SVD (FP64, small matrices).
"""

import numpy as np
import pytest


def round_pair(pi, rnd, np_):
    """Pair pi of round rnd in the circle method over np_ positions (the
    kernel's round_pair)."""
    ia = pi - 1 + rnd
    if ia >= np_ - 1:
        ia -= np_ - 1
    ib = np_ - 2 - pi + rnd
    if ib >= np_ - 1:
        ib -= np_ - 1
    a = 0 if pi == 0 else 1 + ia
    b = 1 + ib
    return min(a, b), max(a, b)


def holder(k, r, NB):
    for pi in range(NB // 2):
        p, q = round_pair(pi, r, NB)
        if p == k or q == k:
            return pi, int(q == k)
    raise AssertionError("block without holder")


def sweep_pairs(P, b):
    """The (global column) pairs of one sweep, round by round."""
    NB = 2 * P
    rounds = []
    for r in range(NB - 1):
        blocks = [round_pair(pi, r, NB) for pi in range(P)]
        if r == 0:
            for rr in range(2 * b - 1):
                rnd = []
                for (k0, k1) in blocks:
                    cols = [k0 * b + i for i in range(b)] + [k1 * b + i for i in range(b)]
                    for w in range(b):
                        p, q = round_pair(w, rr, 2 * b)
                        rnd.append((cols[p], cols[q]))
                rounds.append(rnd)
        else:
            for s in range(b):
                rounds.append([(k0 * b + w, k1 * b + (w + s) % b) for (k0, k1) in blocks for w in range(b)])
    return rounds


@pytest.mark.parametrize("P", [1, 2, 3, 4, 8, 16])
@pytest.mark.parametrize("b", [1, 2, 5, 13, 16])
def test_every_pair_once_per_sweep(P, b):
    rounds = sweep_pairs(P, b)
    n = 2 * P * b
    seen = {}
    for rnd in rounds:
        cols = [c for pair in rnd for c in pair]
        assert len(cols) == len(set(cols)), "pairs of a round overlap"
        for p, q in rnd:
            key = (min(p, q), max(p, q))
            seen[key] = seen.get(key, 0) + 1
    assert len(seen) == n * (n - 1) // 2
    assert set(seen.values()) == {1}
    # local rounds per sweep: (2b - 1) + (2P - 2) b = n - 1, as a cyclic sweep
    assert len(rounds) == n - 1


@pytest.mark.parametrize("P", [2, 3, 4, 8, 16])
def test_handoff_is_a_bijection_and_bytes_match(P):
    NB = 2 * P
    for r in range(NB - 1):
        rn = 0 if r == NB - 2 else r + 1
        dest = {}
        recv_remote = [0] * P
        for pi in range(P):
            c = round_pair(pi, r, NB)
            for s in range(2):
                hc, hs = holder(c[s], rn, NB)
                assert round_pair(hc, rn, NB)[hs] == c[s]
                assert (hc, hs) not in dest
                dest[(hc, hs)] = c[s]
                if hc != pi:
                    recv_remote[hc] += 1
        assert len(dest) == NB
        # what each CTA expects: its next blocks that another CTA holds now
        for pi in range(P):
            nxt = round_pair(pi, rn, NB)
            expect = sum(1 for s in range(2) if holder(nxt[s], r, NB)[0] != pi)
            assert expect == recv_remote[pi]


def block_jacobi_svd(M, P, tol=50 * np.finfo(float).eps, max_sweeps=40):
    """The kernel's schedule and arithmetic in FP64: rotations of W's column
    pairs (t from d = beta - alpha and 2 gamma, c and s, as in the kernel), accumulated per block
    round into J, and V <- V J at the end of each block round."""
    n = M.shape[1]
    NB = 2 * P
    b = -(-n // NB)
    N = NB * b
    W = np.zeros((M.shape[0], N))
    W[:, :n] = M
    V = np.eye(N)
    for sweep in range(max_sweeps):
        rotated = 0
        for r in range(NB - 1):
            blocks = [round_pair(pi, r, NB) for pi in range(P)]
            Js = {blk: np.eye(2 * b) for blk in blocks}
            local = []
            if r == 0:
                for rr in range(2 * b - 1):
                    local.append([round_pair(w, rr, 2 * b) for w in range(b)])
            else:
                for s in range(b):
                    local.append([(w, b + (w + s) % b) for w in range(b)])
            for rnd in local:
                for (k0, k1) in blocks:
                    cols = [k0 * b + i for i in range(b)] + [k1 * b + i for i in range(b)]
                    J = Js[(k0, k1)]
                    for p, q in rnd:
                        x, y = W[:, cols[p]].copy(), W[:, cols[q]].copy()
                        al, be, ga = x @ x, y @ y, x @ y
                        if not (al > 0 and be > 0 and ga * ga > tol * tol * al * be):
                            continue
                        d, g2 = be - al, 2 * ga
                        t = np.copysign(1.0, d) * g2 / (abs(d) + np.sqrt(d * d + g2 * g2))
                        c = 1 / np.sqrt(1 + t * t)
                        s_ = c * t
                        W[:, cols[p]], W[:, cols[q]] = c * x - s_ * y, s_ * x + c * y
                        jp, jq = J[:, p].copy(), J[:, q].copy()
                        J[:, p], J[:, q] = c * jp - s_ * jq, s_ * jp + c * jq
                        rotated += 1
            for (k0, k1), J in Js.items():
                cols = [k0 * b + i for i in range(b)] + [k1 * b + i for i in range(b)]
                V[:, cols] = V[:, cols] @ J
        if rotated == 0:
            break
    sig = np.linalg.norm(W[:, :n], axis=0) / np.linalg.norm(V[:n, :n], axis=0)
    order = np.argsort(-sig, kind="stable")
    return sig[order], W[:, :n][:, order] / np.linalg.norm(W[:, :n][:, order], axis=0), V[:n, :n][:, order], sweep


@pytest.mark.parametrize("n,P", [(7, 1), (24, 2), (30, 3), (33, 4)])
def test_schedule_converges_to_the_svd(n, P):
    rng = np.random.default_rng(n * 10 + P)
    # a graded upper-triangular core, like R^T of the schedules
    M = np.triu(rng.standard_normal((n, n))) * (np.arange(1, n + 1) ** -1.5)[:, None] + np.diag(np.linspace(2, 1, n))
    M = M.T
    s, U, V, sweeps = block_jacobi_svd(M, P)
    assert sweeps < 40
    s_ref = np.linalg.svd(M, compute_uv=False)
    assert np.abs(s - s_ref).max() <= 1e-13 * s_ref[0]
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-13
    assert np.abs(M @ V - U * s).max() <= 1e-13 * s_ref[0]
