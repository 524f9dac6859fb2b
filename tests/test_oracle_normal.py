"""Pins for the normal-matrix TEVDs of Section 4.2.3 (Algs. 3, 4, 5).

They are pinned to other parts of the oracle and to exact results, not to
themselves:
  * Alg. 4 (Nystrom) with v views gives the eigenpairs sigma_i^2, v_i that
    Alg. 2 with v views gives J (the paper: the prolonged sketch is the
    accurate way of using Alg. 2 on J^T J); the shift nu enters only as
    O(nu);
  * Alg. 5 (pinched) with v views equals Alg. 2 with v views on J (v odd)
    or on J^T (v even);
  * exact recovery: rank(J) <= ell gives the exact leading eigenpairs of
    J^T J (numpy's eigh of J^T J as the reference, a library routine);
  * Alg. 3 returns orthonormal bases of the spaces Alg. 2 reaches;
  * a planted mistake (C_L from the Gram of Y_r instead of Q_r^T Y_r) fails.
"""
import numpy as np
import pytest

from oracle import algorithms as Al
from oracle import normal as Nm
from paper_1804_07531_gb300 import synth as S


def _j(m, n, spectrum, seed):
    return S.usv(m, n, S.sigma_config(spectrum, min(m, n)), seed, seed + 1)


def _subspace_dist(v1, v2):
    return np.linalg.norm(v1 @ v1.T - v2 @ v2.T, 2)


@pytest.mark.parametrize("v", [2, 3, 4, 5])
def test_nystrom_equals_alg2_with_v_views(v):
    m, n, k, ell = 300, 200, 6, 12
    j = _j(m, n, "exp25", 5)
    op = Nm.MatrixOperator(j)
    om = S.gaussian(n if v % 2 == 0 else m, ell, seed=7)
    vk, lam2 = Nm.nystrom_tevd(op, om, k, v)
    if v % 2 == 0:
        _, s, vv = Al.gen_subspace_iteration(j, om, k, v)
    else:       # Q_r from v - 2 views of J^T, then two views: Alg. 2 on J^T, U side
        vv, s, _ = Al.gen_subspace_iteration(j.T, om, k, v)
    assert np.max(np.abs(lam2 - s ** 2)) < 1e-12 * s[0] ** 2
    assert _subspace_dist(vk, vv) < 1e-9


@pytest.mark.parametrize("v", [2, 3, 4, 5])
def test_pinched_equals_alg2_on_j_or_its_transpose(v):
    m, n, k, ell = 300, 200, 6, 12
    j = _j(m, n, "exp25", 9)
    op = Nm.MatrixOperator(j)
    om = S.gaussian(m if v % 2 == 0 else n, ell, seed=11)
    vk, lam2 = Nm.pinched_tevd(op, om, k, v)
    if v % 2 == 1:
        _, s, vv = Al.gen_subspace_iteration(j, om, k, v)
    else:
        vv, s, _ = Al.gen_subspace_iteration(j.T, om, k, v)
    assert np.max(np.abs(lam2 - s ** 2)) < 1e-12 * s[0] ** 2
    assert _subspace_dist(vk, vv) < 1e-9


@pytest.mark.parametrize("alg", ["nystrom", "pinched"])
@pytest.mark.parametrize("v", [2, 3, 4])
def test_exact_recovery_of_the_normal_matrix(alg, v):
    m, n, r, k, ell = 250, 180, 10, 6, 12
    sig = np.linspace(3.0, 1.0, r)
    u = S.haar(m, r, 21)
    w = S.haar(n, r, 22)
    j = (u * sig) @ w.T
    op = Nm.MatrixOperator(j)
    rows = (n if v % 2 == 0 else m) if alg == "nystrom" else (m if v % 2 == 0 else n)
    om = S.gaussian(rows, ell, seed=23)
    f = Nm.nystrom_tevd if alg == "nystrom" else Nm.pinched_tevd
    vk, lam2 = f(op, om, k, v)
    ev, evec = np.linalg.eigh(j.T @ j)
    ev, evec = ev[::-1][:k], evec[:, ::-1][:, :k]
    assert np.max(np.abs(lam2 - ev)) < 1e-10 * ev[0]
    assert _subspace_dist(vk, evec) < 1e-8
    assert np.max(np.abs(vk.T @ vk - np.eye(k))) < 1e-12


def test_qrqc_bases_are_orthonormal_and_match_alg2():
    m, n, ell = 200, 150, 10
    j = _j(m, n, "inv", 31)
    op = Nm.MatrixOperator(j)
    om = S.gaussian(n, ell, seed=32)
    for v in (1, 2, 3, 4):
        q = Nm.qrqc(op, om, v)
        assert np.max(np.abs(q.T @ q - np.eye(ell))) < 1e-12
        _, st = Al.gen_subspace_iteration(j, om, 2, max(v, 2), return_state=True)
        ref = st["qc"] if v % 2 == 1 else st["qr"]
        if v >= 2:
            assert _subspace_dist(q, ref) < 1e-9


def test_planted_mistake_in_nystrom_is_caught():
    m, n, k, ell, v = 300, 200, 6, 12, 4
    j = _j(m, n, "exp25", 41)
    op = Nm.MatrixOperator(j)
    om = S.gaussian(n, ell, seed=43)
    good, lam_good = Nm.nystrom_tevd(op, om, k, v)
    _, s, _ = Al.gen_subspace_iteration(j, om, k, v)
    assert np.max(np.abs(lam_good - s ** 2)) < 1e-12 * s[0] ** 2
    # the slip: C_L from the Gram Y_r^T Y_r (a plausible confusion) instead of Q_r^T Y_r
    qr_ = Nm.qrqc(op, om, v - 2)
    yr = op.apply_t(op.apply(qr_))
    cu = np.linalg.cholesky(yr.T @ yr).T
    f = np.linalg.solve(cu.T, yr.T)
    lam_bad = np.linalg.svd(f, compute_uv=False)[:k] ** 2
    assert np.max(np.abs(lam_bad - s ** 2)) > 1e-3 * s[0] ** 2
