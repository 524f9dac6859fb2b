"""Pins for the Woolfe single pass (Alg. 8) and the extended SRFT sketch
(Sec. 6.7, bwz2) of the oracle:
  * the DCT-II matrix is scipy's orthonormal DCT (a library routine, test
    only), and Phi = D F P has orthonormal columns;
  * exact recovery: rank(A) <= ell gives [[A]]_k exactly, for both methods;
  * a restatement with library routines (numpy SVD, least squares and
    pseudo-inverses) gives the same singular values, at l_c < l_1 for Alg. 8;
  * planted mistakes (bwz in place of bwz2; Alg. 8 without the truncation of
    Q_r) fail.
"""
import numpy as np
import pytest

from oracle import algorithms as Al
from oracle import extended as Ex
from paper_1804_07531_gb300 import synth as S

sp_fft = pytest.importorskip("scipy.fft")


def _srft_inputs(n, s, seed):
    rng = np.random.default_rng(seed)
    return rng.choice([-1.0, 1.0], size=n), rng.choice(n, size=s, replace=False)


@pytest.mark.parametrize("n", [1, 7, 64, 300])
def test_dct_matrix_is_scipys_orthonormal_dct(n):
    f = Ex.dct_matrix(n)
    ref = sp_fft.dct(np.eye(n), type=2, norm="ortho", axis=0).T
    assert np.max(np.abs(f - ref)) < 1e-13
    assert np.max(np.abs(f.T @ f - np.eye(n))) < 1e-12


def test_srft_has_orthonormal_columns_and_is_a_signed_dct_of_rows():
    n, s = 500, 40
    d, cols = _srft_inputs(n, s, 3)
    phi = Ex.srft(n, d, cols)
    assert np.max(np.abs(phi.T @ phi - np.eye(s))) < 1e-12
    x = S.gaussian(3, n, seed=4)
    ref = sp_fft.dct(x * d[None, :], type=2, norm="ortho", axis=1)[:, cols]
    assert np.max(np.abs(x @ phi - ref)) < 1e-12


def _lowrank(m, n, r, seed):
    sig = np.linspace(2.0, 1.0, r)
    u, v = S.haar(m, r, seed), S.haar(n, r, seed + 1)
    return (u * sig) @ v.T, u, sig, v


@pytest.mark.parametrize("method", ["woolfe", "extended"])
def test_exact_recovery(method):
    m, n, r, k, ell, s = 300, 200, 12, 8, 16, 40
    a, u, sig, v = _lowrank(m, n, r, 5)
    om = S.gaussian(n, ell, seed=6)
    ps = S.gaussian(m, ell if method == "extended" else ell + 8, seed=7)
    if method == "woolfe":
        ug, sg, vg = Ex.woolfe_single_pass(a, om, ps, k)
    else:
        dc, cc = _srft_inputs(n, s, 8)
        dr, cr = _srft_inputs(m, s, 9)
        ug, sg, vg = Ex.extended_single_pass(a, om, ps, Ex.srft(n, dc, cc), Ex.srft(m, dr, cr), k)
    best = (u[:, :k] * sig[:k]) @ v[:, :k].T
    assert np.max(np.abs(sg - sig[:k])) < 1e-12
    assert np.linalg.norm((ug * sg) @ vg.T - best) < 1e-11 * np.linalg.norm(best)


@pytest.mark.parametrize("l_c", [None, 3, 0])
def test_woolfe_matches_library_restatement(l_c):
    m, n, k, ell1, ell2 = 400, 250, 6, 14, 22
    a = S.usv(m, n, S.sigma_config("exp25", n), 11, 12) + 1e-4 * S.gaussian(m, n, seed=13)
    om, ps = S.gaussian(n, ell1, seed=14), S.gaussian(m, ell2, seed=15)
    _, s, _ = Ex.woolfe_single_pass(a, om, ps, k, l_c=l_c)
    kc = ell1 if l_c is None else k + l_c
    yc, yr = a @ om, a.T @ ps
    qc = np.linalg.svd(yc, full_matrices=False)[0][:, :kc]
    qr_ = np.linalg.svd(yr, full_matrices=False)[0][:, :kc]
    x = np.linalg.lstsq(ps.T @ qc, yr.T @ qr_, rcond=None)[0]
    ref = np.linalg.svd(x, compute_uv=False)[:k]
    assert np.max(np.abs(s - ref)) < 1e-10 * ref[0]
    # planted: step 5b dropped (Q_r keeps all ell2 left singular vectors of Y_r)
    qr_all = np.linalg.svd(yr, full_matrices=False)[0]
    bad = np.linalg.svd(np.linalg.lstsq(ps.T @ qc, yr.T @ qr_all, rcond=None)[0], compute_uv=False)[:k]
    assert np.max(np.abs(bad - ref)) > 1e-6 * ref[0]


def test_extended_matches_pinv_restatement_and_differs_from_bwz():
    m, n, k, ell, s = 400, 260, 6, 16, 48
    a = S.usv(m, n, S.sigma_config("inv", n), 21, 22) + 1e-3 * S.gaussian(m, n, seed=23)
    om, ps = S.gaussian(n, ell, seed=24), S.gaussian(m, ell, seed=25)
    dc, cc = _srft_inputs(n, s, 26)
    dr, cr = _srft_inputs(m, s, 27)
    phc, phr = Ex.srft(n, dc, cc), Ex.srft(m, dr, cr)
    ug, sg, vg = Ex.extended_single_pass(a, om, ps, phc, phr, k)
    qc = np.linalg.qr(a @ om)[0]
    qr_ = np.linalg.qr(a.T @ ps)[0]
    uc, tc = np.linalg.qr(phr.T @ qc)
    ur, tr = np.linalg.qr(phc.T @ qr_)
    z = phr.T @ a @ phc
    core = np.linalg.pinv(tc) @ uc.T @ z @ ur @ np.linalg.pinv(tr.T)
    ref = np.linalg.svd(core, compute_uv=False)[:k]
    assert np.max(np.abs(sg - ref)) < 1e-10 * ref[0]
    # bwz (truncate before applying the pseudo-inverses) is a different approximation
    w, sw, wt = np.linalg.svd(uc.T @ z @ ur)
    bwz = np.linalg.pinv(tc) @ (w[:, :k] * sw[:k]) @ wt[:k] @ np.linalg.pinv(tr.T)
    e2 = np.linalg.norm(a - (ug * sg) @ vg.T)
    e1 = np.linalg.norm(a - qc @ bwz @ qr_.T)
    assert abs(e1 - e2) > 1e-6 * e2
