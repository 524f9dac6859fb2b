"""Pins for the oracle's algorithms (CPU only).

What fixes the result independently of the oracle's own code:
  * exact recovery: rank(A) = r with k <= r <= ell gives sigma^ = sigma and
    U_k S_k V_k^T = [[A]]_k for every algorithm and every v;
  * brute force: ell = n (square invertible Omega) gives the full exact SVD;
  * the paper's algebraic equivalences: Alg. 2 with even v is Alg. 1
    (Section 4), Alg. 9 equals Alg. 2 for v < 4 (Section 7.2), the
    row-streamed block Krylov method with v views equals Alg. 9 with 2v-1
    views (Section 7.3), the row-streamed one-pass QB equals the 2-view
    method (Section 6.8);
  * the 1-view baseline of Section 6.2 written with numpy's least squares;
  * Theorems 3.1 and 4.1 (mean spectral error below the bound) and the
    qualitative claims of Section 8 (error falls with v; block Krylov beats
    subspace iteration at equal v and ell);
  * Eckart-Young: no rank-k output beats the optimal tail.
A planted-mistake test shows these pins catch a plausible error.
"""
import numpy as np
import pytest

from oracle import algorithms as Al
from oracle import linalg as L
from paper_1804_07531_gb300 import synth as S


def _lowrank(m, n, r, seed):
    sig = np.linspace(3.0, 0.5, r)
    return S.usv(m, n, sig, seed, seed + 1), sig


def _recon(u, s, v):
    return (u * s[None, :]) @ v.T


def _best_k(a, k):
    uu, ss, vv = np.linalg.svd(a, full_matrices=False)
    return (uu[:, :k] * ss[:k]) @ vv[:k]


@pytest.mark.parametrize("v", [2, 3, 4, 5])
def test_exact_recovery_subspace_and_krylov(v):
    m, n, r, k, ell = 140, 100, 25, 20, 30
    a, sig = _lowrank(m, n, r, seed=100 + v)
    om = S.gaussian(n, ell, seed=7 + v)
    best = _best_k(a, k)
    fns = [Al.gen_subspace_iteration, Al.block_krylov]
    if v <= 4:      # the row-streamed Krylov basis holds (2v-1)//2 * ell <= n columns
        fns.append(Al.rowwise_block_krylov)
    for fn in fns:
        u, s, vv = fn(a, om, k, v)
        assert np.abs(s - sig[:k]).max() < 1e-11, fn.__name__
        assert np.abs(_recon(u, s, vv) - best).max() < 1e-11, fn.__name__
        assert np.abs(u.T @ u - np.eye(k)).max() < 1e-12
        assert np.abs(vv.T @ vv - np.eye(k)).max() < 1e-12


def test_exact_recovery_single_pass_and_rowwise_qb():
    m, n, r, k = 70, 50, 25, 20
    a, sig = _lowrank(m, n, r, seed=3)
    om = S.gaussian(n, 30, seed=4)
    psi = S.gaussian(m, 40, seed=5)
    best = _best_k(a, k)
    for lc in (None, 5):            # exact once k + l_c >= rank(A)
        u, s, vv = Al.single_pass(a, om, psi, k, l_c=lc)
        assert np.abs(s - sig[:k]).max() < 1e-10, lc
        assert np.abs(_recon(u, s, vv) - best).max() < 1e-10, lc
    a20, sig20 = _lowrank(m, n, k, seed=9)
    u, s, vv = Al.single_pass(a20, om, psi, k, l_c=0)
    assert np.abs(s - sig20).max() < 1e-10
    assert np.abs(_recon(u, s, vv) - a20).max() < 1e-10
    # Section 6.8 needs an invertible R_c: rank(A) = ell keeps Y_c full rank.
    a30, sig30 = _lowrank(m, n, 30, seed=10)
    u, s, vv = Al.rowwise_qb_svd(a30, om, k)
    assert np.abs(s - sig30[:k]).max() < 1e-10
    assert np.abs(_recon(u, s, vv) - _best_k(a30, k)).max() < 1e-10


@pytest.mark.parametrize("v", [2, 3])
def test_brute_force_full_svd_when_ell_equals_n(v):
    a = S.gaussian(12, 8, seed=21)
    om = S.gaussian(8, 8, seed=22)
    u, s, vv = Al.gen_subspace_iteration(a, om, 8, v)
    uu, ss, vt = np.linalg.svd(a, full_matrices=False)
    assert np.allclose(s, ss, atol=1e-12)
    assert np.allclose(_recon(u, s, vv), a, atol=1e-12)
    assert np.allclose(np.abs(u.T @ uu), np.eye(8), atol=1e-9)


@pytest.mark.parametrize("v", [2, 4, 6])
def test_alg2_even_views_is_alg1(v):
    a = S.usv(90, 60, S.sigma_config("inv", 60), 1, 2)
    om = S.gaussian(60, 12, seed=3)
    u1, s1, v1 = Al.subspace_iteration(a, om, 8, (v - 2) // 2)
    u2, s2, v2 = Al.gen_subspace_iteration(a, om, 8, v)
    assert np.allclose(s1, s2, rtol=1e-12, atol=0)
    assert np.allclose(u1, u2, atol=1e-9) and np.allclose(v1, v2, atol=1e-9)


@pytest.mark.parametrize("v", [2, 3])
def test_block_krylov_equals_subspace_for_v_below_4(v):
    a = S.usv(90, 60, S.sigma_config("inv", 60), 4, 5)
    om = S.gaussian(60, 12, seed=6)
    _, s1, _ = Al.gen_subspace_iteration(a, om, 8, v)
    _, s2, _ = Al.block_krylov(a, om, 8, v)
    assert np.allclose(s1, s2, rtol=1e-11, atol=0)


@pytest.mark.parametrize("v", [2, 3, 4])
def test_rowwise_krylov_equals_alg9_with_2v_minus_1_views(v):
    a = S.usv(120, 80, S.sigma_config("pow15", 80), 8, 9)
    om = S.gaussian(80, 10, seed=10)
    u1, s1, v1 = Al.rowwise_block_krylov(a, om, 6, v)
    u2, s2, v2 = Al.block_krylov(a, om, 6, 2 * v - 1)
    assert np.allclose(s1, s2, rtol=1e-10, atol=0)
    assert np.abs(_recon(u1, s1, v1) - _recon(u2, s2, v2)).max() < 1e-10


def test_rowwise_qb_equals_two_view_method():
    a = S.usv(100, 70, S.sigma_config("inv", 70), 11, 12)
    om = S.gaussian(70, 15, seed=13)
    _, s1, _ = Al.rowwise_qb_svd(a, om, 10)
    _, s2, _ = Al.gen_subspace_iteration(a, om, 10, 2)
    assert np.allclose(s1, s2, rtol=1e-11, atol=0)


def test_single_pass_baseline_matches_least_squares_form():
    """Section 6.2 steps 1-5 written with numpy lstsq/svd give Alg. 7 with l_c = l_1."""
    m, n, k = 120, 80, 8
    a = S.usv(m, n, S.sigma_config("exp25", 80), 14, 15) + 1e-3 * S.gaussian(m, n, seed=16)
    om = S.gaussian(n, 14, seed=17)
    psi = S.gaussian(m, 25, seed=18)
    yc, yr = a @ om, a.T @ psi
    qc = np.linalg.qr(yc)[0]
    x = np.linalg.lstsq(psi.T @ qc, yr.T, rcond=None)[0]
    uu, ss, vt = np.linalg.svd(x, full_matrices=False)
    ref = (qc @ uu[:, :k] * ss[:k]) @ vt[:k]
    u, s, vv = Al.single_pass(a, om, psi, k)
    assert np.allclose(s, ss[:k], rtol=1e-10, atol=0)
    assert np.abs(_recon(u, s, vv) - ref).max() < 1e-10


def test_single_pass_truncation_lc_uses_leading_left_vectors():
    """With l_c < l_1, Q_c spans the leading k + l_c left singular vectors of Y_c."""
    m, n, k = 90, 60, 6
    a = S.usv(m, n, S.sigma_config("inv", 60), 19, 20)
    om = S.gaussian(n, 16, seed=21)
    psi = S.gaussian(m, 20, seed=22)
    _, st = Al.single_pass(a, om, psi, k, l_c=4, return_state=True)
    uy = np.linalg.svd(a @ om, full_matrices=False)[0][:, : k + 4]
    assert np.abs(st["qc"] @ st["qc"].T - uy @ uy.T).max() < 1e-10


def _mean_spec_err(a, fn, seeds):
    out = []
    for sd in seeds:
        out.append(fn(sd))
    return float(np.mean(out))


def test_theorem_bounds_hold_on_average():
    """Theorems 3.1/4.1 and their v-parity forms (Section 4.2.2)."""
    n = 150
    sig = S.sigma_config("inv", n)
    a = S.usv(n, n, sig, 30, 31)
    p, l = 6, 4
    for v in (2, 3, 4, 5):
        def qc_err(sd):
            om = S.gaussian(n, p + l, seed=1000 + sd)
            _, st = Al.gen_subspace_iteration(a, om, p, v, return_state=True)
            qc = st["qc"]
            return np.linalg.norm(a - qc @ (qc.T @ a), 2)

        def qr_err(sd):
            om = S.gaussian(n, p + l, seed=2000 + sd)
            _, st = Al.gen_subspace_iteration(a, om, p, v, return_state=True)
            q = st["qr"]
            return np.linalg.norm(a - (a @ q) @ q.T, 2)

        # Q_c: exponent v-1 (even v) / v (odd v); Q_r: v (even) / v-1 (odd).
        ec = v - 1 if v % 2 == 0 else v
        er = v if v % 2 == 0 else v - 1
        bc = Al.thm31_bound(sig, p, l, (ec - 1) // 2)
        assert _mean_spec_err(a, qc_err, range(20)) <= bc
        br = Al.thm41_bound(sig, p, l, er // 2)
        assert _mean_spec_err(a, qr_err, range(20)) <= br


def test_error_decays_with_views_and_krylov_beats_subspace():
    """Section 8.3: error falls as v grows; Alg. 9 is more accurate at equal v, ell."""
    n, k, ell = 200, 10, 20
    a = S.lowrank_noise(n=n, R=10, eta=1.0, seed=3)
    tail = np.sqrt(np.sum(np.linalg.svd(a, compute_uv=False)[k:] ** 2))
    errs = {}
    for fn in (Al.gen_subspace_iteration, Al.block_krylov):
        errs[fn.__name__] = []
        for v in (2, 3, 4, 5, 6):
            e = []
            for sd in range(6):
                om = S.gaussian(n, ell, seed=500 + sd)
                u, s, vv = fn(a, om, k, v)
                e.append(Al.rel_frob_error(a, u, s, vv, tail))
            errs[fn.__name__].append(np.mean(e))
    g = errs["gen_subspace_iteration"]
    assert all(g[i + 1] < g[i] for i in range(len(g) - 1))
    b = errs["block_krylov"]
    assert all(b[i] <= g[i] * (1 + 1e-9) for i in range(len(g)))
    assert b[-1] < g[-1]


def test_eckart_young_lower_bound_and_convergence_to_tail():
    n, k = 120, 8
    sig = S.sigma_config("inv", n)
    a = S.usv(n, n, sig, 40, 41)
    tail = np.sqrt(np.sum(sig[k:] ** 2))
    om = S.gaussian(n, 12, seed=42)
    prev = np.inf
    for v in (2, 4, 8):
        u, s, vv = Al.gen_subspace_iteration(a, om, k, v)
        e = Al.frob_error(a, u, s, vv)
        assert e >= tail * (1 - 1e-12)
        assert e < prev
        prev = e
    assert prev / tail - 1 < 1e-3


def test_view_count_formula():
    """Section 7.2: Alg. 9 multiplies A by (v + floor(v/2) - 1)(p+l) vectors.

    v-1 inner views of ell columns each, then one view with the whole Krylov
    basis (floor(v/2) blocks of ell columns)."""
    a = S.gaussian(40, 30, seed=1)
    om = S.gaussian(30, 5, seed=2)
    for v in (2, 3, 4, 5, 6):
        _, st = Al.block_krylov(a, om, 3, v, return_state=True)
        assert (v - 1) * 5 + st["k"].shape[1] == Al.view_count_block_krylov(v, 5), v


def test_planted_mistake_is_caught():
    """A plausible slip (tsvd of R_r read with U and V swapped) fails exact recovery."""
    m, n, r, k, ell = 60, 40, 20, 15, 24
    a, sig = _lowrank(m, n, r, seed=55)
    om = S.gaussian(n, ell, seed=56)

    def mutated(a, om, k, v):
        qr_ = om
        for j in range(1, v + 1):
            if j % 2:
                qc, rc = L.householder_qr(a @ qr_)
            else:
                qr_, rr = L.householder_qr(a.T @ qc)
        uh, s, vh = L.tsvd(rr, k)       # mistake: R_r = V^ L U^T, not U^ L V^T
        return qc @ uh, s, qr_ @ vh

    u, s, vv = mutated(a, om, k, 2)
    assert np.abs(s - sig[:k]).max() < 1e-10          # sigma alone misses it ...
    assert np.abs(_recon(u, s, vv) - _best_k(a, k)).max() > 1e-3   # ... the recovery pin does not
