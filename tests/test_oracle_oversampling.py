"""Pins for the parameter rules of Sections 6.3 (FLAT, DECAY, RAPID) and 6.6 (l_c): hand-evaluated values of the
oversampling formulas, the package's host helpers against the oracle's own
statement of them, and the minimum-variance selection on constructed spectra
whose answer is known."""
import numpy as np
import pytest

from oracle import algorithms as Al
from paper_1804_07531_gb300 import oversampling as O
from paper_1804_07531_gb300 import synth as S

# (T, p): (flat, decay, rapid) (l_1, l_2), evaluated by hand from the formulas
HAND = {
    (30, 5): ((4, 16), (4, 16), (9, 11)),
    (100, 5): ((14, 76), (28, 62), (44, 46)),
    (40, 10): ((4, 16), (3, 17), (9, 11)),
    (16, 5): ((2, 4), (2, 4), (2, 4)),      # the smallest budget, T = 2p + 6
}


@pytest.mark.parametrize("T,p", sorted(HAND))
def test_schemes_match_hand_values(T, p):
    fl, de, ra = HAND[(T, p)]
    assert Al.oversampling_flat(T, p) == fl and O.flat(T, p) == fl
    assert Al.oversampling_decay(T, p) == de and O.decay(T, p) == de
    assert Al.oversampling_rapid(T, p) == ra and O.rapid(T, p) == ra


def test_schemes_agree_and_respect_the_budget_on_a_grid():
    for p in range(1, 21):
        for T in range(2 * p + 6, 2 * p + 200, 7):
            for f_o, f_p in ((Al.oversampling_flat, O.flat), (Al.oversampling_decay, O.decay),
                             (Al.oversampling_rapid, O.rapid)):
                l1, l2 = f_p(T, p)
                assert (l1, l2) == f_o(T, p)
                assert 2 * p + l1 + l2 == T and 0 <= l1 <= l2
    assert O.equal_split(101, 5) == (45, 46)
    assert O.fixed_ratio(45, 0.5) == Al.lc_fixed_ratio(45, 0.5) == 22
    with pytest.raises(ValueError):
        O.flat(2 * 5 + 5, 5)


def test_minvar_picks_the_flattest_neighbourhood():
    # constructed trial spectra: singular values vary wildly except around
    # l_c = 3, where the three neighbouring spectra coincide -> variance 0
    k, l1 = 4, 8
    rng = np.random.default_rng(0)
    lam = 1.0 + rng.uniform(0.0, 2.0, size=(l1 + 1, k))
    lam[2] = lam[3] = lam[4] = np.array([4.0, 3.0, 2.0, 1.0])
    assert Al.minvar_lc(lam) == 3
    # l_c = 0 uses only its upper neighbour
    lam2 = 1.0 + rng.uniform(0.0, 2.0, size=(l1 + 1, k))
    lam2[1] = lam2[0]
    assert Al.minvar_lc(lam2) == 0


def test_minvar_on_a_rapidly_decaying_matrix_prefers_large_lc():
    """Section 6.6: with l_1 = l_2, l_c near l_1 is ill-conditioned (large
    variance) and l_c near 0 loses accuracy; the rule picks an interior
    l_c, and Alg. 7 with it is at least as accurate as with l_c = 0."""
    m, n, k = 300, 200, 5
    a = S.usv(m, n, S.sigma_config("exp25", n), 1, 2) + 1e-6 * S.gaussian(m, n, seed=3)
    l1, l2 = O.equal_split(2 * k + 40, k)
    om = S.gaussian(n, k + l1, seed=4)
    ps = S.gaussian(m, k + l2, seed=5)
    (u, s, v), lc = Al.single_pass_minvar(a, om, ps, k)
    assert 0 <= lc < l1
    e_mv = Al.frob_error(a, u, s, v)
    u0, s0, v0 = Al.single_pass(a, om, ps, k, l_c=0)
    assert e_mv <= 1.0001 * Al.frob_error(a, u0, s0, v0)


def _trial_spectra_by_lstsq(a, om, ps, k):
    """Section 6.5 with each trial l_c written with library routines (test
    only): Q_c = the leading k + l_c left singular vectors of Y_c = A Omega
    (numpy SVD), X = the least-squares solution of (Psi^T Q_c) X = Y_r^T,
    and the leading k singular values of X (numpy SVD)."""
    yc, yr = a @ om, a.T @ ps
    uy = np.linalg.svd(yc, full_matrices=False)[0]
    rows = []
    for lc in range(om.shape[1] - k + 1):
        qc = uy[:, :k + lc]
        x = np.linalg.lstsq(ps.T @ qc, yr.T, rcond=None)[0]
        rows.append(np.linalg.svd(x, compute_uv=False)[:k])
    return np.array(rows)


def _spectra_with_qr_basis(a, om, ps, k):
    """A plausible slip in minvar_spectra: Q_c from the QR of Y_c (its
    columns span the right space only for l_c = l_1) instead of the left
    singular vectors."""
    yc, yr = a @ om, a.T @ ps
    q = np.linalg.qr(yc)[0]
    rows = []
    for lc in range(om.shape[1] - k + 1):
        x = np.linalg.lstsq(ps.T @ q[:, :k + lc], yr.T, rcond=None)[0]
        rows.append(np.linalg.svd(x, compute_uv=False)[:k])
    return np.array(rows)


def test_minvar_spectra_rows_match_library_restatement_and_single_pass():
    """Every row l_c of minvar_spectra is the spectrum Alg. 7 returns with that
    l_c: against numpy's SVD / least squares, against single_pass(l_c), and
    row l_1 against the untruncated single pass; the QR-basis slip fails."""
    m, n, k = 180, 120, 4
    a = S.usv(m, n, S.sigma_config("exp25", n), 11, 12) + 1e-5 * S.gaussian(m, n, seed=13)
    om = S.gaussian(n, k + 6, seed=14)
    ps = S.gaussian(m, k + 9, seed=15)
    spec = Al.minvar_spectra(a, om, ps, k)
    assert spec.shape == (7, k)
    ref = _trial_spectra_by_lstsq(a, om, ps, k)
    assert np.max(np.abs(spec - ref) / ref[:, :1]) < 1e-10
    for lc in range(7):
        s_lc = Al.single_pass(a, om, ps, k, l_c=lc)[1]
        assert np.max(np.abs(spec[lc] - s_lc)) < 1e-10 * s_lc[0]
    s_full = Al.single_pass(a, om, ps, k)[1]
    assert np.max(np.abs(spec[-1] - s_full)) < 1e-10 * s_full[0]
    slip = _spectra_with_qr_basis(a, om, ps, k)
    assert np.max(np.abs(slip[-1] - ref[-1]) / ref[-1, 0]) < 1e-10   # same span at l_c = l_1
    assert np.max(np.abs(slip[:-1] - ref[:-1]) / ref[:-1, :1]) > 1e-4  # differs below l_1
