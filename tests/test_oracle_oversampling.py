"""Pins for the Section 6.5 parameter rules: hand-evaluated values of the
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
    """Section 6.5: with l_1 = l_2, l_c near l_1 is ill-conditioned (large
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
