"""Pins for the oracle's reverse pass (CPU only).

The reverse pass of Alg. 2's top-k singular-value sum is checked against
central finite differences along seeded directions (FP64) and, for a
well-separated spectrum, against the exact gradient U_k V_k^T of the sum of
the top-k singular values of A (valid when sigma_k > sigma_{k+1}).
"""
import numpy as np
import pytest

from oracle import grad as G
from oracle import linalg as L
from paper_1804_07531_gb300 import synth as S


def _gap_matrix(m, n, seed):
    s = S.sigma_config("gap32", min(m, n))
    return S.usv(m, n, s, seed, seed + 1), s


def test_qr_backward_matches_finite_differences():
    y = S.gaussian(30, 6, seed=1)
    qb = S.gaussian(30, 6, seed=2)
    rb = np.triu(S.gaussian(6, 6, seed=3))

    def f(yy):
        q, r = L.householder_qr(yy)
        return float(np.sum(q * qb) + np.sum(r * rb))

    q, r = L.householder_qr(y)
    g = G.qr_backward(q, r, qb, rb)
    for sd in range(5):
        e = S.gaussian(30, 6, seed=10 + sd)
        h = 1e-6
        fd = (f(y + h * e) - f(y - h * e)) / (2 * h)
        assert abs(fd - np.sum(g * e)) < 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("v", [2, 3, 4])
def test_grad_matches_finite_differences(v):
    m, n, k, ell = 60, 45, 6, 10
    a, _ = _gap_matrix(m, n, 5)
    a = a + 1e-3 * S.gaussian(m, n, seed=6)
    om = S.gaussian(n, ell, seed=7)
    g = G.grad_topk_sigma_sum(a, om, k, v)
    h = 1e-6 * np.abs(a).max()
    for sd in range(16):
        e = S.gaussian(m, n, seed=100 + sd)
        fd = (G.topk_sigma_sum(a + h * e, om, k, v) - G.topk_sigma_sum(a - h * e, om, k, v)) / (2 * h)
        an = float(np.sum(g * e))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (sd, fd, an)


def test_grad_approaches_exact_top_k_gradient():
    """With the gap after j = 32, sum_{i<=32} sigma_i has gradient U_32 V_32^T."""
    m, n, k = 200, 120, 32
    s = S.sigma_config("gap32", n)
    u = S.haar(m, n, 51)
    vv = S.haar(n, n, 52)
    a = (u * s) @ vv.T
    om = S.gaussian(n, 40, seed=53)
    g = G.grad_topk_sigma_sum(a, om, k, 6)
    exact = u[:, :k] @ vv[:, :k].T
    assert np.linalg.norm(g - exact) / np.linalg.norm(exact) < 1e-3


def test_svd_backward_matches_finite_differences():
    n = 8
    r = np.triu(S.gaussian(n, n, seed=61)) + np.diag(np.arange(n, 0, -1.0))
    wb, sb, zb = S.gaussian(n, n, seed=62), S.gaussian(n, 1, seed=63)[:, 0], S.gaussian(n, n, seed=64)

    def f(rr):
        w, s, z = L.jacobi_svd(rr)
        # the sign of each singular pair is fixed by w's largest entry, as the library does
        idx = np.argmax(np.abs(w), axis=0)
        d = np.sign(w[idx, np.arange(n)])
        return float(np.sum(w * d * wb) + s @ sb + np.sum(z * d * zb))

    w, s, z = L.jacobi_svd(r)
    idx = np.argmax(np.abs(w), axis=0)
    d = np.sign(w[idx, np.arange(n)])
    g = G.svd_backward(w, s, z, wb * d, sb, zb * d)
    for sd in range(6):
        e = S.gaussian(n, n, seed=70 + sd)
        h = 1e-6
        fd = (f(r + h * e) - f(r - h * e)) / (2 * h)
        assert abs(fd - np.sum(g * e)) < 1e-6 * max(1.0, abs(fd)), (sd, fd, np.sum(g * e))


@pytest.mark.parametrize("v", [2, 3, 4])
def test_grad_through_u_s_v_matches_finite_differences(v):
    """L = <Ub, U> + <Sb, S> + <Vb, V> of Alg. 2's outputs: the reverse pass
    against central differences along 12 seeded directions."""
    m, n, k, ell = 60, 45, 5, 10
    a, _ = _gap_matrix(m, n, 81)
    a = a + 1e-3 * S.gaussian(m, n, seed=82)
    om = S.gaussian(n, ell, seed=83)
    ub, sb, vb = S.gaussian(m, k, seed=84), S.gaussian(k, 1, seed=85)[:, 0], S.gaussian(n, k, seed=86)

    def f(aa):
        u, s, vv = G.lowrank_outputs(aa, om, k, v)
        return float(np.sum(u * ub) + s @ sb + np.sum(vv * vb))

    g = G.grad_lowrank(a, om, k, v, ub, sb, vb)
    h = 1e-6 * np.abs(a).max()
    for sd in range(12):
        e = S.gaussian(m, n, seed=200 + sd)
        fd = (f(a + h * e) - f(a - h * e)) / (2 * h)
        an = float(np.sum(g * e))
        assert abs(fd - an) <= 2e-6 * max(1.0, abs(an)), (sd, fd, an)
    # with Ub = Vb = 0 it is the singular-value gradient of before
    g0 = G.grad_lowrank(a, om, k, v, None, np.ones(k), None)
    assert np.max(np.abs(g0 - G.grad_topk_sigma_sum(a, om, k, v))) < 1e-12 * np.abs(g0).max()
