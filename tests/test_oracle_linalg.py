"""Pins for the oracle's FP64 primitives (CPU only).

Each primitive is checked against something other than itself: its defining
identities, closed-form constructions, brute force on tiny inputs, hand-derived
golden values (tests/golden) and independent LAPACK routines from numpy.
"""
import json
import os

import numpy as np
import pytest

from oracle import linalg as L
from paper_1804_07531_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("shape", [(60, 17), (17, 17), (200, 40), (5, 1)])
def test_qr_definition_and_lapack(shape):
    y = S.gaussian(*shape, seed=shape[0] * 7 + shape[1])
    q, r = L.householder_qr(y)
    n = shape[1]
    assert np.abs(q @ r - y).max() < 1e-13 * max(1.0, np.abs(y).max()) * shape[0]
    assert np.abs(q.T @ q - np.eye(n)).max() < 1e-13
    assert np.all(np.tril(r, -1) == 0.0)
    assert np.all(np.diag(r) >= 0.0)
    # The thin QR with positive diagonal is unique: LAPACK's, sign-normalised, agrees.
    q2, r2 = np.linalg.qr(y)
    d = np.sign(np.diag(r2))
    assert np.allclose(q, q2 * d, atol=1e-12)
    assert np.allclose(r, r2 * d[:, None], atol=1e-12)


def test_qr_rank_deficient_does_not_divide_by_zero():
    g = S.gaussian(30, 3, seed=5)
    y = np.concatenate([g, g[:, :1] * 2.0, np.zeros((30, 1))], axis=1)
    q, r = L.householder_qr(y)
    assert np.isfinite(q).all() and np.isfinite(r).all()
    assert np.abs(q @ r - y).max() < 1e-12
    assert abs(r[3, 3]) < 1e-12 and abs(r[4, 4]) < 1e-12


def test_cholesky_and_solves():
    y = S.gaussian(80, 20, seed=9)
    g = y.T @ y
    r = L.cholesky_upper(g)
    assert np.abs(r.T @ r - g).max() < 1e-11 * np.abs(g).max()
    assert np.allclose(r.T, np.linalg.cholesky(g), atol=1e-11)
    b = S.gaussian(20, 3, seed=10)
    x = L.solve_upper(r, b)
    assert np.allclose(r @ x, b, atol=1e-11)
    x2 = L.solve_upper_right(b.T, r)
    assert np.allclose(x2 @ r, b.T, atol=1e-11)
    with pytest.raises(np.linalg.LinAlgError):
        L.cholesky_upper(-np.eye(3))


@pytest.mark.parametrize("m,n", [(40, 40), (90, 30), (30, 90), (7, 1)])
def test_jacobi_svd_closed_form(m, n):
    r = min(m, n)
    sig = np.sort(S.rng(m + n).uniform(0.1, 10.0, r))[::-1]
    u = S.haar(m, r, seed=m)
    v = S.haar(n, r, seed=n + 1000)
    a = (u * sig) @ v.T
    uu, ss, vv = L.jacobi_svd(a)
    assert np.abs(ss[:r] - sig).max() < 1e-12 * sig[0]
    assert np.abs((uu * ss) @ vv.T - a).max() < 1e-12 * sig[0]
    assert np.abs(uu[:, :r].T @ uu[:, :r] - np.eye(r)).max() < 1e-12
    assert np.abs(vv[:, :r].T @ vv[:, :r] - np.eye(r)).max() < 1e-12
    # Projectors onto leading singular subspaces match the construction.
    assert np.abs(uu[:, :3] @ uu[:, :3].T - u[:, :3] @ u[:, :3].T).max() < 1e-10


def test_jacobi_svd_matches_lapack_and_zero_singular_values():
    a = S.gaussian(25, 10, seed=3)
    a[:, 9] = a[:, 0] - a[:, 1]                 # rank 9
    _, s, _ = L.jacobi_svd(a)
    assert np.allclose(s, np.linalg.svd(a, compute_uv=False), atol=1e-12)
    assert s[-1] < 1e-12


def test_golden_closed_forms():
    with open(os.path.join(GOLDEN, "closed_form_svd.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        a = np.array(c["matrix"], dtype=np.float64)
        _, s, _ = L.jacobi_svd(a)
        exp = np.array(c["singular_values"], dtype=np.float64)
        assert np.allclose(s[: len(exp)], exp, rtol=0, atol=1e-12 * max(1.0, exp[0])), c["name"]


def test_fix_signs():
    u = np.array([[0.1, -0.9], [-0.8, 0.2]])
    v = np.array([[1.0, 2.0], [3.0, 4.0]])
    u2, v2 = L.fix_signs(u, v)
    assert np.allclose(u2, [[-0.1, 0.9], [0.8, -0.2]])
    assert np.allclose(v2, [[-1.0, -2.0], [-3.0, -4.0]])
