"""GPU reverse pass of Alg. 2 against the FP64 oracle's reverse pass and the
exact gradient U_k V_k^T of the top-k singular-value sum (GPU).

The oracle's reverse pass is itself pinned to central finite differences in
tests/test_oracle_grad.py.  Tolerance: relative Frobenius error 1e-4 against
the oracle (FP32 recomputation of v views and QRs); 1e-3 against U_k V_k^T
on the differentiation workload (the randomized estimate converges to it as
the sketch captures the top-k subspace).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grad as G  # noqa: E402
from paper_1804_07531_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("v", [2, 3, 4])
def test_backward_matches_oracle_reverse_pass(v):
    from paper_1804_07531_gb300 import api
    m, n, k, p = 600, 400, 6, 4
    a64 = S.usv(m, n, S.sigma_config("gap32", n), 71, 72) + 1e-3 * S.gaussian(m, n, seed=73)
    a32 = a64.astype(np.float32)
    om = S.gaussian(n, k + p, seed=74).astype(np.float32)
    da = api.subspace_iter_backward(torch.tensor(a32, device=DEV), k, p, v, torch.tensor(om, device=DEV),
                                    torch.ones(k, device=DEV))
    assert api.device_status(0) == 0
    ref = G.grad_topk_sigma_sum(a32.astype(np.float64), om.astype(np.float64), k, v)
    assert _rel(da.double().cpu().numpy(), ref) < 1e-4


def test_autograd_function_on_differentiation_workload():
    """8192 x 4096, sigma_j = exp(-j/40) with a x0.1 gap after j = 32, k = 32,
    p = 8, v = 4; loss = sum of the top-k estimated singular values."""
    from paper_1804_07531_gb300.autograd import lowrank_svd
    cfg = S.CONFIGS["grad_8192x4096_v4"]
    m, n, k, p, v = cfg["m"], cfg["n"], cfg["k"], cfg["p"], cfg["v"]
    sig = S.sigma_config("gap32", n)
    u = S.haar(m, n, cfg["seed_u"])
    vv = S.haar(n, n, cfg["seed_v"])
    a64 = (u * sig) @ vv.T
    a = torch.tensor(a64, dtype=torch.float32, device=DEV, requires_grad=True)
    om = torch.tensor(S.gaussian(n, k + p, seed=cfg["seed_omega"]), dtype=torch.float32, device=DEV)
    _, s, _ = lowrank_svd(a, k, p, v, om)
    s.sum().backward()
    g = a.grad.double().cpu().numpy()
    exact = u[:, :k] @ vv[:, :k].T
    assert _rel(g, exact) < 1e-3
    ref = G.grad_topk_sigma_sum(a.detach().double().cpu().numpy(), om.double().cpu().numpy(), k, v)
    assert _rel(g, ref) < 1e-4


@pytest.mark.parametrize("v", [2, 3, 4])
def test_backward_through_u_s_v_matches_oracle(v):
    """L = <dU, U> + <dS, S> + <dV, V>: the GPU reverse pass (lifts, core SVD,
    thin QRs, views) against the oracle's (pinned by finite differences);
    relative Frobenius 1e-3 -- the core SVD's reverse divides by
    s_j^2 - s_i^2, which amplifies the FP32 rounding of the recomputed
    forward pass."""
    from paper_1804_07531_gb300 import api
    m, n, k, p = 600, 400, 6, 4
    a64 = S.usv(m, n, S.sigma_config("gap32", n), 81, 82) + 1e-3 * S.gaussian(m, n, seed=83)
    a32 = a64.astype(np.float32)
    om = S.gaussian(n, k + p, seed=84).astype(np.float32)
    du = S.gaussian(m, k, seed=85).astype(np.float32)
    ds = S.gaussian(k, 1, seed=86)[:, 0].astype(np.float32)
    dv = S.gaussian(n, k, seed=87).astype(np.float32)
    t = lambda x: torch.tensor(x, device=DEV)  # noqa: E731
    da = api.subspace_iter_backward(t(a32), k, p, v, t(om), ds=t(ds), du=t(du), dv=t(dv))
    assert api.device_status(0) == 0
    ref = G.grad_lowrank(a32.astype(np.float64), om.astype(np.float64), k, v, du.astype(np.float64),
                         ds.astype(np.float64), dv.astype(np.float64))
    assert _rel(da.double().cpu().numpy(), ref) < 1e-3
    # U alone and V alone
    da_u = api.subspace_iter_backward(t(a32), k, p, v, t(om), du=t(du))
    ref_u = G.grad_lowrank(a32.astype(np.float64), om.astype(np.float64), k, v, du.astype(np.float64), None, None)
    assert _rel(da_u.double().cpu().numpy(), ref_u) < 1e-3
    da_v = api.subspace_iter_backward(t(a32), k, p, v, t(om), dv=t(dv))
    ref_v = G.grad_lowrank(a32.astype(np.float64), om.astype(np.float64), k, v, None, None, dv.astype(np.float64))
    assert _rel(da_v.double().cpu().numpy(), ref_v) < 1e-3


def test_autograd_loss_on_u_and_v():
    """A loss on U and V through LowRankSVD reaches A (the earlier form marked
    U and V non-differentiable)."""
    from paper_1804_07531_gb300.autograd import lowrank_svd
    m, n, k, p, v = 1024, 512, 8, 8, 4
    a64 = S.usv(m, n, S.sigma_config("gap32", n), 91, 92) + 1e-3 * S.gaussian(m, n, seed=93)
    a = torch.tensor(a64, dtype=torch.float32, device=DEV, requires_grad=True)
    om = torch.tensor(S.gaussian(n, k + p, seed=94), dtype=torch.float32, device=DEV)
    gu = torch.tensor(S.gaussian(m, k, seed=95), dtype=torch.float32, device=DEV)
    gv = torch.tensor(S.gaussian(n, k, seed=96), dtype=torch.float32, device=DEV)
    u, s, vv = lowrank_svd(a, k, p, v, om)
    loss = (u * gu).sum() + (vv * gv).sum() + s.sum()
    loss.backward()
    g = a.grad.double().cpu().numpy()
    ref = G.grad_lowrank(a.detach().double().cpu().numpy(), om.double().cpu().numpy(), k, v,
                         gu.double().cpu().numpy(), np.ones(k), gv.double().cpu().numpy())
    assert _rel(g, ref) < 1e-3
