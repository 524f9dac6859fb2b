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
