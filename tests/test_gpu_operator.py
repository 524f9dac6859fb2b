"""The matrix-free operator boundary and the normal-matrix TEVDs (GPU).

J is given to the library as a callback (lr_operator).  Checked against the
FP64 oracle (oracle/normal.py) at the FP32 bars:
  * Alg. 4 (Nystrom) and Alg. 5 (pinched) for v = 2..5: eigenvalues
    max_i |lam_i - lam_i^oracle| <= 2e-5 lam_1 (twice the sigma bar: lam =
    sigma^2), V orthonormal to 1e-5 and spanning the oracle's leading
    eigenspace (projector distance <= 1e-3 on a spectrum with gaps);
    the oracle uses the library's FP32 shift rule (2^-23 ||Y_r||_F);
  * Alg. 2 through the callback gives the device-resident Alg. 2's result;
  * the callback may be user code (torch matmul here);
  * a failing callback is reported as LR_ERR_INVALID_ARG, synchronously.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import algorithms as Al  # noqa: E402
from oracle import normal as Nm  # noqa: E402
from paper_1804_07531_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def api():
    from paper_1804_07531_gb300 import api as _api
    return _api


def f64(t):
    return t.detach().double().cpu().numpy()


@pytest.fixture(scope="module")
def jmat():
    m, n = 3000, 1500
    a64 = S.usv(m, n, S.sigma_config("exp25", n), 71, 72)
    a32 = a64.astype(np.float32)
    return a32, torch.tensor(a32, device=DEV)


def _check(vg, lg, vo, lo, k):
    vg, lg = f64(vg), f64(lg)
    e_l = np.abs(lg - lo).max() / lo[0]
    orth = np.abs(vg.T @ vg - np.eye(k)).max()
    dist = np.linalg.norm(vg @ vg.T - vo @ vo.T, 2)
    msg = f"lambda {e_l:.2e} orth {orth:.2e} subspace {dist:.2e}"
    assert e_l <= 2e-5 and orth <= 1e-5 and dist <= 1e-3, msg
    return msg


@pytest.mark.parametrize("v", [2, 3, 4, 5])
def test_nystrom_tevd_matches_oracle(jmat, v):
    a32, j = jmat
    m, n = a32.shape
    k, p = 20, 10
    om = S.gaussian(n if v % 2 == 0 else m, k + p, seed=73 + v).astype(np.float32)
    op = api().MatrixOperator(j)
    vg, lg = api().nystrom_tevd(op, k, p, v, torch.tensor(om, device=DEV))
    assert api().device_status(0) == 0
    vo, lo = Nm.nystrom_tevd(Nm.MatrixOperator(a32.astype(np.float64)), om.astype(np.float64), k, v,
                             eps=2.0 ** -23, norm="fro")
    print(_check(vg, lg, vo, lo, k))


@pytest.mark.parametrize("v", [2, 3, 4, 5])
def test_pinched_tevd_matches_oracle(jmat, v):
    a32, j = jmat
    m, n = a32.shape
    k, p = 20, 10
    om = S.gaussian(m if v % 2 == 0 else n, k + p, seed=83 + v).astype(np.float32)
    op = api().MatrixOperator(j)
    vg, lg = api().pinched_tevd(op, k, p, v, torch.tensor(om, device=DEV))
    assert api().device_status(0) == 0
    vo, lo = Nm.pinched_tevd(Nm.MatrixOperator(a32.astype(np.float64)), om.astype(np.float64), k, v)
    print(_check(vg, lg, vo, lo, k))


@pytest.mark.parametrize("v", [2, 3])
def test_subspace_iteration_through_the_callback_matches_device_run(jmat, v):
    a32, j = jmat
    n = a32.shape[1]
    k, p = 20, 10
    om = torch.tensor(S.gaussian(n, k + p, seed=91).astype(np.float32), device=DEV)
    u1, s1, v1 = api().subspace_iter_op(api().MatrixOperator(j), k, p, v, om)
    u2, s2, v2 = api().subspace_iter(j, k, p, v, om)
    assert api().device_status(0) == 0
    assert np.abs(f64(s1) - f64(s2)).max() / f64(s2)[0] < 1e-6
    uo, so, vo = Al.gen_subspace_iteration(a32.astype(np.float64), f64(om), k, v)
    assert np.abs(f64(s1) - so).max() / so[0] < 1e-5


def test_user_callback_with_torch_matmul(jmat):
    a32, j = jmat
    m, n = a32.shape
    k, p, v = 10, 6, 4

    def apply(transpose, x, y):
        y.copy_((j.t() @ x) if transpose else (j @ x))

    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        op = api().Operator(m, n, apply)
        om = S.gaussian(n, k + p, seed=95).astype(np.float32)
        vg, lg = api().nystrom_tevd(op, k, p, v, torch.tensor(om, device=DEV))
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    assert api().device_status(0) == 0
    vo, lo = Nm.nystrom_tevd(Nm.MatrixOperator(a32.astype(np.float64)), om.astype(np.float64), k, v,
                             eps=2.0 ** -23, norm="fro")
    print(_check(vg, lg, vo, lo, k))


def test_failing_callback_is_reported(jmat):
    from paper_1804_07531_gb300._binding import LowrankError
    a32, j = jmat
    m, n = a32.shape

    def apply(transpose, x, y):
        raise RuntimeError("the user's operator failed")

    op = api().Operator(m, n, apply)
    om = torch.randn(n, 16, device=DEV)
    with pytest.raises((LowrankError, RuntimeError)):
        api().pinched_tevd(op, 8, 8, 3, om)
    assert api().device_status(0) == 0
