"""The other single-view methods on the GPU against the FP64 oracle: Woolfe's
variant (Alg. 8) and the extended SRFT sketch (Sec. 6.7, bwz2), at the FP32
bars of the other parity tests (singular values norm-wise 1e-5,
reconstruction error 1e-5 relative, orthonormality 1e-5).  The SRFT test
matrices are formed by each side from the same Rademacher signs and sampled
DCT columns (lr_srft on the device, oracle/extended.srft on the host);
lr_srft itself is compared element by element with the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import algorithms as Al  # noqa: E402
from oracle import extended as Ex  # noqa: E402
from paper_1804_07531_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def api():
    from paper_1804_07531_gb300 import api as _api
    return _api


def f64(t):
    return t.detach().double().cpu().numpy()


def t32(x):
    return torch.tensor(np.asarray(x, dtype=np.float32), device=DEV)


def _check(a64, u, s, v, uo, so, vo, tol=1e-5):
    u, s, v = f64(u), f64(s), f64(v)
    k = s.shape[0]
    e_s = np.abs(s - so).max() / so[0]
    e_g, e_o = Al.frob_error(a64, u, s, v), Al.frob_error(a64, uo, so, vo)
    orth = max(np.abs(u.T @ u - np.eye(k)).max(), np.abs(v.T @ v - np.eye(k)).max())
    msg = f"sigma {e_s:.2e} recon {abs(e_g - e_o) / e_o:.2e} orth {orth:.2e}"
    assert e_s <= tol and abs(e_g - e_o) / e_o <= tol and orth <= tol, msg
    return msg


def _srft_inputs(n, s, seed):
    rng = np.random.default_rng(seed)
    return rng.choice([-1.0, 1.0], size=n), rng.choice(n, size=s, replace=False)


@pytest.mark.parametrize("n,s", [(1000, 64), (4093, 200), (65536, 300)])
def test_srft_matches_oracle(n, s):
    d, cols = _srft_inputs(n, s, n + s)
    phi = f64(api().srft(n, d, cols))
    assert api().device_status(0) == 0
    ref = Ex.srft(n, d, cols)
    assert np.abs(phi - ref).max() < 2e-6 * np.abs(ref).max()


@pytest.mark.parametrize("l_c", [None, 10, 0])
def test_woolfe_single_pass_matches_oracle(l_c):
    m, n, k, ell1, ell2 = 3000, 1500, 20, 40, 80
    a64 = S.usv(m, n, S.sigma_config("exp25", 256), 121, 122) + 1e-4 * S.gaussian(m, n, seed=123)
    a32 = a64.astype(np.float32)
    a = a32.astype(np.float64)
    om = S.gaussian(n, ell1, seed=124).astype(np.float32)
    ps = S.gaussian(m, ell2, seed=125).astype(np.float32)
    u, s, v = api().single_pass_woolfe(t32(a32), k, t32(om), t32(ps), l_c=l_c)
    assert api().device_status(0) == 0
    uo, so, vo = Ex.woolfe_single_pass(a, om.astype(np.float64), ps.astype(np.float64), k, l_c=l_c)
    print(_check(a, u, s, v, uo, so, vo))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_extended_single_pass_matches_oracle(dtype):
    m, n, k, ell, s = 3000, 1504, 20, 40, 120   # n * 2 bytes a multiple of 16 (BF16 rows)
    a64 = S.usv(m, n, S.sigma_config("inv", n), 131, 132) + 1e-4 * S.gaussian(m, n, seed=133)
    at = t32(a64) if dtype == "f32" else t32(a64).bfloat16()
    a = at.double().cpu().numpy()
    om = S.gaussian(n, ell, seed=134).astype(np.float32)
    ps = S.gaussian(m, ell, seed=135).astype(np.float32)
    dc, cc = _srft_inputs(n, s, 136)
    dr, cr = _srft_inputs(m, s, 137)
    phc, phr = api().srft(n, dc, cc), api().srft(m, dr, cr)
    u, sv, v = api().single_pass_extended(at, k, t32(om), t32(ps), phc, phr)
    assert api().device_status(0) == 0
    if dtype == "bf16":   # the views see the operands rounded to BF16
        rb = lambda x: torch.tensor(np.asarray(x, dtype=np.float32)).bfloat16().double().numpy()  # noqa: E731
        omr, psr, pcr, prr = rb(om), rb(ps), rb(Ex.srft(n, dc, cc)), rb(Ex.srft(m, dr, cr))
        uo, so, vo = Ex.extended_single_pass(a, omr, psr, pcr, prr, k)
        e_g = Al.frob_error(a, f64(u), f64(sv), f64(v))
        assert abs(e_g - Al.frob_error(a, uo, so, vo)) / Al.frob_error(a, uo, so, vo) < 1e-3
        assert np.abs(f64(sv) - so).max() / so[0] < 1e-3
    else:
        uo, so, vo = Ex.extended_single_pass(a, om.astype(np.float64), ps.astype(np.float64),
                                             Ex.srft(n, dc, cc), Ex.srft(m, dr, cr), k)
        print(_check(a, u, sv, v, uo, so, vo))
