"""GPU edge cases of the method and of the boundary (through the C ABI).

  * exact recovery: A of rank r with k <= r <= ell = k + p is recovered
    exactly (up to FP32 rounding) by every schedule (Sections 3-4: the sketch
    then spans range(A)); r = ell with an ill-conditioned spectrum forces the
    shifted CholeskyQR retry (the FP32 Cholesky of the first Gram breaks
    down), and r < ell makes every sketch rank-deficient;
  * a NaN in A is reported as LR_ERR_NONFINITE in the device status word;
  * argument errors come back synchronously, before anything is launched:
    LR_ERR_INVALID_ARG (k + p > min(m, n), v < 2, ell2 < ell1), LR_ERR_SHAPE
    (Omega of the wrong shape), LR_ERR_DTYPE (column-major or F64 A) and
    LR_ERR_ALIGNMENT (A not 16-byte aligned, or a row stride that is not a
    multiple of 16 bytes);
  * the views element by element: max_i |y_ij - ref_ij| <= tol max_i |ref_ij|
    in every column j, at shapes with ragged tiles.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import algorithms as Al  # noqa: E402
from paper_1804_07531_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

LR_ERR_INVALID_ARG, LR_ERR_SHAPE, LR_ERR_DTYPE, LR_ERR_ALIGNMENT = 1, 2, 3, 4
LR_ERR_NONFINITE = 6


def api():
    from paper_1804_07531_gb300 import api as _api
    return _api


def t32(x):
    return torch.tensor(np.asarray(x, dtype=np.float32), device=DEV)


def f64(t):
    return t.detach().double().cpu().numpy()


def _rank_r(m, n, sig, seed):
    """A = U diag(sig) V^T with Haar U (m x r), V (n x r): rank r = len(sig)."""
    r = len(sig)
    u = np.linalg.qr(S.gaussian(m, r, seed=seed))[0]
    v = np.linalg.qr(S.gaussian(n, r, seed=seed + 1))[0]
    return (u * sig) @ v.T, u, v


def _check_exact(a64, u, s, vv, sig, uk, vk, k, tol=2e-5):
    """sigma and [[A]]_k = U_k diag(sig_k) V_k^T recovered to FP32 level."""
    U, sv, V = f64(u), f64(s), f64(vv)
    e_s = np.abs(sv - sig[:k]).max() / sig[0]
    best = (uk[:, :k] * sig[:k]) @ vk[:, :k].T
    e_a = np.linalg.norm((U * sv) @ V.T - best) / np.linalg.norm(best)
    orth = max(np.abs(U.T @ U - np.eye(k)).max(), np.abs(V.T @ V - np.eye(k)).max())
    msg = f"sigma {e_s:.2e} [[A]]_k {e_a:.2e} orth {orth:.2e}"
    assert e_s <= tol and e_a <= tol and orth <= 1e-5, msg
    return msg


@pytest.mark.parametrize("r,cond,robust", [(30, 1e4, False), (30, 1e4, True), (25, 1e2, True)])
@pytest.mark.parametrize("algo,v", [("subspace", 2), ("subspace", 3), ("krylov", 4), ("single_pass", 1)])
def test_exact_recovery_on_the_device(r, cond, robust, algo, v):
    """r = ell: the plain first Cholesky breaks down (kappa(Y) ~ 1e4 or more)
    and the shifted retry carries the factorisation; r < ell: the sketches are
    rank-deficient, which the four-pass form of opts.shifted_fallback handles."""
    m, n, k, p = 2048, 1024, 20, 10
    sig = np.geomspace(1.0, 1.0 / cond, r)
    a64, uk, vk = _rank_r(m, n, sig, 41)
    a32 = a64.astype(np.float32)
    om = S.gaussian(n, k + p, seed=43).astype(np.float32)
    if algo == "subspace":
        u, s, vv = api().subspace_iter(t32(a32), k, p, v, t32(om), shifted_fallback=robust)
        uo, so, vo = Al.gen_subspace_iteration(a32.astype(np.float64), om.astype(np.float64), k, v)
    elif algo == "krylov":
        u, s, vv = api().block_krylov(t32(a32), k, p, v, t32(om), shifted_fallback=robust)
        uo, so, vo = Al.block_krylov(a32.astype(np.float64), om.astype(np.float64), k, v)
    else:
        ps = S.gaussian(m, 2 * (k + p), seed=44).astype(np.float32)
        u, s, vv = api().single_pass(t32(a32), k, t32(om), t32(ps), shifted_fallback=robust)
        uo, so, vo = Al.single_pass(a32.astype(np.float64), om.astype(np.float64), ps.astype(np.float64), k)
    st = api().device_status(0)
    assert st == 0, f"device status {st}"
    # the oracle recovers it exactly too (its own pin), so both bars hold
    assert np.abs(so - sig[:k]).max() / sig[0] < 1e-6
    print(_check_exact(a64, u, s, vv, sig, uk, vk, k))


def test_rank_deficient_sketch_without_fallback_reports_breakdown():
    """Without opts.shifted_fallback a rank-deficient sketch is reported, not
    silently returned: LR_ERR_BREAKDOWN in the status word."""
    m, n, k, p = 2048, 1024, 20, 10
    a64, _, _ = _rank_r(m, n, np.geomspace(1.0, 1e-2, 25), 45)
    om = S.gaussian(n, k + p, seed=46).astype(np.float32)
    api().subspace_iter(t32(a64.astype(np.float32)), k, p, 2, t32(om))
    assert api().device_status(0) == 5  # LR_ERR_BREAKDOWN
    assert api().device_status(0) == 0


def test_nan_in_a_is_reported_nonfinite():
    m, n, k, p = 1024, 512, 10, 6
    a = S.gaussian(m, n, seed=51).astype(np.float32)
    a[300, 77] = np.nan
    om = S.gaussian(n, k + p, seed=52).astype(np.float32)
    assert api().device_status(0) == 0
    api().subspace_iter(t32(a), k, p, 2, t32(om))
    assert api().device_status(0) == LR_ERR_NONFINITE
    # the context stays usable and the status word was cleared by the read
    a[300, 77] = 0.0
    u, s, vv = api().subspace_iter(t32(a), k, p, 2, t32(om))
    assert api().device_status(0) == 0
    assert np.all(np.isfinite(f64(s)))


def _status_of(fn):
    from paper_1804_07531_gb300._binding import Handle, LowrankError
    h = Handle.get(0)
    n0 = h.kernel_launches()
    with pytest.raises(LowrankError) as ei:
        fn()
    assert h.kernel_launches() == n0, "an argument error launched kernels"
    return ei.value.status


def test_argument_errors_are_synchronous():
    m, n = 512, 256
    a = torch.randn(m, n, device=DEV)
    om = torch.randn(n, 30, device=DEV)
    ps = torch.randn(m, 20, device=DEV)
    A = api()
    torch.cuda.synchronize()
    # k + p > min(m, n)
    assert _status_of(lambda: A.subspace_iter(a, 200, 100, 2, torch.randn(n, 300, device=DEV))) == LR_ERR_INVALID_ARG
    # v < 2 for subspace iteration and block Krylov
    assert _status_of(lambda: A.subspace_iter(a, 20, 10, 1, om)) == LR_ERR_INVALID_ARG
    assert _status_of(lambda: A.block_krylov(a, 20, 10, 1, om)) == LR_ERR_INVALID_ARG
    # ell2 < ell1 (l_2 >= l_1 is required)
    assert _status_of(lambda: A.single_pass(a, 10, om, ps)) == LR_ERR_INVALID_ARG
    # Omega of the wrong shape
    assert _status_of(lambda: A.subspace_iter(a, 20, 10, 2, torch.randn(n, 31, device=DEV))) == LR_ERR_SHAPE
    # A not 16-byte aligned: a view starting one FP32 element in
    store = torch.randn(m, n + 4, device=DEV)
    a_off = store[:, 1:n + 1]
    assert a_off.stride(1) == 1 and a_off.data_ptr() % 16 == 4
    assert _status_of(lambda: A.subspace_iter(a_off, 20, 10, 2, om)) == LR_ERR_ALIGNMENT
    # a row stride that is not a multiple of 16 bytes (n + 1 FP32 elements)
    store2 = torch.randn(m, n + 1, device=DEV)
    assert _status_of(lambda: A.subspace_iter(store2[:, :n], 20, 10, 2, om)) == LR_ERR_ALIGNMENT
    assert api().device_status(0) == 0


@pytest.mark.parametrize("case", ["col_major", "f64"])
def test_unsupported_layout_or_dtype_is_rejected_through_the_abi(case):
    import ctypes

    from paper_1804_07531_gb300._binding import Handle, LrMat, _opts, _stream, empty_cm, lib, mat_thin
    m, n, k, p = 256, 128, 8, 4
    om = empty_cm(n, k + p, DEV)
    u, vv = empty_cm(m, k, DEV), empty_cm(n, k, DEV)
    s = torch.empty(k, device=DEV)
    h = Handle.get(0)
    h.reserve(m, n, k + p, 0, 2)
    if case == "col_major":
        a = torch.randn(n, m, device=DEV).t()      # column-major m x n
        ma = LrMat(a.data_ptr(), m, n, m, 0, 1)
    else:
        a = torch.randn(m, n, device=DEV, dtype=torch.float64)
        ma = LrMat(a.data_ptr(), m, n, n, 2, 0)   # LR_F64 A
    n0 = h.kernel_launches()
    mats = [mat_thin(om), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts()
    st = lib().lr_subspace_iter(h.h, ctypes.byref(ma), k, p, 2, *[ctypes.byref(x) for x in mats],
                                ctypes.byref(o), ctypes.c_void_p(_stream()))
    assert st == LR_ERR_DTYPE
    assert h.kernel_launches() == n0


def _colwise(y, ref):
    d = np.abs(y - ref).max(axis=0)
    return float((d / np.abs(ref).max(axis=0)).max())


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("m,n,ell", [(1000, 704, 30), (777, 1304, 1), (2048, 1024, 120), (520, 328, 250),
                                     (4100, 2056, 64)])
def test_views_elementwise(dtype, m, n, ell):
    a = S.gaussian(m, n, seed=m + 7 * n).astype(np.float32)
    x = S.gaussian(n, ell, seed=8).astype(np.float32)
    w = S.gaussian(m, ell + 5, seed=9).astype(np.float32)
    at = t32(a) if dtype == "f32" else t32(a).bfloat16()
    y, z = api().sketch(at, t32(x), t32(w))
    assert api().device_status(0) == 0
    a64 = at.double().cpu().numpy()
    if dtype == "bf16":
        xr, wr = t32(x).bfloat16().double().cpu().numpy(), t32(w).bfloat16().double().cpu().numpy()
    else:
        xr, wr = x.astype(np.float64), w.astype(np.float64)
    ey, ez = _colwise(f64(y), a64 @ xr), _colwise(f64(z), a64.T @ wr)
    assert ey < 2e-5 and ez < 2e-5, (ey, ez)
