"""The fused one-read dual sketch (Alg. 7 steps a and b) against FP64 (GPU).

Y = A Omega and Z = A^T Psi of a BF16 A come from one kernel in which each
staged tile of A feeds both products.  Checked element by element against the
FP64 products of the same BF16 values (max_i |y_ij - ref_ij| <= 2e-5
max_i |ref_ij| in every column j: FP32 accumulation over K terms), at shapes
with a ragged last strip (m not a multiple of 256), a ragged last k-block (n
not a multiple of 64 or of 128), ell2 on both sides of 64 (the narrow form
with 128-column k-blocks) and of 128, and a Z whose leading dimension forbids
vector reductions; and against the two-pass form (opts.band_mb = -1) on the
same inputs.  The default picks the fused kernel for ell2 <= 64, and for
ell2 <= 128 when ell1 <= 64 (checked by the launch trace).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_07531_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def api():
    from paper_1804_07531_gb300 import api as _api
    return _api


def _colwise(y, ref):
    d = np.abs(y - ref).max(axis=0)
    return float((d / np.maximum(np.abs(ref).max(axis=0), 1e-30)).max())


def _bf16_matrix(m, n, seed, ld=None):
    a = torch.tensor(S.gaussian(m, n, seed=seed), dtype=torch.float32).bfloat16()
    if ld is None or ld == n:
        return a.to(DEV)
    store = torch.zeros(m, ld, dtype=torch.bfloat16)
    store[:, :n] = a
    return store.to(DEV)[:, :n]


@pytest.mark.parametrize("m,n,ell1,ell2,ld", [
    (1000, 704, 30, 60, None),
    (777, 1304, 1, 1, None),
    (2048, 1024, 120, 240, None),
    (520, 328, 64, 130, None),
    (4100, 2056, 128, 256, None),
    (300, 4096, 16, 200, None),
    (1500, 1302, 100, 90, 1304),      # n % 4 != 0: Z (ld n) takes scalar reductions
    (1500, 1302, 40, 64, 1304),       # narrow co-range form (ell2 <= 64), ragged 128-column k-blocks
    (2100, 1000, 128, 64, None),      # narrow co-range form beside the widest Y
    (1000, 704, 60, 120, None),       # the same form with 128 lines of Psi
    (1500, 1302, 40, 100, 1304),      # ... ragged, scalar reductions
])
def test_fused_dual_sketch_elementwise(m, n, ell1, ell2, ld):
    from paper_1804_07531_gb300._binding import Handle
    a = _bf16_matrix(m, n, m + 3 * n, ld)
    x = torch.tensor(S.gaussian(n, ell1, seed=11), dtype=torch.float32, device=DEV)
    w = torch.tensor(S.gaussian(m, ell2, seed=12), dtype=torch.float32, device=DEV)
    h = Handle.get(0)
    h.set_trace(True)
    h.trace_read("view_dual", reset=True)
    y, z = api().sketch(a, x, w, band_mb=-2)             # the fused kernel at every width
    _, launches = h.trace_read("view_dual", reset=True)
    h.set_trace(False)
    assert api().device_status(0) == 0
    assert launches == 1, "the fused kernel did not run"
    a64 = a.double().cpu().numpy()
    xr = x.bfloat16().double().cpu().numpy()
    wr = w.bfloat16().double().cpu().numpy()
    ey = _colwise(y.double().cpu().numpy(), a64 @ xr)
    ez = _colwise(z.double().cpu().numpy(), a64.T @ wr)
    assert ey < 2e-5 and ez < 2e-5, (ey, ez)
    # the two-pass form gives the same sketches to the same tolerance
    y2, z2 = api().sketch(a, x, w, band_mb=-1)
    assert api().device_status(0) == 0
    assert _colwise(y2.double().cpu().numpy(), a64 @ xr) < 2e-5
    assert _colwise(z2.double().cpu().numpy(), a64.T @ wr) < 2e-5


def test_fused_dual_sketch_single_pass_factorisation_matches_two_pass():
    """Alg. 7 on a BF16 A: the fused sketch and the two-pass sketch give the
    same factorisation to FP32 accumulation level."""
    m, n, k, ell1, ell2 = 4096, 2048, 20, 40, 80
    a64 = S.usv(m, n, S.sigma_config("exp25", 256), 21, 22) + 1e-4 * S.gaussian(m, n, seed=23)
    a = torch.tensor(a64, dtype=torch.float32).bfloat16().to(DEV)
    om = torch.tensor(S.gaussian(n, ell1, seed=24), dtype=torch.float32, device=DEV)
    ps = torch.tensor(S.gaussian(m, ell2, seed=25), dtype=torch.float32, device=DEV)
    u, s, v = api().single_pass(a, k, om, ps)
    assert api().device_status(0) == 0
    s1 = s.double().cpu().numpy()
    # reference: the same sketches from two separate views
    y, _ = api().sketch(a, om)
    _, z = api().sketch(a, None, ps)
    y2, z2 = api().sketch(a, om, ps, band_mb=-2)
    assert _colwise(y2.double().cpu().numpy(), y.double().cpu().numpy()) < 2e-5
    assert _colwise(z2.double().cpu().numpy(), z.double().cpu().numpy()) < 2e-5
    assert np.all(np.diff(s1) <= 0) and s1[0] > 0


def test_default_picks_fused_kernel_for_narrow_sketches_only():
    from paper_1804_07531_gb300._binding import Handle
    a = _bf16_matrix(1024, 768, 5)
    h = Handle.get(0)
    h.set_trace(True)
    for ell1, ell2, want in ((32, 64, 1), (64, 128, 1), (65, 128, 0), (32, 129, 0)):
        x = torch.randn(768, ell1, device=DEV)
        w = torch.randn(1024, ell2, device=DEV)
        h.trace_read("view_dual", reset=True)
        api().sketch(a, x, w)
        _, launches = h.trace_read("view_dual", reset=True)
        assert launches == want, (ell1, ell2, launches)
    h.set_trace(False)
    assert api().device_status(0) == 0
