"""The allocation-free range view (GPU).

lr_sketch_range_static serves callers that cannot call cudaMalloc (for
example a host program whose own pool owns the device memory, or one that
cannot accept the synchronisation an allocation may imply), so it takes no
handle and keeps its only scratch -- the BF16 copy of X -- in a static device
array.  Checked here, on two calls in a row that reuse the shared array with
different operands and sizes:
  * the result against the FP64 product of the same operands (for a BF16 A
    the operand X rounded to BF16, as the kernel reads it), element-wise per
    column, and against lr_sketch's range view;
  * the status word the call leaves (lr_sketch_range_static_status) is 0;
  * a call leaves the device's free memory unchanged (it allocates nothing).
This file is collected last so that a run stopping at the first failure has
run every other test first.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _static_view(a, x, y=None):
    from paper_1804_07531_gb300._binding import _stream, col_major, empty_cm, lib, mat_a, mat_thin
    x = col_major(x)
    if y is None:
        y = empty_cm(a.shape[0], x.shape[1], a.device)
    ma, mx, my = mat_a(a), mat_thin(x), mat_thin(y)
    st = lib().lr_sketch_range_static(ctypes.byref(ma), ctypes.byref(mx), ctypes.byref(my),
                                      ctypes.c_void_p(_stream()))
    return st, y


def _static_status():
    from paper_1804_07531_gb300._binding import _stream, lib
    s = ctypes.c_int(-1)
    st = lib().lr_sketch_range_static_status(ctypes.c_void_p(_stream()), ctypes.byref(s))
    assert st == 0
    return s.value


def _colwise_err(y, ref):
    """max over columns of max_i |y_ij - ref_ij| / max_i |ref_ij|."""
    d = (y.double() - ref).abs().amax(dim=0)
    return float((d / ref.abs().amax(dim=0)).max())


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
def test_static_range_view_matches_fp64_and_lr_sketch_twice(dtype):
    from paper_1804_07531_gb300 import api
    g = torch.Generator(device=DEV)
    g.manual_seed(7)
    for (m, n, ell) in [(3000, 2048, 120), (1000, 704, 30)]:   # two calls in a row
        a = torch.randn(m, n, device=DEV, generator=g).to(dtype)
        x = torch.randn(n, ell, device=DEV, generator=g)
        st, y = _static_view(a, x)
        assert st == 0
        xr = x.bfloat16() if dtype == torch.bfloat16 else x
        ref = a.double() @ xr.double()
        y_ref, _ = api.sketch(a, x)
        torch.cuda.synchronize()
        assert _static_status() == 0
        assert _colwise_err(y, ref) < 2e-5
        assert _colwise_err(y_ref, ref) < 2e-5


def test_static_range_view_allocates_nothing():
    g = torch.Generator(device=DEV)
    g.manual_seed(8)
    a = torch.randn(2048, 1024, device=DEV, generator=g).bfloat16()
    x = torch.randn(1024, 64, device=DEV, generator=g)
    st, y = _static_view(a, x)                         # first call: set-up done
    assert st == 0
    a2 = torch.randn(1536, 768, device=DEV, generator=g).bfloat16()
    x2 = torch.randn(768, 48, device=DEV, generator=g)
    from paper_1804_07531_gb300._binding import col_major, empty_cm
    x2 = col_major(x2)                                 # the layout the call takes, made beforehand
    y2 = empty_cm(1536, 48, a2.device)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    st, _ = _static_view(a2, x2, y2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert st == 0
    assert free1 == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == stats0
    ref = a2.double() @ x2.bfloat16().double()
    assert _colwise_err(y2, ref) < 2e-5


def test_static_range_view_rejects_oversized_operand():
    from paper_1804_07531_gb300._binding import LR_F32
    a = torch.zeros(64, 65536, device=DEV, dtype=torch.bfloat16)
    x = torch.zeros(65536, 64, device=DEV)           # 65536 * 64 * 2 bytes = 8 MiB > 4 MiB
    st, _ = _static_view(a, x)
    assert st == 10                                    # LR_ERR_UNSUPPORTED
    assert LR_F32 == 0
