"""The allocation-free range view against lr_sketch (GPU).

lr_sketch_range_static serves callers that cannot call cudaMalloc (for
example a host program whose own pool owns the device memory), so it takes no
handle and keeps its only scratch -- the BF16 copy of X -- in a static device
array.  Its result must match lr_sketch's range view within the view
tolerance (relative Frobenius 2e-5), on two calls in a row that reuse the
shared array with different operands and sizes.  This file is collected last
so that a run stopping at the first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _static_view(a, x):
    from paper_1804_07531_gb300._binding import _stream, col_major, empty_cm, lib, mat_a, mat_thin
    x = col_major(x)
    y = empty_cm(a.shape[0], x.shape[1], a.device)
    ma, mx, my = mat_a(a), mat_thin(x), mat_thin(y)
    st = lib().lr_sketch_range_static(ctypes.byref(ma), ctypes.byref(mx), ctypes.byref(my),
                                      ctypes.c_void_p(_stream()))
    return st, y


def _rel(a, b):
    return float((a - b).double().norm() / b.double().norm())


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
def test_static_range_view_matches_lr_sketch_twice(dtype):
    from paper_1804_07531_gb300 import api
    g = torch.Generator(device=DEV)
    g.manual_seed(7)
    for (m, n, ell) in [(3000, 2048, 120), (1000, 704, 30)]:   # two calls in a row
        a = torch.randn(m, n, device=DEV, generator=g).to(dtype)
        x = torch.randn(n, ell, device=DEV, generator=g)
        st, y = _static_view(a, x)
        assert st == 0
        y_ref, _ = api.sketch(a, x)
        torch.cuda.synchronize()
        assert _rel(y, y_ref) < 2e-5


def test_static_range_view_rejects_oversized_operand():
    from paper_1804_07531_gb300._binding import LR_F32
    a = torch.zeros(64, 65536, device=DEV, dtype=torch.bfloat16)
    x = torch.zeros(65536, 64, device=DEV)           # 65536 * 64 * 2 bytes = 8 MiB > 4 MiB
    st, _ = _static_view(a, x)
    assert st == 10                                    # LR_ERR_UNSUPPORTED
    assert LR_F32 == 0
