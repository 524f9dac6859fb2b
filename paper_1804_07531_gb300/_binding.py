"""ctypes binding of liblowrank.so (argument marshalling only).

Every function forwards torch tensors' device pointers, shapes and the current
CUDA stream to the C ABI declared in include/lowrank.h; all arithmetic runs in
the library's CUDA kernels.  There is no fallback: if the shared library is
missing or a call fails, a RuntimeError is raised.

Thin matrices are column-major: an m x ell operand is a torch tensor of shape
(m, ell) with stride (1, ld) (e.g. ``torch.empty(ell, m).t()``).  A is an
(m, n) row-major tensor (float32 or bfloat16).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblowrank.so")

LR_F32, LR_BF16, LR_F64 = 0, 1, 2
STATUS = {
    0: "LR_OK", 1: "LR_ERR_INVALID_ARG", 2: "LR_ERR_SHAPE", 3: "LR_ERR_DTYPE",
    4: "LR_ERR_ALIGNMENT", 5: "LR_ERR_BREAKDOWN", 6: "LR_ERR_NONFINITE", 7: "LR_ERR_TIMEOUT",
    8: "LR_ERR_CUDA", 9: "LR_ERR_NOMEM", 10: "LR_ERR_UNSUPPORTED",
}
EXPORTS = [
    "lr_create", "lr_destroy", "lr_status_string", "lr_last_error", "lr_workspace_size",
    "lr_set_workspace", "lr_get_status", "lr_sketch", "lr_sketch_chained", "lr_orth",
    "lr_subspace_iter", "lr_single_pass", "lr_block_krylov", "lr_rowwise_single_pass",
    "lr_single_pass_host", "lr_subspace_iter_host", "lr_block_krylov_host", "lr_subspace_iter_op",
    "lr_nystrom_tevd", "lr_pinched_tevd", "lr_single_pass_woolfe", "lr_single_pass_extended", "lr_srft", "lr_subspace_iter_backward",
    "lr_subspace_iter_backward_uv", "lr_subspace_iter_sharded", "lr_set_trace", "lr_trace_read",
    "lr_kernel_launches", "lr_sketch_range_static", "lr_sketch_range_static_status", "lr_selftest_bounded_wait",
]
TRACE_KINDS = {"view_range": 0, "view_corange": 1, "orth": 2, "core_svd": 3, "view_dual": 4}


class LrMat(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("dtype", ctypes.c_int32), ("col_major", ctypes.c_int32)]


class LrOpts(ctypes.Structure):
    _fields_ = [("l_c", ctypes.c_int32), ("enhanced", ctypes.c_int32), ("split_last", ctypes.c_int32),
                ("shifted_fallback", ctypes.c_int32), ("band_mb", ctypes.c_int32),
                ("host_panels", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


# int apply(void* ctx, int transpose, const float* X, int64_t ldx, int64_t ncols, float* Y, int64_t ldy,
#           void* stream)
APPLY_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                            ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p)


class LrOperator(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("apply", APPLY_FN), ("ctx", ctypes.c_void_p)]


# int allreduce(void* ctx, void* buf, int64_t count, int dtype, void* stream)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                ctypes.c_void_p)


class LrComm(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int), ("world", ctypes.c_int), ("allreduce", ALLREDUCE_FN),
                ("ctx", ctypes.c_void_p)]


class LowrankError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded liblowrank.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"liblowrank.so not found at {LIB_PATH}; build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            P, I, I64, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
            M = ctypes.POINTER(LrMat)
            O = ctypes.POINTER(LrOpts)
            L.lr_create.argtypes = [ctypes.POINTER(P), I]
            L.lr_destroy.argtypes = [P]
            L.lr_status_string.argtypes = [I]
            L.lr_status_string.restype = ctypes.c_char_p
            L.lr_last_error.argtypes = [P]
            L.lr_last_error.restype = ctypes.c_char_p
            L.lr_workspace_size.argtypes = [P, I64, I64, I, I, I, ctypes.POINTER(S)]
            L.lr_set_workspace.argtypes = [P, P, S]
            L.lr_get_status.argtypes = [P, P, ctypes.POINTER(I)]
            L.lr_sketch.argtypes = [P, M, M, M, M, M, O, P]
            L.lr_sketch_chained.argtypes = [P, M, M, M, M, O, P]
            L.lr_orth.argtypes = [P, M, M, O, P]
            L.lr_subspace_iter.argtypes = [P, M, I, I, I, M, M, M, M, O, P]
            L.lr_block_krylov.argtypes = [P, M, I, I, I, M, M, M, M, O, P]
            L.lr_single_pass.argtypes = [P, M, I, M, M, M, M, M, O, P]
            L.lr_rowwise_single_pass.argtypes = [P, M, I, M, M, M, M, O, P]
            L.lr_single_pass_host.argtypes = [P, M, I64, I, M, M, M, M, M, O, P]
            L.lr_subspace_iter_host.argtypes = [P, M, I64, I, I, I, M, M, M, M, O, P]
            L.lr_block_krylov_host.argtypes = [P, M, I, I, I, M, M, M, M, O, P]
            OP = ctypes.POINTER(LrOperator)
            L.lr_subspace_iter_op.argtypes = [P, OP, I, I, I, M, M, M, M, O, P]
            L.lr_nystrom_tevd.argtypes = [P, OP, I, I, I, M, M, M, O, P]
            L.lr_pinched_tevd.argtypes = [P, OP, I, I, I, M, M, M, O, P]
            L.lr_single_pass_woolfe.argtypes = [P, M, I, M, M, M, M, M, O, P]
            L.lr_single_pass_extended.argtypes = [P, M, I, M, M, M, M, M, M, M, O, P]
            L.lr_srft.argtypes = [P, I64, I, P, P, M, P]
            L.lr_subspace_iter_backward.argtypes = [P, M, I, I, I, M, M, M, O, P]
            L.lr_subspace_iter_backward_uv.argtypes = [P, M, I, I, I, M, M, M, M, M, O, P]
            L.lr_subspace_iter_sharded.argtypes = [P, M, I, I, I, M, M, M, M, ctypes.POINTER(LrComm), O, P]
            L.lr_set_trace.argtypes = [P, I]
            L.lr_trace_read.argtypes = [P, I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), I]
            L.lr_kernel_launches.argtypes = [P, ctypes.POINTER(ctypes.c_uint64)]
            L.lr_sketch_range_static.argtypes = [M, M, M, P]
            L.lr_sketch_range_static_status.argtypes = [P, ctypes.POINTER(I)]
            L.lr_selftest_bounded_wait.argtypes = [P, I64, P]
            for name in EXPORTS:
                f = getattr(L, name)
                if name not in ("lr_status_string", "lr_last_error"):
                    f.restype = I
            _lib = L
        return _lib


# ------------------------------------------------------------ matrices
def col_major(t: torch.Tensor) -> torch.Tensor:
    """t (rows, cols) laid out column-major (stride (1, ld)); copies if needed."""
    if t.dim() == 1:
        t = t[:, None]
    if t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


def empty_cm(rows, cols, device, dtype=torch.float32):
    return torch.empty(cols, rows, device=device, dtype=dtype).t()


def mat_a(a: torch.Tensor) -> LrMat:
    if a.dtype not in (torch.float32, torch.bfloat16):
        raise TypeError("A must be float32 or bfloat16")
    if a.dim() != 2 or a.stride(1) != 1:
        raise ValueError("A must be a row-major 2-D tensor")
    dt = LR_F32 if a.dtype == torch.float32 else LR_BF16
    return LrMat(a.data_ptr(), a.shape[0], a.shape[1], a.stride(0), dt, 0)


def mat_thin(t: torch.Tensor) -> LrMat:
    if t.dtype == torch.float32:
        dt = LR_F32
    elif t.dtype == torch.float64:
        dt = LR_F64
    else:
        raise TypeError("thin matrices are float32 (R: float64)")
    if t.dim() == 1:
        return LrMat(t.data_ptr(), t.shape[0], 1, t.shape[0], dt, 1)
    if t.stride(0) != 1:
        raise ValueError("thin matrices must be column-major")
    return LrMat(t.data_ptr(), t.shape[0], t.shape[1], max(t.stride(1), t.shape[0]), dt, 1)


# -------------------------------------------------------------- handle
class Handle:
    """One lr_handle per CUDA device, with a workspace grown on demand."""

    _handles: dict = {}

    def __init__(self, device: int):
        self.device = device
        h = ctypes.c_void_p()
        st = lib().lr_create(ctypes.byref(h), device)
        if st != 0:
            raise LowrankError(st, "lr_create failed")
        self.h = h
        self.ws = None

    @classmethod
    def get(cls, device) -> "Handle":
        dev = torch.device(device).index if not isinstance(device, int) else device
        dev = torch.cuda.current_device() if dev is None else dev
        if dev not in cls._handles:
            cls._handles[dev] = Handle(dev)
        return cls._handles[dev]

    def check(self, st):
        if st != 0:
            msg = lib().lr_last_error(self.h).decode()
            raise LowrankError(st, msg)

    def reserve(self, m, n, ell1, ell2=0, v=2, extra=0):
        size = ctypes.c_size_t()
        self.check(lib().lr_workspace_size(self.h, m, n, ell1, ell2, v, ctypes.byref(size)))
        need = size.value + int(extra)
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(need + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
            ptr = (self.ws.data_ptr() + 255) // 256 * 256
            self.check(lib().lr_set_workspace(self.h, ctypes.c_void_p(ptr), need))

    def set_trace(self, on: bool):
        self.check(lib().lr_set_trace(self.h, int(bool(on))))

    def trace_read(self, kind: str, reset=False):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self.check(lib().lr_trace_read(self.h, TRACE_KINDS[kind], ctypes.byref(ms), ctypes.byref(n), int(reset)))
        return ms.value, n.value

    def kernel_launches(self) -> int:
        c = ctypes.c_uint64()
        self.check(lib().lr_kernel_launches(self.h, ctypes.byref(c)))
        return c.value

    def status(self, stream=None) -> int:
        s = ctypes.c_int()
        self.check(lib().lr_get_status(self.h, ctypes.c_void_p(_stream(stream)), ctypes.byref(s)))
        return s.value


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _opts(l_c=-1, enhanced=False, split_last=False, shifted_fallback=False, band_mb=0, host_panels=False) -> LrOpts:
    o = LrOpts()
    o.band_mb = int(band_mb)
    o.host_panels = int(bool(host_panels))
    o.l_c = -1 if l_c is None else -2 if l_c == "minvar" else int(l_c)
    o.enhanced = int(bool(enhanced))
    o.split_last = int(bool(split_last))
    o.shifted_fallback = int(bool(shifted_fallback))
    return o
