"""Python API over liblowrank.so: the paper's algorithms on torch CUDA tensors.

Names follow the C ABI (include/lowrank.h).  Every call takes A (m x n,
row-major float32 or bfloat16, on a CUDA device) and the caller's random test
matrices, runs on the current CUDA stream and returns new column-major
float32 tensors.  Letters: k = target rank, p = oversampling, ell = k + p,
v = number of views (the paper's p, l, p + l, v).
"""
from __future__ import annotations

import ctypes

import torch

from ._binding import (ALLREDUCE_FN, APPLY_FN, Handle, LowrankError, LrComm, LrMat, LrOperator, _opts, _stream,
                       col_major, empty_cm, lib, mat_a, mat_thin)

__all__ = [
    "Comm", "TorchDistComm", "subspace_iter_sharded",
    "sketch", "sketch_chained", "orth", "subspace_iter", "single_pass", "block_krylov",
    "rowwise_single_pass", "subspace_iter_backward", "single_pass_host", "subspace_iter_host", "block_krylov_host",
    "Operator", "MatrixOperator", "subspace_iter_op", "nystrom_tevd", "pinched_tevd", "single_pass_woolfe",
    "single_pass_extended", "srft", "device_status",
    "LowrankError",
]


def _prep(a, *thin):
    if not a.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if a.stride(1) != 1:
        a = a.contiguous()
    return a, [None if t is None else col_major(t.to(device=a.device, dtype=torch.float32)) for t in thin]


def _call(h, fn, *args):
    h.check(fn(h.h, *args))


def _p(m: LrMat):
    return ctypes.byref(m)


def sketch(a, x=None, w=None, stream=None, band_mb=0):
    """Y = A X and/or Z = A^T W (both from one read of A when both are given)."""
    a, (x, w) = _prep(a, x, w)
    h = Handle.get(a.device)
    m, n = a.shape
    y = empty_cm(m, x.shape[1], a.device) if x is not None else None
    z = empty_cm(n, w.shape[1], a.device) if w is not None else None
    h.reserve(m, n, max(1, x.shape[1] if x is not None else 1), w.shape[1] if w is not None else 0)
    mA = mat_a(a)
    args = [_p(mA)]
    keep = []
    for t in (x, w, y, z):
        if t is None:
            args.append(None)
        else:
            mt = mat_thin(t)
            keep.append(mt)
            args.append(_p(mt))
    o = _opts(band_mb=band_mb)
    _call(h, lib().lr_sketch, *args, ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return y, z


def sketch_chained(a, x, stream=None, band_mb=0):
    """Y = A X and Z = A^T Y from one read of A (Section 6.8)."""
    a, (x,) = _prep(a, x)
    h = Handle.get(a.device)
    m, n = a.shape
    y = empty_cm(m, x.shape[1], a.device)
    z = empty_cm(n, x.shape[1], a.device)
    h.reserve(m, n, x.shape[1])
    mA, mx, my, mz = mat_a(a), mat_thin(x), mat_thin(y), mat_thin(z)
    o = _opts(band_mb=band_mb)
    _call(h, lib().lr_sketch_chained, _p(mA), _p(mx), _p(my), _p(mz), ctypes.byref(o),
          ctypes.c_void_p(_stream(stream)))
    return y, z


def orth(y, want_r=True, shifted_fallback=False, stream=None):
    """Thin QR of y (rows >= cols) by block CholeskyQR2: returns (Q, R)."""
    q = col_major(y.to(torch.float32)).clone() if y.stride(0) != 1 else y.to(torch.float32).clone()
    q = col_major(q)
    h = Handle.get(q.device)
    rows, cols = q.shape
    h.reserve(rows, cols, cols)
    r = torch.zeros(cols, cols, dtype=torch.float64, device=q.device).t() if want_r else None
    mq = mat_thin(q)
    mr = mat_thin(r) if want_r else None
    o = _opts(shifted_fallback=shifted_fallback)
    _call(h, lib().lr_orth, _p(mq), _p(mr) if want_r else None, ctypes.byref(o),
          ctypes.c_void_p(_stream(stream)))
    return q, r


def _outs(a, k):
    m, n = a.shape
    return empty_cm(m, k, a.device), torch.empty(k, dtype=torch.float32, device=a.device), empty_cm(n, k, a.device)


def subspace_iter(a, k, p, v, omega, shifted_fallback=False, split_last=False, stream=None):
    """Alg. 2: generalized subspace iteration with v >= 2 views -> (U, S, V).

    split_last (BF16 A only): the last view's operand enters as two BF16
    terms (hi + lo), so that view's products carry ~16 operand bits."""
    a, (omega,) = _prep(a, omega)
    h = Handle.get(a.device)
    m, n = a.shape
    h.reserve(m, n, k + p, 0, v)
    u, s, vv = _outs(a, k)
    mats = [mat_a(a), mat_thin(omega), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts(shifted_fallback=shifted_fallback, split_last=split_last)
    _call(h, lib().lr_subspace_iter, _p(mats[0]), k, p, v, _p(mats[1]), _p(mats[2]), _p(mats[3]),
          _p(mats[4]), ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return u, s, vv


def block_krylov(a, k, p, v, omega, enhanced=False, shifted_fallback=False, split_last=False, stream=None):
    """Alg. 9 (or the row-streamed variant of Section 7.3 with enhanced=True);
    split_last as in subspace_iter."""
    a, (omega,) = _prep(a, omega)
    h = Handle.get(a.device)
    m, n = a.shape
    h.reserve(m, n, k + p, 0, v)
    u, s, vv = _outs(a, k)
    mats = [mat_a(a), mat_thin(omega), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts(enhanced=enhanced, shifted_fallback=shifted_fallback, split_last=split_last)
    _call(h, lib().lr_block_krylov, _p(mats[0]), k, p, v, _p(mats[1]), _p(mats[2]), _p(mats[3]),
          _p(mats[4]), ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return u, s, vv


def rowwise_single_pass(a, k, omega, stream=None):
    """Section 6.8: 2-view-accurate TSVD from one row-streamed read of A."""
    a, (omega,) = _prep(a, omega)
    h = Handle.get(a.device)
    m, n = a.shape
    h.reserve(m, n, omega.shape[1])
    u, s, vv = _outs(a, k)
    mats = [mat_a(a), mat_thin(omega), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts()
    _call(h, lib().lr_rowwise_single_pass, _p(mats[0]), k, _p(mats[1]), _p(mats[2]), _p(mats[3]),
          _p(mats[4]), ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return u, s, vv


def single_pass(a, k, omega, psi, l_c=None, shifted_fallback=False, stream=None):
    """Alg. 7: 1-view TSVD.  l_c=None: the baseline (l_c = l_1); an int
    0 <= l_c <= l_1 (e.g. oversampling.fixed_ratio(l_1, 0.5)); "minvar": the
    minimum-variance rule of Section 6.6, chosen on the device from the
    sketches (the call synchronises the stream once)."""
    a, (omega, psi) = _prep(a, omega, psi)
    h = Handle.get(a.device)
    m, n = a.shape
    h.reserve(m, n, omega.shape[1], psi.shape[1], 1)
    u, s, vv = _outs(a, k)
    mats = [mat_a(a), mat_thin(omega), mat_thin(psi), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts(l_c=l_c, shifted_fallback=shifted_fallback)
    _call(h, lib().lr_single_pass, _p(mats[0]), k, _p(mats[1]), _p(mats[2]), _p(mats[3]), _p(mats[4]),
          _p(mats[5]), ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return u, s, vv


def device_status(device=None, stream=None) -> int:
    """Read and clear the device status word (synchronises the stream)."""
    h = Handle.get(device if device is not None else torch.cuda.current_device())
    return h.status(stream)


def selftest_bounded_wait(timeout_us=20000, device=None, stream=None) -> int:
    """Run the cluster kernels' bounded wait on a phase nothing completes
    (lr_selftest_bounded_wait) and return the device status it leaves
    (LR_ERR_TIMEOUT = 7 when the bound works)."""
    h = Handle.get(device if device is not None else torch.cuda.current_device())
    h.check(lib().lr_selftest_bounded_wait(h.h, int(timeout_us), ctypes.c_void_p(_stream(stream))))
    return h.status(stream)


def subspace_iter_backward(a, k, p, v, omega, ds=None, du=None, dv=None, stream=None):
    """dA for L = <du, U> + <ds, S> + <dv, V> of Alg. 2 (views recomputed, dA
    written once); any of du, ds, dv may be None (zero), not all."""
    a, (omega,) = _prep(a, omega)
    h = Handle.get(a.device)
    m, n = a.shape
    h.reserve(m, n, k + p, 0, v)
    da = torch.empty(m, n, device=a.device, dtype=torch.float32)
    keep = []

    def opt_mat(t, thin=True):
        if t is None:
            return None
        t = col_major(t.detach().to(device=a.device, dtype=torch.float32)) if thin else \
            t.detach().to(device=a.device, dtype=torch.float32).contiguous()
        mt = mat_thin(t)
        keep.append((t, mt))
        return _p(mt)

    mA, mom, mda = mat_a(a), mat_thin(omega), mat_a(da)
    o = _opts()
    _call(h, lib().lr_subspace_iter_backward_uv, _p(mA), k, p, v, _p(mom), opt_mat(du), opt_mat(ds, thin=False),
          opt_mat(dv), _p(mda), ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return da


def _host_a(a_host, panel_cols, n):
    """(LrMat, m, n, panel width, panel layout?) for a pinned host A: a 2-D
    row-major m x n tensor, or a 3-D (panels, m, panel_cols) tensor holding
    contiguous column panels (the last one's columns past n unused)."""
    if a_host.is_cuda or a_host.dtype != torch.float32 or not a_host.is_contiguous() and a_host.stride(-1) != 1:
        raise ValueError("a_host must be a row-major float32 CPU tensor")
    if not a_host.is_pinned():
        raise ValueError("a_host must be in pinned memory (tensor.pin_memory())")
    if a_host.dim() == 3:
        if not a_host.is_contiguous():
            raise ValueError("a panel-stored A must be contiguous")
        npan, m, pc = a_host.shape
        n = npan * pc if n is None else int(n)
        if not (npan - 1) * pc < n <= npan * pc:
            raise ValueError("n does not match the number of panels")
        return LrMat(a_host.data_ptr(), m, n, pc, 0, 0), m, n, pc, True
    m, n = a_host.shape
    return LrMat(a_host.data_ptr(), m, n, a_host.stride(0), 0, 0), m, n, min(int(panel_cols), n), False


def single_pass_host(a_host, k, omega, psi, panel_cols=4096, l_c=None, n=None, device=None, stream=None):
    """Alg. 7 on a pinned host A (float32), streamed in column panels.

    A crosses the host link once: panels are copied through two device
    buffers (2 * m * panel_cols floats of workspace) while the previous panel
    is sketched.  a_host is row-major m x n, or a (panels, m, panel_cols)
    tensor of contiguous column panels (each panel then one contiguous copy;
    n gives the true column count).  omega / psi may live on the host or the
    device.
    """
    mh, m, n, pc, panels = _host_a(a_host, panel_cols, n)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    omega = col_major(omega.to(device=dev, dtype=torch.float32))
    psi = col_major(psi.to(device=dev, dtype=torch.float32))
    h = Handle.get(dev)
    h.reserve(m, n, omega.shape[1], psi.shape[1], 1, extra=2 * m * ((pc + 3) // 4 * 4) * 4 + 1024)
    u = empty_cm(m, k, dev)
    s = torch.empty(k, dtype=torch.float32, device=dev)
    vv = empty_cm(n, k, dev)
    mats = [mat_thin(omega), mat_thin(psi), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts(l_c=l_c, host_panels=panels)
    _call(h, lib().lr_single_pass_host, _p(mh), pc, k, _p(mats[0]), _p(mats[1]), _p(mats[2]), _p(mats[3]),
          _p(mats[4]), ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return u, s, vv


def subspace_iter_host(a_host, k, p, v, omega, panel_cols=4096, n=None, device=None, stream=None):
    """Alg. 2 on a pinned host A (float32; layouts as in single_pass_host):
    every view streams A in column panels through two device buffers
    (2 * m * panel_cols floats of workspace) while the previous panel is
    multiplied."""
    mh, m, n, pc, panels = _host_a(a_host, panel_cols, n)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    omega = col_major(omega.to(device=dev, dtype=torch.float32))
    h = Handle.get(dev)
    h.reserve(m, n, k + p, 0, v, extra=2 * m * ((pc + 3) // 4 * 4) * 4 + 1024)
    u = empty_cm(m, k, dev)
    s = torch.empty(k, dtype=torch.float32, device=dev)
    vv = empty_cm(n, k, dev)
    mats = [mat_thin(omega), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts(host_panels=panels)
    _call(h, lib().lr_subspace_iter_host, _p(mh), pc, k, p, v, _p(mats[0]), _p(mats[1]), _p(mats[2]),
          _p(mats[3]), ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return u, s, vv


def block_krylov_host(a_host, k, p, v, omega_host, out=None, enhanced=False, split_last=False, device=None,
                      stream=None):
    """Alg. 9 end to end from pinned host buffers (lr_block_krylov_host): A
    and Omega are copied once into the device workspace, all views read the
    device copy, and U, S, V come back into pinned host tensors (`out`, or new
    ones).  The results are valid after the stream synchronises."""
    if a_host.is_cuda or a_host.dtype not in (torch.float32, torch.bfloat16) or a_host.stride(1) != 1:
        raise ValueError("a_host must be a row-major float32 or bfloat16 CPU tensor")
    if not a_host.is_pinned():
        raise ValueError("a_host must be in pinned memory (tensor.pin_memory())")
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    m, n = a_host.shape
    ell = k + p
    om = omega_host
    if om.is_cuda or om.dtype != torch.float32 or om.stride(0) != 1 or om.stride(1) < n or not om.is_pinned():
        om = torch.empty(ell, n, dtype=torch.float32).pin_memory().t()   # pinned, column-major
        om.copy_(omega_host)
    if out is None:
        u = torch.empty(k, m, dtype=torch.float32).pin_memory().t()
        s = torch.empty(k, dtype=torch.float32).pin_memory()
        vv = torch.empty(k, n, dtype=torch.float32).pin_memory().t()
    else:
        u, s, vv = out
    h = Handle.get(dev)
    esz = a_host.element_size()
    staging = sum((b + 255) // 256 * 256 for b in (m * a_host.stride(0) * esz, n * ell * 4, m * k * 4, n * k * 4, k * 4))
    h.reserve(m, n, ell, 0, v, extra=staging + 1024)
    mh = LrMat(a_host.data_ptr(), m, n, a_host.stride(0), 1 if a_host.dtype == torch.bfloat16 else 0, 0)
    mats = [mat_thin(om), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts(enhanced=enhanced, split_last=split_last)
    with torch.cuda.device(dev):
        _call(h, lib().lr_block_krylov_host, _p(mh), k, p, v, _p(mats[0]), _p(mats[1]), _p(mats[2]), _p(mats[3]),
              ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return u, s, vv


# ------------------------------------------------------- operators
class _DeviceArray:
    """A column-major float32 device array described by __cuda_array_interface__
    (wrapped by torch.as_tensor without a copy)."""

    def __init__(self, ptr, rows, cols, ld):
        self.__cuda_array_interface__ = {"shape": (int(rows), int(cols)), "typestr": "<f4",
                                         "data": (int(ptr), False), "strides": (4, 4 * int(ld)), "version": 2}


class Operator:
    """A matrix-free J (rows x cols) for the operator entry points (Section
    4.2.3: J applied by direct and adjoint methods).  apply(transpose, X, Y)
    must write Y = J X (transpose = 0; X cols x ncols, Y rows x ncols) or
    Y = J^T X (transpose = 1) into the given column-major float32 CUDA
    tensors, on the current stream."""

    def __init__(self, rows, cols, apply, device=None):
        self.rows, self.cols = int(rows), int(cols)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._apply = apply
        self.error = None

        def cb(ctx, transpose, xp, ldx, ncols, yp, ldy, stream):
            try:
                rx, ry = (self.cols, self.rows) if transpose == 0 else (self.rows, self.cols)
                x = torch.as_tensor(_DeviceArray(xp, rx, ncols, ldx), device=self.device)
                y = torch.as_tensor(_DeviceArray(yp, ry, ncols, ldy), device=self.device)
                self._apply(int(transpose), x, y)
                return 0
            except Exception as e:  # reported to the caller by the entry point's status
                self.error = e
                return 1

        self._cb = APPLY_FN(cb)
        self.c = LrOperator(self.rows, self.cols, self._cb, None)


class MatrixOperator(Operator):
    """J as a device matrix (float32 or bfloat16, row-major), applied by this
    library's own views on a handle of its own."""

    def __init__(self, j):
        if not j.is_cuda or j.stride(1) != 1:
            raise ValueError("J must be a row-major CUDA matrix")
        self.j = j
        self.h = Handle(j.device.index)

        def apply(transpose, x, y):
            m, n = self.j.shape
            self.h.reserve(m, n, max(1, x.shape[1]))
            mA, mx, my = mat_a(self.j), mat_thin(x), mat_thin(y)
            o = _opts()
            if transpose == 0:
                st = lib().lr_sketch(self.h.h, _p(mA), _p(mx), None, _p(my), None, ctypes.byref(o),
                                     ctypes.c_void_p(_stream()))
            else:
                st = lib().lr_sketch(self.h.h, _p(mA), None, _p(mx), None, _p(my), ctypes.byref(o),
                                     ctypes.c_void_p(_stream()))
            self.h.check(st)

        super().__init__(j.shape[0], j.shape[1], apply, device=j.device.index)


def subspace_iter_op(op, k, p, v, omega, stream=None):
    """Alg. 2 with J given as an Operator: (U, S, V)."""
    dev = op.device
    h = Handle.get(dev)
    h.reserve(op.rows, op.cols, k + p, 0, v)
    omega = col_major(omega.to(device=dev, dtype=torch.float32))
    u = empty_cm(op.rows, k, dev)
    s = torch.empty(k, dtype=torch.float32, device=dev)
    vv = empty_cm(op.cols, k, dev)
    mats = [mat_thin(omega), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts()
    _call(h, lib().lr_subspace_iter_op, ctypes.byref(op.c), k, p, v, _p(mats[0]), _p(mats[1]), _p(mats[2]),
          _p(mats[3]), ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return u, s, vv


def _tevd(fn, op, k, p, v, omega, stream):
    dev = op.device
    h = Handle.get(dev)
    h.reserve(op.rows, op.cols, k + p, 0, v)
    omega = col_major(omega.to(device=dev, dtype=torch.float32))
    vv = empty_cm(op.cols, k, dev)
    lam2 = torch.empty(k, dtype=torch.float32, device=dev)
    mats = [mat_thin(omega), mat_thin(vv), mat_thin(lam2)]
    o = _opts()
    st = fn(h.h, ctypes.byref(op.c), k, p, v, _p(mats[0]), _p(mats[1]), _p(mats[2]), ctypes.byref(o),
            ctypes.c_void_p(_stream(stream)))
    if st != 0 and op.error is not None:
        raise op.error
    h.check(st)
    return vv, lam2


def nystrom_tevd(op, k, p, v, omega, stream=None):
    """Alg. 4: (V, Lambda2), the Nystrom rank-k EVD of J^T J from v >= 2 views
    of J.  omega: cols x (k+p) for even v, rows x (k+p) for odd v."""
    return _tevd(lib().lr_nystrom_tevd, op, k, p, v, omega, stream)


def pinched_tevd(op, k, p, v, omega, stream=None):
    """Alg. 5: (V, Lambda2), the pinched rank-k EVD of J^T J from v >= 2 views
    of J.  omega: rows x (k+p) for even v, cols x (k+p) for odd v."""
    return _tevd(lib().lr_pinched_tevd, op, k, p, v, omega, stream)



# ------------------------------------------- other single-view methods
def single_pass_woolfe(a, k, omega, psi, l_c=None, stream=None):
    """Alg. 8 (Woolfe variant of the single view): (U, S, V)."""
    a, (omega, psi) = _prep(a, omega, psi)
    h = Handle.get(a.device)
    m, n = a.shape
    h.reserve(m, n, omega.shape[1], psi.shape[1], 1)
    u, s, vv = _outs(a, k)
    mats = [mat_a(a), mat_thin(omega), mat_thin(psi), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts(l_c=l_c)
    _call(h, lib().lr_single_pass_woolfe, _p(mats[0]), k, _p(mats[1]), _p(mats[2]), _p(mats[3]), _p(mats[4]),
          _p(mats[5]), ctypes.byref(o), ctypes.c_void_p(_stream(stream)))
    return u, s, vv


def srft(n, signs, cols, device=None, stream=None):
    """Phi = D F P (n x s, column-major float32 on the device): D = diag(signs)
    (+-1), F the orthonormal DCT-II matrix, P the columns `cols`."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    signs = torch.as_tensor(signs, dtype=torch.float32).to(dev).contiguous()
    cols = torch.as_tensor(cols, dtype=torch.int32).to(dev).contiguous()
    s = int(cols.numel())
    phi = empty_cm(n, s, dev)
    h = Handle.get(dev)
    mp = mat_thin(phi)
    h.check(lib().lr_srft(h.h, int(n), s, ctypes.c_void_p(signs.data_ptr()), ctypes.c_void_p(cols.data_ptr()),
                          _p(mp), ctypes.c_void_p(_stream(stream))))
    return phi


def single_pass_extended(a, k, omega, psi, phi_c, phi_r, stream=None):
    """Section 6.7 (bwz2): single view with the extended sketch Z = Phi_r^T A
    Phi_c, e.g. with SRFT test matrices from srft(); (U, S, V)."""
    a, (omega, psi, phi_c, phi_r) = _prep(a, omega, psi, phi_c, phi_r)
    h = Handle.get(a.device)
    m, n = a.shape
    w = omega.shape[1] + phi_c.shape[1]
    h.reserve(m, n, w, w, 1, extra=4 * (2 * (m + n) * w) + 1024)
    u, s, vv = _outs(a, k)
    mats = [mat_a(a), mat_thin(omega), mat_thin(psi), mat_thin(phi_c), mat_thin(phi_r), mat_thin(u), mat_thin(s),
            mat_thin(vv)]
    o = _opts()
    _call(h, lib().lr_single_pass_extended, _p(mats[0]), k, *[_p(x) for x in mats[1:]], ctypes.byref(o),
          ctypes.c_void_p(_stream(stream)))
    return u, s, vv


# ------------------------------------------------ rows over several GPUs
def _wrap_buffer(ptr, count, dtype, device):
    """A 1-D tensor over the library's buffer (float32 for dtype 0, float64
    for dtype 2): device memory through __cuda_array_interface__, host
    memory through ctypes."""
    if dtype not in (0, 2):
        raise ValueError(f"unsupported all-reduce dtype {dtype}")
    if device.type == "cuda":
        class _Buf:
            __cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f4" if dtype == 0 else "<f8",
                                        "data": (int(ptr), False), "strides": None, "version": 2}
        return torch.as_tensor(_Buf(), device=device)
    ctype = ctypes.c_float if dtype == 0 else ctypes.c_double
    arr = (ctype * int(count)).from_address(int(ptr))
    return torch.frombuffer(arr, dtype=torch.float32 if dtype == 0 else torch.float64)


class Comm:
    """The collective of the row-sharded entry points: this process's rank,
    the number of ranks, and allreduce(t), which sums the 1-D tensor t
    (float32 or float64, on `device`) over the ranks in place, ordered on
    the current stream (the library's stream while it runs)."""

    def __init__(self, rank, world, allreduce, device=None):
        self.rank, self.world = int(rank), int(world)
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        self._allreduce = allreduce
        self.error = None

        def cb(ctx, buf, count, dtype, stream):
            try:
                t = _wrap_buffer(buf, count, dtype, self.device)
                if self.device.type == "cuda":
                    st = (torch.cuda.ExternalStream(stream, device=self.device) if stream
                          else torch.cuda.default_stream(self.device))
                    with torch.cuda.stream(st):
                        self._allreduce(t)
                else:
                    self._allreduce(t)
                return 0
            except Exception as e:  # reported to the caller by the entry point's status
                self.error = e
                return 1

        self._cb = ALLREDUCE_FN(cb)
        self.c = LrComm(self.rank, self.world, self._cb, None)


class TorchDistComm(Comm):
    """Comm over a torch.distributed process group (NCCL for device buffers;
    gloo serves host buffers)."""

    def __init__(self, group=None, device=None):
        import torch.distributed as dist
        super().__init__(dist.get_rank(group), dist.get_world_size(group),
                         lambda t: dist.all_reduce(t, group=group), device)


def subspace_iter_sharded(a_local, k, p, v, omega, comm, shifted_fallback=False, split_last=False, handle=None,
                          stream=None):
    """Alg. 2 on a matrix whose rows are split over comm.world ranks: this
    rank holds a_local (its block of rows, in rank order) and the common
    omega (n x (k + p)); returns (U_local, S, V) -- its rows of U, and S and
    V, the same on every rank."""
    a, (omega,) = _prep(a_local, omega)
    h = handle if handle is not None else Handle.get(a.device)
    m, n = a.shape
    h.reserve(m, n, k + p, 0, v)
    u, s, vv = _outs(a, k)
    mats = [mat_a(a), mat_thin(omega), mat_thin(u), mat_thin(s), mat_thin(vv)]
    o = _opts(shifted_fallback=shifted_fallback, split_last=split_last)
    comm.error = None
    st = lib().lr_subspace_iter_sharded(h.h, _p(mats[0]), k, p, v, _p(mats[1]), _p(mats[2]), _p(mats[3]),
                                        _p(mats[4]), ctypes.byref(comm.c), ctypes.byref(o),
                                        ctypes.c_void_p(_stream(stream)))
    if st != 0 and comm.error is not None:
        raise comm.error
    h.check(st)
    return u, s, vv
