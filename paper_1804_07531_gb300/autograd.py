"""torch.autograd.Function over the library's forward and reverse passes.

``LowRankSVD.apply(A, k, p, v, Omega)`` runs Alg. 2 (generalized subspace
iteration, v views) and returns (U, S, V).  Gradients of a loss on any of
the three flow to A: the backward calls lr_subspace_iter_backward_uv, which
recomputes the forward views from A and Omega (no panels are kept between
the two passes), reverses the lifts, the core SVD, the thin QRs and the
views, and writes dL/dA once.
"""
from __future__ import annotations

import torch

from . import api


class LowRankSVD(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, k, p, v, omega):
        if a.dtype != torch.float32:
            raise TypeError("the differentiable form needs a float32 A")
        u, s, vv = api.subspace_iter(a, k, p, v, omega)
        ctx.save_for_backward(a, omega)
        ctx.cfg = (int(k), int(p), int(v))
        return u, s, vv

    @staticmethod
    def backward(ctx, du, ds, dv):
        a, omega = ctx.saved_tensors
        k, p, v = ctx.cfg
        if du is None and ds is None and dv is None:
            return None, None, None, None, None
        da = api.subspace_iter_backward(a, k, p, v, omega, ds=ds, du=du, dv=dv)
        return da, None, None, None, None


def lowrank_svd(a, k, p, v, omega):
    """Differentiable rank-k TSVD of A by Alg. 2 (gradients through U, S and V)."""
    return LowRankSVD.apply(a, k, p, v, omega)
