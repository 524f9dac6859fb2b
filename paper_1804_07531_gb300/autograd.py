"""torch.autograd.Function over the library's forward and reverse passes.

``LowRankSVD.apply(A, k, p, v, Omega)`` runs Alg. 2 (generalized subspace
iteration, v views) and returns (U, S, V).  Gradients flow to A through the
singular values S: the backward calls lr_subspace_iter_backward, which
recomputes the forward views from A and Omega (no panels are kept between
the two passes) and writes dL/dA once.  U and V are returned as constants.
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
        ctx.mark_non_differentiable(u, vv)
        return u, s, vv

    @staticmethod
    def backward(ctx, du, ds, dv):
        a, omega = ctx.saved_tensors
        k, p, v = ctx.cfg
        if ds is None:
            return None, None, None, None, None
        da = api.subspace_iter_backward(a, k, p, v, omega, ds)
        return da, None, None, None, None


def lowrank_svd(a, k, p, v, omega):
    """Differentiable rank-k TSVD of A by Alg. 2 (gradients through S)."""
    return LowRankSVD.apply(a, k, p, v, omega)
