"""``torch.autograd.Function`` over G-GPDF distance queries.

Forward: ``vgp_query_distance_gradient``.  Backward: ``vgp_query_backward``, which
recomputes each instance's factorisation and alpha and returns d(distance)/d(query) and
d(distance)/d(surface points) through the derivative of alpha = (K + sigma^2 I)^-1 1
(Eq. 1) and of the reverting function (Eq. 3).
"""
from __future__ import annotations

import torch

from .api import Map


class GPDFDistance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q: torch.Tensor, X: torch.Tensor, gmap: Map):
        if not gmap.surface_is(X):
            gmap.set_surface(X)
        out = gmap.query(q, grad=False, var=False)
        ctx.save_for_backward(q, X)
        ctx.gmap = gmap
        return out["d"].to(q.dtype)

    @staticmethod
    def backward(ctx, gd: torch.Tensor):
        q, X = ctx.saved_tensors
        gmap: Map = ctx.gmap
        if not gmap.surface_is(X):
            gmap.set_surface(X)
        dq, dX = gmap.query_backward(q, gd.detach(), want_dq=ctx.needs_input_grad[0],
                                     want_dX=ctx.needs_input_grad[1])
        return (dq.to(q.dtype) if dq is not None else None,
                dX.to(X.dtype) if dX is not None else None, None)


def gpdf_distance(q: torch.Tensor, X: torch.Tensor, gmap: Map) -> torch.Tensor:
    """Distance of each query point ``q`` [n, 3] to the surface ``X`` [m, 3] (differentiable in
    both), through the G-GPDF of ``gmap``."""
    return GPDFDistance.apply(q, X, gmap)
