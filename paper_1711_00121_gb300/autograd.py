"""torch.autograd.Function over simrank_grad: a pair loss on SimRank scores as a
differentiable function of the edge weights (forward and backward both run in
libsimrank; this module only moves tensors)."""
from __future__ import annotations

import numpy as np
import torch

from ._binding import SimRank, MODE_COLUMN


class PairLoss(torch.autograd.Function):
    """L(w) = sum_p (S_K[a_p, b_p] - t_p)^2 for the K-truncated SimRank of the
    graph (src -> dst) with edge weights w; backward returns dL/dw."""

    @staticmethod
    def forward(ctx, weight, n, src, dst, a, b, target, C, K):
        w = weight.detach().to("cpu", torch.float32).numpy()
        sr = SimRank(int(n), src, dst, weight=w, C=float(C), K=int(K), s_precision=64,
                     mode=MODE_COLUMN)
        try:
            L, g = sr.grad(a, b, target, w.size)
        finally:
            sr.close()
        ctx.save_for_backward(torch.as_tensor(g, dtype=weight.dtype, device=weight.device))
        return torch.tensor(L, dtype=weight.dtype, device=weight.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return (grad_out * g, None, None, None, None, None, None, None, None)


def pair_loss(weight, n, src, dst, a, b, target, C=0.6, K=20):
    return PairLoss.apply(weight, n, np.asarray(src), np.asarray(dst), np.asarray(a),
                          np.asarray(b), np.asarray(target, np.float64), C, K)
