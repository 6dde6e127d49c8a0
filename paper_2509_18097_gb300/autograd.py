"""torch.autograd.Function over the library's hand-written forward and backward kernels.

`GridLoss.apply(fitter_ctx, *thetas)` returns the frame loss
    L(theta) = w_mesh CD_R(X_hat, P_t) + w_pts CD_R(P_hat, P_t) + w_iso L_iso
(Sec. 3.4) as a float64 scalar tensor; its backward is dL/dtheta_l for every level, computed
by the kernels (trilinear adjoint of Eq. 1, robust-Chamfer gradient, isometry gradient), not
by torch.  The context must be inside a frame (pdg_begin_frame); the grids are written into
it for the evaluation.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class GridLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, handle, *thetas):
        res = []
        for l, th in enumerate(thetas):
            t = th.detach().to(torch.float32).contiguous().reshape(-1, 3)
            if t.is_cuda:
                B.pdg_write_theta(handle, l, t)
            else:
                B.pdg_write_theta(handle, l, t.numpy())
            res.append(th.shape)
        loss = B.pdg_eval(handle)
        grads = []
        for l, shp in enumerate(res):
            n3 = int(np.prod(shp[:-1]))
            dev = thetas[l].device
            g = torch.empty((n3, 3), dtype=torch.float32, device=dev if dev.type == "cuda" else "cpu")
            B.pdg_read(handle, B.BUF_GRAD, l, g if g.is_cuda else g.numpy())
            grads.append(g.reshape(shp).to(thetas[l].dtype))
        fctx.save_for_backward(*grads)
        return torch.tensor(loss[0], dtype=torch.float64, device=thetas[0].device)

    @staticmethod
    def backward(fctx, grad_out):
        grads = fctx.saved_tensors
        return (None, *[g * grad_out.to(g.dtype) for g in grads])


def grid_loss(handle, thetas):
    """Loss at the given per-level grids ([n, n, n, 3] tensors) with autograd support."""
    return GridLoss.apply(handle, *thetas)
