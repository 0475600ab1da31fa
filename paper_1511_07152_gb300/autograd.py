"""Differentiable gridding and prediction (torch.autograd over the C ABI).

Gridding is C-linear in the visibilities, G = A V, with A the separable
W-projection operator including the weights (Sec. 5); degridding is exactly
its adjoint A^H (the prediction of Sec. 2).  Prediction from a model image I
is V = D A_img I with A_img = IMAGE_TO_GRID (the image divided by n and the
taper, then the shifted DFT) and D degridding with unit weights.

PyTorch's complex autograd propagates conjugate Wirtinger gradients: for a
C-linear y = M x the vector-Jacobian product is grad_x = M^H grad_y.  Hence
  * Grid.backward      = degridding of the incoming gradient;
  * Predict.backward   = gridding (unit weights), then the exact adjoint of
                         IMAGE_TO_GRID; for a real image the real part.
Every step runs in the CUDA library; this module only allocates outputs and
passes pointers.  A plan (sepw_plan) of the visibilities' u, v, w must be
current on the context while the graph is built and differentiated.
"""
from __future__ import annotations

import torch

from . import sepw as S


class Grid(torch.autograd.Function):
    """grid = sum_i W_i V_i F~(u - u_i) (N x N complex64) from vis (complex64)."""

    @staticmethod
    def forward(ctx_, vis, sctx, taps, weight):
        N = sctx.params.grid_size
        grid = torch.zeros((N, N), dtype=torch.complex64, device=vis.device)
        S.sepw_grid_planned(sctx, taps, vis.contiguous(), weight, grid)
        ctx_.sctx, ctx_.taps, ctx_.weight = sctx, taps, weight
        return grid

    @staticmethod
    def backward(ctx_, g):
        out = torch.empty(ctx_.sctx.plan_nvis, dtype=torch.complex64, device=g.device)
        S.sepw_degrid_planned(ctx_.sctx, ctx_.taps, g.contiguous().to(torch.complex64),
                              ctx_.weight, out)
        return out, None, None, None


class Predict(torch.autograd.Function):
    """V_i = sum_pixels I / n exp(-2 pi i (u l + v m)) g~*(l, m) (Sec. 2, pixel
    area omitted) through IMAGE_TO_GRID + separable degridding; the model
    image I is N x N, real (float32) or complex64, indexed [m][l]."""

    @staticmethod
    def forward(ctx_, image, sctx, taps):
        buf = image.detach().to(torch.complex64).contiguous().clone()
        S.sepw_image(sctx, S.IMAGE_TO_GRID, buf)
        out = torch.empty(sctx.plan_nvis, dtype=torch.complex64, device=image.device)
        S.sepw_degrid_planned(sctx, taps, buf, None, out)
        ctx_.sctx, ctx_.taps, ctx_.real = sctx, taps, not image.is_complex()
        return out

    @staticmethod
    def backward(ctx_, g):
        sctx = ctx_.sctx
        N = sctx.params.grid_size
        grid = torch.zeros((N, N), dtype=torch.complex64, device=g.device)
        S.sepw_grid_planned(sctx, ctx_.taps, g.contiguous().to(torch.complex64), None, grid)
        S.sepw_image(sctx, S.IMAGE_TO_GRID_ADJOINT, grid)
        return (grid.real if ctx_.real else grid), None, None


def grid(vis, sctx, taps, weight=None):
    return Grid.apply(vis, sctx, taps, weight)


def predict(image, sctx, taps):
    return Predict.apply(image, sctx, taps)


def chi2(pred, target, weight=None):
    """sum_i W_i |pred_i - target_i|^2 accumulated in float64."""
    r = (pred - target).to(torch.complex128)
    a = r.real * r.real + r.imag * r.imag
    if weight is not None:
        a = a * weight.to(torch.float64)
    return a.sum()
