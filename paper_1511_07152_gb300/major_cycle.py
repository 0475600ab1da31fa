"""Least-squares major cycles over the C ABI.

Imaging as weighted least squares, min over real images x of
    chi^2(x) = sum_i W_i |(M x)_i - V_i|^2,
with M the prediction (IMAGE_TO_GRID then separable degridding, Sec. 2) and
M^H its adjoint (separable gridding then the adjoint image step), solved by
conjugate gradients on the normal equations.  Each cycle degrids the
visibilities of a search direction and grids them back: the alternation of
major cycles (Sec. 6, where the plan of the visibilities is reused across
cycles), with the least-squares model update in place of a CLEAN minor cycle.

CG runs on y with x = D y, D = n c1 c1 the grid correction: M divides the
image by n c1 c1 (up to 1e8 at the edge for support 16), which unconditioned
FP32 CG does not survive; M D is prediction without that division.

Every gridding, degridding and FFT step runs in the CUDA library through the
context's current plan (sepw_plan of the visibilities' u, v, w); this module
holds the CG vectors as torch tensors and takes their inner products in
float64.
"""
from __future__ import annotations

import torch

from . import sepw as S


class _Operators:
    """M D and D M^H on preallocated buffers of one context and plan."""

    def __init__(self, ctx: S.Context, taps):
        self.ctx, self.taps = ctx, taps
        p = ctx.params
        N = p.grid_size
        dev = taps.device
        self.buf = torch.empty((N, N), dtype=torch.complex64, device=dev)
        c = S.sepw_taper(ctx).double()
        l = (torch.arange(N, device=dev, dtype=torch.float64) - N // 2) * (p.fov / N)
        n = torch.sqrt(1.0 - l[None, :] ** 2 - l[:, None] ** 2)
        self.D = (n * c[None, :] * c[:, None]).float()

    def predict(self, y, out):
        """out (complex64 [nvis]) = M D y for a real image y [N][N]."""
        self.buf.copy_(y * self.D)
        S.sepw_image(self.ctx, S.IMAGE_TO_GRID, self.buf)
        S.sepw_degrid_planned(self.ctx, self.taps, self.buf, None, out)
        return out

    def adjoint(self, r, weight, out):
        """out (float32 [N][N]) = Re(D M^H W r)."""
        self.buf.zero_()
        S.sepw_grid_planned(self.ctx, self.taps, r, weight, self.buf)
        S.sepw_image(self.ctx, S.IMAGE_TO_GRID_ADJOINT, self.buf)
        torch.mul(self.buf.real, self.D, out=out)
        return out


def _dot(a, b) -> float:
    return float(torch.sum(a.double() * b.double()))


def _chi2(r, weight) -> float:
    a = r.real.double() ** 2 + r.imag.double() ** 2
    if weight is not None:
        a = a * weight.double()
    return float(a.sum())


def cg_major_cycles(ctx: S.Context, taps, vis, weight, n_cycles: int, x0=None):
    """n_cycles conjugate-gradient major cycles from x0 (zero image if None).

    vis: complex64 [nvis] (the plan's visibilities, in plan order); weight:
    float32 [nvis] or None.  Returns (x float32 [N][N], chi^2 after each cycle
    starting with chi^2(x0)).  The prediction of the current model is updated
    by linearity, so a cycle costs one degridding and one gridding."""
    N = ctx.params.grid_size
    dev = vis.device
    ops = _Operators(ctx, taps)
    x = torch.zeros((N, N), dtype=torch.float32, device=dev) if x0 is None \
        else (x0.to(torch.float32) / ops.D)  # CG runs on y = x / D
    pred = torch.empty_like(vis)
    md = torch.empty_like(vis)
    r = torch.empty((N, N), dtype=torch.float32, device=dev)
    q = torch.empty_like(r)
    ops.predict(x, pred)
    ops.adjoint(vis - pred, weight, r)
    d = r.clone()
    rr = _dot(r, r)
    losses = [_chi2(pred - vis, weight)]
    for _ in range(n_cycles):
        ops.predict(d, md)
        ops.adjoint(md, weight, q)
        dq = _dot(d, q)
        if dq <= 0.0 or rr == 0.0:
            break
        alpha = rr / dq
        x.add_(d, alpha=alpha)
        pred.add_(md, alpha=alpha)
        r.sub_(q, alpha=alpha)
        rr_new = _dot(r, r)
        d.mul_(rr_new / rr).add_(r)
        rr = rr_new
        losses.append(_chi2(pred - vis, weight))
    return x * ops.D, losses
