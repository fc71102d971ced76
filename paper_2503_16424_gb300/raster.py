"""One rasterizer step and its torch.autograd.Function, on top of the binding.

``Rasterizer`` owns the device buffers of a fixed problem (canvas, curve
counts, sampling) and runs the hot path call by call:
  bs_curve_order -> bs_sample_curves -> bs_bin_tiles -> bs_render_fwd
  -> bs_l2_loss_grad -> bs_render_bwd (render backward + sampling backward).
Only the blend state T_final/n_contrib (8 bytes per pixel) is kept between
forward and backward; everything per Gaussian is recomputed.  Every few
hundred steps ``prune_densify`` edits the curve set in place against the
last rendered image (bs_prune_densify); the next forward recomputes the
draw order.
"""

from __future__ import annotations

import torch

from . import bs
from .bs import Binning, Canvas, CurveSet, SampleCfg


class Rasterizer:
    def __init__(self, canvas: Canvas, cfg: SampleCfg, n_open: int, n_closed: int, device="cuda",
                 pair_capacity: int = 1 << 22):
        self.canvas, self.cfg = canvas, cfg
        self.n_open, self.n_closed = n_open, n_closed
        self.n_gauss = bs.num_gaussians(n_open, n_closed, cfg)
        self.device = device
        H, W = canvas.height, canvas.width
        f32 = dict(dtype=torch.float32, device=device)
        self.gauss = torch.empty(self.n_gauss, bs.GAUSS_FLOATS, **f32)
        self.dgauss = torch.empty(self.n_gauss, bs.DGAUSS_FLOATS, **f32)
        self.img = torch.empty(3, H, W, **f32)
        self.T = torch.empty(H, W, **f32)
        self.nc = torch.empty(H, W, dtype=torch.int32, device=device)
        self.dimg = torch.empty(3, H, W, **f32)
        self.loss = torch.empty((), dtype=torch.float64, device=device)
        self.binning = Binning(canvas, device, pair_capacity)
        self.rank = self.first = None
        self.pd_ws = None

    def forward(self, curves: CurveSet):
        self.rank, self.first = bs.curve_order(curves, self.cfg)
        bs.sample_curves(curves, self.cfg, self.first, out=self.gauss)
        self.binning.run(self.gauss)
        bs.render_fwd(self.gauss, self.canvas, self.binning, out=(self.img, self.T, self.nc))
        return self.img

    def backward(self, curves: CurveSet, dimg: torch.Tensor, grad: CurveSet = None):
        dimg = dimg.contiguous()
        _, grad = bs.render_bwd(self.gauss, self.canvas, self.binning, self.T, self.nc, dimg, self.dgauss,
                                curves=curves, cfg=self.cfg, first=self.first, grad=grad)
        return grad

    def step(self, curves: CurveSet, target: torch.Tensor, grad: CurveSet = None, xing: float = 0.0):
        """sample -> bin -> render with the L2 loss/grad fused -> render bwd
        -> sample bwd; with xing > 0 also the Xing term of Eq. 13 (lambda_2 =
        xing; its value in self.xing_loss, its gradient added to the closed
        curves' control points)."""
        self.rank, self.first = bs.curve_order(curves, self.cfg)
        bs.sample_curves(curves, self.cfg, self.first, out=self.gauss)
        self.binning.run(self.gauss)
        bs.render_fwd_l2(self.gauss, self.canvas, self.binning, target, out=(self.img, self.T, self.nc),
                         dimg=self.dimg, loss=self.loss)
        grad = self.backward(curves, self.dimg, grad)
        if xing > 0.0:
            self.xing_loss = bs.xing_loss(curves, xing, grad.closed_ctrl)
        return self.loss, grad


    def prune_densify(self, curves: CurveSet, target: torch.Tensor, cfg: bs.PDCfg, img: torch.Tensor = None):
        """One pruning/densification pass against `img` (default: the last
        forward's image).  Returns (changed mask, counts)."""
        img = self.img if img is None else img
        if self.pd_ws is None:
            n = bs.prune_densify_workspace(self.n_open, self.n_closed, self.canvas)
            self.pd_ws = torch.empty(n, dtype=torch.uint8, device=self.device)
        return bs.prune_densify(curves, img, target, cfg, self.canvas, ws=self.pd_ws)


class BezierRasterize(torch.autograd.Function):
    """img = render(curves).  Inputs are the seven curve tensors of CurveSet
    (pixel space, activated values); the backward returns their gradients."""

    @staticmethod
    def forward(ctx, rasterizer: Rasterizer, open_ctrl, open_width, open_color, open_opac,
                closed_ctrl, closed_color, closed_opac):
        curves = CurveSet(*(t.detach().contiguous() for t in (open_ctrl, open_width, open_color, open_opac,
                                                               closed_ctrl, closed_color, closed_opac)))
        img = rasterizer.forward(curves).clone()
        ctx.rasterizer = rasterizer
        ctx.curves = curves
        return img

    @staticmethod
    def backward(ctx, dimg):
        g = ctx.rasterizer.backward(ctx.curves, dimg)
        return (None, g.open_ctrl, g.open_width, g.open_color, g.open_opac,
                g.closed_ctrl, g.closed_color, g.closed_opac)


def rasterize(rasterizer: Rasterizer, curves: CurveSet) -> torch.Tensor:
    return BezierRasterize.apply(rasterizer, *(getattr(curves, k) for k in bs.CURVE_FIELDS))
