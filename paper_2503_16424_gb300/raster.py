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

``StepGraph`` captures one whole step of one canvas (with the binning that
reads nothing back, bs_bin_tiles_async) and an optional update after it as
one CUDA graph.
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
        n = n_open + n_closed
        self.rank = torch.empty(n, dtype=torch.int32, device=device)
        self.first = torch.empty(n, dtype=torch.int32, device=device)
        self.binning = Binning(canvas, device, pair_capacity)
        self.pd_ws = None
        # forwards run so far: the buffers hold the state of the last one
        self.generation = 0

    def _bin(self, sync: bool):
        if sync:
            self.binning.run(self.gauss)
        else:
            self.binning.run_async(self.gauss)

    def forward(self, curves: CurveSet, sync: bool = True):
        bs.curve_order(curves, self.cfg, out=(self.rank, self.first))
        bs.sample_curves(curves, self.cfg, self.first, out=self.gauss)
        self._bin(sync)
        bs.render_fwd(self.gauss, self.canvas, self.binning, out=(self.img, self.T, self.nc))
        self.generation += 1
        return self.img

    def backward(self, curves: CurveSet, dimg: torch.Tensor, grad: CurveSet = None):
        dimg = dimg.contiguous()
        _, grad = bs.render_bwd(self.gauss, self.canvas, self.binning, self.T, self.nc, dimg, self.dgauss,
                                curves=curves, cfg=self.cfg, first=self.first, grad=grad)
        return grad

    def step(self, curves: CurveSet, target: torch.Tensor, grad: CurveSet = None, xing: float = 0.0,
             sync: bool = True):
        """sample -> bin -> render with the L2 loss/grad fused -> render bwd
        -> sample bwd; with xing > 0 also the Xing term of Eq. 13 (lambda_2 =
        xing; its value in self.xing_loss, its gradient added to the closed
        curves' control points).  sync=False bins with no read-back (the
        buffers must be sized, Binning.prepare), so the step can be captured."""
        bs.curve_order(curves, self.cfg, out=(self.rank, self.first))
        bs.sample_curves(curves, self.cfg, self.first, out=self.gauss)
        self._bin(sync)
        bs.render_fwd_l2(self.gauss, self.canvas, self.binning, target, out=(self.img, self.T, self.nc),
                         dimg=self.dimg, loss=self.loss)
        self.generation += 1
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


class StepGraph:
    """One optimisation step of one canvas as one CUDA graph replay: draw
    order, sampling, binning with no read-back (bs_bin_tiles_async), blend
    with the fused L2 loss, the backward to the curves, then `after()` (for
    instance an Adam step) if given.

    The first call runs the step eagerly with the synchronising binning and
    fits the pair capacity to `headroom` times the pairs found (growing or
    shrinking it: the captured binning's grids are sized by it); the graph is
    captured on the second call and replayed from then on.  check() reads the
    binning's outcome (one synchronisation): a replay whose pairs overflowed
    the capacity blended nothing, so the capacity is grown and the graph
    captured again at the next call; so is it whenever the binning's buffers
    were allocated anew since the capture (a synchronising call in between,
    Rasterizer.forward for instance, grows them when its pairs overflow).
    Curves, target and grad must keep their storage (the graph holds their
    addresses)."""

    def __init__(self, rast: Rasterizer, curves: CurveSet, target: torch.Tensor, grad: CurveSet, after=None,
                 headroom: float = 1.25):
        self.r, self.curves, self.target, self.grad, self.after = rast, curves, target, grad, after
        self.headroom = headroom
        self.graph = None
        self.calls = 0
        self.overflows = 0
        self._allocations = None   # the binning's allocation count the graph was captured with

    def _eager_fit(self):
        r = self.r
        r.step(self.curves, self.target, self.grad)
        r.binning.fit(r.n_gauss, int(r.binning.n_pairs * self.headroom) + 1024)
        if self.after is not None:
            self.after()

    def _capture(self):
        self._allocations = self.r.binning.allocations
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                self.r.step(self.curves, self.target, self.grad, sync=False)
                if self.after is not None:
                    self.after()
        torch.cuda.current_stream().wait_stream(side)

    def __call__(self):
        if self.calls == 0:
            self._eager_fit()
        else:
            if self.graph is None or self._allocations != self.r.binning.allocations:
                self._capture()
            self.graph.replay()
        self.calls += 1

    def check(self):
        """(status, pairs) of the last binning; on an overflow the capacity
        grows and the next call captures again.  Synchronises."""
        st, n_pairs = self.r.binning.result()
        if st == bs.BS_ERR_CAPACITY:
            self.overflows += 1
            self.r.binning.prepare(self.r.n_gauss, int(n_pairs * 1.5) + 4096)
            self.graph = None   # captured again at the next call
        return st, n_pairs


class BezierRasterize(torch.autograd.Function):
    """img = render(curves).  Inputs are the seven curve tensors of CurveSet
    (pixel space, activated values); the backward returns their gradients.

    The rasterizer's buffers hold the state of its latest forward.  When
    another forward has run on the same rasterizer since this call's (two
    renders in one loss, re-entrant checkpointing), the backward first
    recomputes this call's forward state from its saved inputs (draw order,
    sampling, binning and blend are deterministic: the same bits), then
    walks back."""

    @staticmethod
    def forward(ctx, rasterizer: Rasterizer, open_ctrl, open_width, open_color, open_opac,
                closed_ctrl, closed_color, closed_opac):
        inputs = (open_ctrl, open_width, open_color, open_opac, closed_ctrl, closed_color, closed_opac)
        curves = CurveSet(*(t.detach().contiguous() for t in inputs))
        img = rasterizer.forward(curves).clone()
        ctx.rasterizer = rasterizer
        ctx.generation = rasterizer.generation
        ctx.save_for_backward(*inputs)
        return img

    @staticmethod
    def backward(ctx, dimg):
        r = ctx.rasterizer
        curves = CurveSet(*(t.detach().contiguous() for t in ctx.saved_tensors))
        if r.generation != ctx.generation:
            r.forward(curves)
            ctx.generation = r.generation
        g = r.backward(curves, dimg)
        return (None, g.open_ctrl, g.open_width, g.open_color, g.open_opac,
                g.closed_ctrl, g.closed_color, g.closed_opac)


def rasterize(rasterizer: Rasterizer, curves: CurveSet) -> torch.Tensor:
    return BezierRasterize.apply(rasterizer, *(getattr(curves, k) for k in bs.CURVE_FIELDS))
