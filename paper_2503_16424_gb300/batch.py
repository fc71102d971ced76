"""Many images optimised together, on top of the binding's batched calls.

``BatchRasterizer`` owns the device buffers of a batch (images of different
sizes and curve counts, concatenated image after image) and runs one step:
  bs_batch_curve_order -> bs_batch_sample_curves -> bs_batch_bin_tiles
  -> bs_batch_render_fwd (blend + per-image L2 loss and gradient)
  -> bs_batch_render_bwd (blend backward + sampling backward).
Each kernel covers every image of the batch in one launch; the blend
kernels are persistent and take (image, tile) items from an atomic queue.

``BatchOptimizer`` adds Adam (bs_adam_step) and captures the whole step in
a CUDA graph: no call of the step synchronises or reads a value back, and
the Adam step counter lives on the device, so one graph replay is one
optimisation step of every image.  ``PlainOptimizer`` is the same
optimisation run image by image through the single-canvas calls, for
comparison.

Learning rates (Section 4.1 gives 2e-4 for control points in [-1, 1]
coordinates, 0.01 for colour and 0.1 for opacity, both before a sigmoid).
The calls take pixel coordinates and activated values, so the step sizes
are carried over: control points 2e-4 x (half the image's longer side) px,
colour 0.01 / 4 and opacity 0.1 / 4 (the sigmoid's largest slope is 1/4),
width 0.01 px (not given in the paper).  Colours and opacities are kept in
[0, 1], widths >= 0.1 px.
"""

from __future__ import annotations

from dataclasses import dataclass

import torch

from . import bs
from .bs import Batch, BatchImage, CurveSet  # noqa: F401

CURVE_FIELDS = bs.CURVE_FIELDS


@dataclass
class AdamCfg:
    lr_ctrl: float = 2e-4       # per unit of half the longer image side
    lr_color: float = 0.01 / 4
    lr_opac: float = 0.1 / 4
    lr_width: float = 0.01
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    width_min: float = 0.1


class BatchRasterizer:
    """Device buffers and the step of one batch."""

    def __init__(self, images, tile: int = 16, pair_capacity: int = 1 << 22, device="cuda"):
        self.batch = Batch(images, tile, pair_capacity, device)
        self.device = device
        b = self.batch
        f32 = dict(dtype=torch.float32, device=device)
        self.gauss = torch.empty(max(1, b.n_gauss), bs.GAUSS_FLOATS, **f32)[:b.n_gauss]
        self.dgauss = torch.empty(max(1, b.n_gauss), bs.DGAUSS_FLOATS, **f32)[:b.n_gauss]
        self.img = torch.empty(3 * b.n_pixels, **f32)
        self.dimg = torch.empty(3 * b.n_pixels, **f32)
        self.T = torch.empty(b.n_pixels, **f32)
        self.nc = torch.empty(b.n_pixels, dtype=torch.int32, device=device)
        self.loss = torch.empty(len(b.images), dtype=torch.float64, device=device)
        n_curves = b.n_open + b.n_closed
        self.rank = torch.empty(max(1, n_curves), dtype=torch.int32, device=device)[:n_curves]
        self.first = torch.empty(max(1, n_curves), dtype=torch.int32, device=device)[:n_curves]
        self.ranges = torch.empty(b.n_tiles, 2, dtype=torch.int32, device=device)
        self.vals = torch.empty(b.pair_capacity, dtype=torch.int32, device=device)

    def forward(self, curves: CurveSet, target: torch.Tensor = None):
        b = self.batch
        b.curve_order(curves, self.rank, self.first)
        b.sample_curves(curves, self.first, out=self.gauss)
        b.bin_tiles(self.gauss, self.vals, self.ranges)
        if target is None:
            b.render_fwd(self.gauss, self.vals, self.ranges, self.img, self.T, self.nc)
        else:
            b.render_fwd(self.gauss, self.vals, self.ranges, self.img, self.T, self.nc, target, self.dimg,
                         self.loss)
        return self.img

    def backward(self, curves: CurveSet, dimg: torch.Tensor, grad: CurveSet):
        self.batch.render_bwd(self.gauss, self.vals, self.ranges, self.T, self.nc, dimg, self.dgauss, curves,
                              self.first, grad)
        return grad

    def step(self, curves: CurveSet, target: torch.Tensor, grad: CurveSet):
        """One step of every image: per-image loss in self.loss, curve
        gradients in grad."""
        self.forward(curves, target)
        return self.backward(curves, self.dimg, grad)

    def fit_capacity(self, curves: CurveSet, headroom: float = 1.5):
        """Bin once and grow the pair capacity to headroom x the pairs found
        when they do not fit (synchronises)."""
        b = self.batch
        b.curve_order(curves, self.rank, self.first)
        b.sample_curves(curves, self.first, out=self.gauss)
        b.bin_tiles(self.gauss, self.vals, self.ranges)
        st, n_pairs = b.status()
        if st != bs.BS_OK:
            self.grow(int(n_pairs * headroom) + 4096)
        return n_pairs

    def grow(self, pair_capacity: int):
        self.batch.grow(pair_capacity)
        self.vals = torch.empty(self.batch.pair_capacity, dtype=torch.int32, device=self.device)

    def psnr(self, target: torch.Tensor):
        """Per-image PSNR (dB, peak 1) of the last forward against target."""
        out = []
        for i in range(len(self.batch.images)):
            d = self.batch.image(self.img, i) - self.batch.image(target, i)
            mse = float((d.double() ** 2).mean())
            out.append(float("inf") if mse == 0 else -10.0 * torch.log10(torch.tensor(mse)).item())
        return out


def partition_images(weights, world: int):
    """The images each of `world` ranks optimises when a batch is split
    across GPUs (independent images: no exchange between ranks).  Longest
    processing time first: images by descending weight (pixel count; equal
    weights by index) each go to the rank with the least weight so far (the
    lowest rank on a tie).  Returns one ascending index list per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += weights[i]
    return [sorted(p) for p in parts]


def _curve_scales(images, field_rows, device):
    """Per-curve control-point lr multipliers: half the longer side of the
    curve's image, for the open (field_rows = 'open') or closed curves."""
    vals = []
    for im in images:
        n = im.n_open if field_rows == "open" else im.n_closed
        vals += [0.5 * max(im.width, im.height)] * n
    return torch.tensor(vals, dtype=torch.float32, device=device)


class CurveAdam:
    """Adam state of a curve set and its bs_adam_step groups."""

    def __init__(self, curves: CurveSet, grad: CurveSet, images, cfg: AdamCfg, device):
        self.cfg = cfg
        self.m = curves.zeros_like()
        self.v = curves.zeros_like()
        self.t = torch.zeros(1, dtype=torch.int32, device=device)
        self.s_open = _curve_scales(images, "open", device)
        self.s_closed = _curve_scales(images, "closed", device)
        big = 3.0e38
        spec = {
            "open_ctrl": (cfg.lr_ctrl, -big, big, self.s_open, 20),
            "closed_ctrl": (cfg.lr_ctrl, -big, big, self.s_closed, 24),
            "open_width": (cfg.lr_width, cfg.width_min, big, None, 1),
            "open_color": (cfg.lr_color, 0.0, 1.0, None, 1),
            "open_opac": (cfg.lr_opac, 0.0, 1.0, None, 1),
            "closed_color": (cfg.lr_color, 0.0, 1.0, None, 1),
            "closed_opac": (cfg.lr_opac, 0.0, 1.0, None, 1),
            "closed_color2": (cfg.lr_color, 0.0, 1.0, None, 1),
            "closed_opac2": (cfg.lr_opac, 0.0, 1.0, None, 1),
        }
        self.groups = []
        for k, (lr, lo, hi, rs, rl) in spec.items():
            p = getattr(curves, k)
            if p is None or p.numel() == 0:
                continue
            self.groups.append(bs.AdamGroup(p, getattr(grad, k), getattr(self.m, k), getattr(self.v, k), lr, lo, hi,
                                            rs, rl))

    def step(self):
        bs.adam_step(self.groups, self.t, self.cfg.beta1, self.cfg.beta2, self.cfg.eps)


class BatchOptimizer:
    """Adam on every image of a batch; with graph=True the whole step
    (draw order, sampling, binning, blend + loss, backward, Adam) is one
    CUDA graph replay.  The first step runs eagerly and fits the pair
    capacity; the graph is captured on the second.  Every check_every steps
    the binning status is read (one synchronisation); a step whose pairs
    overflowed the capacity renders nothing, so the capacity is then grown
    and the graph captured again."""

    def __init__(self, rast: BatchRasterizer, curves: CurveSet, target: torch.Tensor, cfg: AdamCfg = None,
                 graph: bool = True, check_every: int = 50):
        self.rast, self.curves, self.target = rast, curves, target
        self.cfg = cfg or AdamCfg()
        self.grad = curves.zeros_like()
        self.adam = CurveAdam(curves, self.grad, rast.batch.images, self.cfg, rast.device)
        self.use_graph = graph
        self.check_every = check_every
        self.graph = None
        self.steps = 0
        self.overflows = 0

    def _step(self):
        self.rast.step(self.curves, self.target, self.grad)
        self.adam.step()

    def _capture(self):
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                self._step()
        torch.cuda.current_stream().wait_stream(side)

    def step(self):
        if self.steps == 0:
            self.rast.fit_capacity(self.curves)
            self._step()
        elif not self.use_graph:
            self._step()
        else:
            if self.graph is None:
                self._capture()
            self.graph.replay()
        self.steps += 1
        if self.check_every and self.steps % self.check_every == 0:
            self.check()

    def check(self):
        st, n_pairs = self.rast.batch.status()
        if st != bs.BS_OK:
            self.overflows += 1
            self.rast.grow(int(n_pairs * 1.5) + 4096)
            self.graph = None
        return st, n_pairs


class PlainOptimizer:
    """The same optimisation image by image through the single-canvas calls
    (bs_curve_order ... bs_render_bwd, then bs_adam_step per image).  With
    graph=True each image's step and Adam update is one CUDA-graph replay
    (raster.StepGraph), so the comparison with the batch is not about host
    launches."""

    def __init__(self, images, curves_per_image, targets, cfg: AdamCfg = None, device="cuda",
                 pair_capacity: int = 1 << 20, tile: int = 16, graph: bool = False, headroom: float = 1.25):
        from .raster import Rasterizer, StepGraph
        self.cfg = cfg or AdamCfg()
        self.items = []
        self.graphs = []
        for im, cv, tg in zip(images, curves_per_image, targets):
            r = Rasterizer(bs.Canvas(im.width, im.height, tile, im.bg), im.sample, im.n_open, im.n_closed,
                           device=device, pair_capacity=pair_capacity)
            grad = cv.zeros_like()
            adam = CurveAdam(cv, grad, [im], self.cfg, device)
            self.items.append((r, cv, tg, grad, adam))
            if graph:
                self.graphs.append(StepGraph(r, cv, tg, grad, after=adam.step, headroom=headroom))

    def step(self):
        if self.graphs:
            for g in self.graphs:
                g()
            return
        for r, cv, tg, grad, adam in self.items:
            r.step(cv, tg, grad)
            adam.step()

    def check(self):
        """Read every image's binning status (synchronises); regrow where a
        captured step overflowed."""
        return [g.check() for g in self.graphs]

    def losses(self):
        """Each image's loss of its last step (device doubles)."""
        return torch.stack([r.loss for r, *_ in self.items])


def main():
    """Optimise the 64-image ragged workload (synth.BATCH_WORKLOAD, each image
    sampled by the autotuner's spacing rule) with BatchOptimizer: one eager
    step, one captured step, then graph replays; prints one JSON line with
    the ms per replayed step.  The batched step's launch list is taken on
    this command."""
    import argparse
    import json

    import numpy as np

    from . import autotune, synth
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--steps", type=int, default=5, help="steps in all (at least 3)")
    ap.add_argument("--tile", type=int, default=16, choices=(8, 16, 32))
    args = ap.parse_args()
    steps = max(3, args.steps)
    dev = torch.device("cuda", 0)
    W = synth.BATCH_WORKLOAD
    layout = synth.batch_layout(W["seed"], W["n_images"], W["side"], W["aspect"], W["curves"])
    arrs, cat, targets = synth.batch_inputs(layout, W["n_shapes"])
    base = [BatchImage(e["W"], e["H"], e["n_open"], e["n_closed"], bs.SampleCfg()) for e in layout]
    images = autotune.with_sampling(base, autotune.spacing_sampling(base, arrs))
    target = torch.as_tensor(np.concatenate([t.reshape(-1) for t in targets]), device=dev)
    curves = CurveSet.from_arrays(cat, device=dev)
    rast = BatchRasterizer(images, tile=args.tile, pair_capacity=1 << 24, device=dev)
    opt = BatchOptimizer(rast, curves, target, graph=True, check_every=0)
    opt.step()
    opt.step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps - 2):
        opt.step()
    e1.record()
    torch.cuda.synchronize()
    st, n_pairs = rast.batch.status()
    print(json.dumps({"workload": W["name"], "images": len(images), "gaussians": rast.batch.n_gauss,
                      "pairs": n_pairs, "binning_status": st, "tile": args.tile,
                      "ms_per_step": round(e0.elapsed_time(e1) / (steps - 2), 4)}))


if __name__ == "__main__":
    main()
