"""Optimisation runs of the method on one canvas (Section 3.5, Algorithm 1;
the Section 4.1 schedule).

``fit`` optimises a curve set against a target image: every step is one
replay of a ``StepGraph`` (draw order, sampling, binning, blend with the L2
loss of Eq. 13, backward to the curves) followed by Adam (bs_adam_step), the
whole step one CUDA graph.  Every ``prune_every`` steps (from
``prune_every`` up to ``prune_stop``) one pruning and densification pass
(bs_prune_densify) edits the curves in place against the image of the
current curves, outside the graph.  The opacity threshold of the pass
decays linearly from ``pd.op_start`` to ``pd.op_end`` over the run (t_end =
the number of steps).  A curve the pass replaced or split starts with
zeroed Adam moments (reading: the paper does not say; a new curve has no
gradient history).  After a pass the pair capacity is checked against the
new curves' binning and the graph captured again when it has to grow.

The loss of every step is kept on the device (one 8-byte copy a step) and
read once at the end.

python -m paper_2503_16424_gb300.fit --workload mid_1024_768 --iters 500
python -m paper_2503_16424_gb300.fit --workload hires_2048_4096 --iters 2000 --prune-every 200
print one JSON line: the PSNR curve, wall-clock, steps per second and the
counts of every pass.
"""

from __future__ import annotations

import math
import time
from dataclasses import dataclass, field, replace

import torch

from . import bs
from .batch import AdamCfg, CurveAdam
from .raster import Rasterizer, StepGraph


@dataclass
class FitCfg:
    iters: int = 500
    prune_every: int = 0            # steps between passes; 0: no pass
    prune_stop: int = None          # no pass after this step (default: the last step)
    pd: bs.PDCfg = field(default_factory=bs.PDCfg)
    adam: AdamCfg = field(default_factory=AdamCfg)
    check_every: int = 50           # steps between reads of the binning status
    headroom: float = 1.25          # pair capacity over the pairs found


def psnr_of_mse(mse: float) -> float:
    """PSNR in dB for images in [0, 1] (peak 1)."""
    return float("inf") if mse <= 0 else -10.0 * math.log10(mse)


def _reset_moments(adam: CurveAdam, changed: torch.Tensor, n_open: int):
    """Zero the Adam moments of the curves a pass changed (an element-wise
    masked fill; boolean indexing would gather the indices first)."""
    ch_open, ch_closed = changed[:n_open].bool(), changed[n_open:].bool()
    for st in (adam.m, adam.v):
        for k in bs.CURVE_FIELDS + bs.FILL_FIELDS:
            t = getattr(st, k)
            if t is None or t.numel() == 0:
                continue
            mask = ch_open if k.startswith("open") else ch_closed
            t.masked_fill_(mask.view(-1, *([1] * (t.dim() - 1))), 0.0)


def fit(rast: Rasterizer, curves: bs.CurveSet, target: torch.Tensor, cfg: FitCfg, pass_hook=None) -> dict:
    """Run cfg.iters steps; returns dict(loss [iters] per-step L2 loss (of
    the curves before that step's update), passes [list of counts], wall_s,
    steps_per_s, overflows).  pass_hook(step, before, img, changed, stats,
    after), when given, is called after every pass with host copies of the
    curves before and after it and of the image it was run against."""
    dev = rast.device
    im = bs.BatchImage(rast.canvas.width, rast.canvas.height, rast.n_open, rast.n_closed, rast.cfg)
    grad = curves.zeros_like()
    adam = CurveAdam(curves, grad, [im], cfg.adam, dev)
    sg = StepGraph(rast, curves, target, grad, after=adam.step, headroom=cfg.headroom)
    hist = torch.zeros(cfg.iters, dtype=torch.float64, device=dev)
    stop = cfg.iters if cfg.prune_stop is None else cfg.prune_stop
    passes = []
    if cfg.prune_every:
        # the torch element-wise kernels of the moment reset load on their
        # first use (seconds on a fresh process): once here, on a mask that
        # changes nothing, so the timed run holds only the method's work
        _reset_moments(adam, torch.zeros(rast.n_open + rast.n_closed, dtype=torch.uint8, device=dev), rast.n_open)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(cfg.iters):
        sg()
        hist[it].copy_(rast.loss)
        step = it + 1
        if cfg.check_every and step % cfg.check_every == 0:
            sg.check()
        if cfg.prune_every and step % cfg.prune_every == 0 and step < min(stop, cfg.iters):
            host = (lambda c: {k: getattr(c, k).cpu().numpy().copy() for k in c.fields()}) if pass_hook else None
            before = host(curves) if host else None
            img = rast.forward(curves)                     # the image of the current curves
            img_host = img.cpu().numpy().copy() if pass_hook else None
            pd = replace(cfg.pd, step=step, t_end=cfg.iters)
            changed, stats = rast.prune_densify(curves, target, pd)
            _reset_moments(adam, changed, rast.n_open)
            passes.append(dict(step=step, **stats))
            rast.forward(curves)                           # the new curves' pairs, read back
            # room for the new curves' pairs (new buffers: the step graph
            # captures again at its next call)
            rast.binning.fit(rast.n_gauss, int(rast.binning.n_pairs * cfg.headroom) + 1024)
            if pass_hook:
                pass_hook(step, before, img_host, changed.cpu().numpy().copy(), stats, host(curves))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st, n_pairs = sg.check()
    loss = hist.cpu().numpy()
    return dict(loss=loss, passes=passes, wall_s=wall, steps_per_s=cfg.iters / wall, overflows=sg.overflows,
                binning_status=st, pairs=n_pairs)


def main():
    import argparse
    import json

    import numpy as np

    from . import synth
    ap = argparse.ArgumentParser(description="Optimise one synthetic workload; prints one JSON line.")
    ap.add_argument("--workload", default="mid_1024_768", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--prune-every", type=int, default=0)
    ap.add_argument("--log-every", type=int, default=50)
    ap.add_argument("--tangent-mode", type=int, default=0, choices=(0, 1))
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    w = synth.WORKLOADS[args.workload]
    arrays = synth.make_curves(w["seed"], w["W"], w["H"], w["n_open"], w["n_closed"], style=w["style"]).as_dict()
    target = torch.as_tensor(synth.procedural_target(w["seed"] + 1, w["W"], w["H"], w.get("n_shapes", 40)),
                             device=dev)
    cfg = bs.SampleCfg(g_open=w["g_open"], rows_closed=w["rows_closed"], k_closed=w["k_closed"],
                       tangent_mode=args.tangent_mode)
    curves = bs.CurveSet.from_arrays(arrays, device=dev)
    rast = Rasterizer(bs.Canvas(w["W"], w["H"], w["tile"]), cfg, curves.n_open, curves.n_closed, device=dev,
                      pair_capacity=1 << 22)
    res = fit(rast, curves, target, FitCfg(iters=args.iters, prune_every=args.prune_every))
    loss = res["loss"]
    every = max(1, args.log_every)
    curve = [(i + 1, round(psnr_of_mse(float(loss[i])), 3)) for i in range(every - 1, args.iters, every)]
    rast.forward(curves)
    final = psnr_of_mse(float(((rast.img - target).double() ** 2).mean()))
    print(json.dumps({
        "workload": args.workload, "W": w["W"], "H": w["H"], "n_open": w["n_open"], "n_closed": w["n_closed"],
        "gaussians": rast.n_gauss, "iters": args.iters, "prune_every": args.prune_every,
        "tangent_mode": args.tangent_mode,
        "psnr_first_db": round(psnr_of_mse(float(loss[0])), 3), "psnr_final_db": round(final, 3),
        "psnr_curve": curve, "wall_s": round(res["wall_s"], 3), "steps_per_s": round(res["steps_per_s"], 2),
        "ms_per_step": round(1e3 * res["wall_s"] / args.iters, 4), "passes": res["passes"],
        "overflows": res["overflows"], "pairs_last": res["pairs"],
        "loss_monotone_frac": round(float(np.mean(np.diff(loss) <= 0)), 3)}), flush=True)


if __name__ == "__main__":
    main()
