"""One optimisation step of the rasterizer, end to end, in fp64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

sample (Section 3.3) -> blend every pixel over every Gaussian (Section 3.4)
-> L2 loss (Eq. 13) -> gradients.  The gradients are taken in the same two
stages the rasterizer uses: first the vector-Jacobian product of the blend
with respect to the Gaussian table (render_grads), then the product of that
with the Jacobian of the sampling with respect to the curve parameters
(autograd through curves.gaussian_table).
"""

from __future__ import annotations

import numpy as np
import torch

from .curves import SampleCfg, gaussian_table
from .loss import l2_loss
from .raster import GRAD_KEYS, render_grads, render_image

CURVE_KEYS = ("open_ctrl", "open_width", "open_color", "open_opac",
              "closed_ctrl", "closed_color", "closed_opac")


FILL_KEYS = ("closed_color2", "closed_opac2")


def as_curves(d: dict, requires_grad=False):
    out = {}
    for k in CURVE_KEYS + FILL_KEYS:
        if k in d and d[k] is not None:
            v = torch.as_tensor(np.asarray(d[k]), dtype=torch.float64).clone()
            out[k] = v.requires_grad_(requires_grad)
    return out


def sample_vjp(curves: dict, cfg: SampleCfg, dtab: dict, first=None):
    """dL/d(curve parameters) given dL/d(table field) for the fields of
    GRAD_KEYS (mx, my, ux, uy, isx, isy, o, col)."""
    cv = {k: v.detach().clone().requires_grad_(True) for k, v in curves.items()}
    tab = gaussian_table(cv, cfg, first)
    outs = [tab[k] for k in GRAD_KEYS]
    grads = [torch.as_tensor(dtab[k], dtype=torch.float64) for k in GRAD_KEYS]
    keys = [k for k in CURVE_KEYS + FILL_KEYS if k in cv]
    gs = torch.autograd.grad(outs, [cv[k] for k in keys], grad_outputs=grads, allow_unused=True)
    return {k: (g if g is not None else torch.zeros_like(cv[k])) for k, g in zip(keys, gs)}


def step(curves: dict, cfg: SampleCfg, W: int, H: int, target, bg=(0.0, 0.0, 0.0),
         with_grads=True):
    """Loss, image, per-Gaussian gradients and curve gradients of one step."""
    with torch.no_grad():
        tab = gaussian_table({k: v.detach() for k, v in curves.items()}, cfg)
    out = render_image(tab, W, H, bg)
    loss, dimg = l2_loss(out["img"], target)
    res = dict(loss=float(loss), img=out["img"], T=out["T"], last=out["last"],
               flag=out["flag"], table=tab)
    if not with_grads:
        return res
    ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64),
                            torch.arange(W, dtype=torch.float64), indexing="ij")
    dC = dimg.permute(1, 2, 0).reshape(-1, 3)
    dtab = render_grads(tab, xs.reshape(-1), ys.reshape(-1), dC, bg)
    res["dtable"] = dtab
    res["dcurves"] = sample_vjp(curves, cfg, dtab)
    return res


def loss_only(curves: dict, cfg: SampleCfg, W: int, H: int, target, bg=(0.0, 0.0, 0.0)):
    with torch.no_grad():
        tab = gaussian_table(curves, cfg)
        img = render_image(tab, W, H, bg)["img"]
        return float(l2_loss(img, target)[0])
