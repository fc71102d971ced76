"""Autotuning of a batch: the Gaussians-per-curve sampling of each image and
the tile side of the batch.

Sampling.  The paper fixes the number of Gaussians per curve per experiment
(Section 3.3; Table 4 varies the rows of closed curves).  With rho = 1 a
Gaussian's scale along the curve is the sample spacing (Eq. 7), so a shape
rendered from K samples overhangs its outline by about one spacing: the
render converges only linearly in K, and a fixed K under-samples the long
curves of a large image while over-sampling the short curves of a small
one.  The default rule here ("spacing") gives each image the sparsest
sampling of a schedule whose spacing is at most `max_spacing` pixels along
its median open curve (control-polygon length / (K - 1)), across its median
closed curve (the distance between the middles of its two boundaries /
(rows - 1)) and along it (boundary polygon length / (K - 1)).  The
"fidelity" rule instead renders every image at each sampling and at a dense
reference through the library's batched forward and keeps the sparsest
whose PSNR against the reference reaches `psnr_min`.

Tile side.  8, 16 and 32 give the same images (culling is exact); they
trade binning work (pairs grow as the tiles shrink) against blend work
(larger tiles stage more Gaussians that miss most blocks).  Each side is
timed on a few eager steps with CUDA events and the fastest is kept.
"""

from __future__ import annotations

import math

import torch

from . import bs
from .batch import BatchRasterizer

import numpy as np

# (g_open, rows_closed, k_closed): Gaussians per open / closed curve
SCHEDULE = ((16, 4, 4), (32, 4, 8), (64, 8, 8))
REFERENCE = (128, 16, 8)
TILES = (8, 16, 32)
OPEN_CHOICES = (16, 32, 64, 128)
ROW_CHOICES = (4, 8, 16)
K_CHOICES = (4, 8, 16, 32)


def _smallest(choices, length, max_spacing):
    for c in choices:
        if length / (c - 1) <= max_spacing:
            return c
    return choices[-1]


def spacing_sampling(images, arrs, max_spacing: float = 8.0):
    """Per image (host curve arrays `arrs`, one dict per image): g_open,
    rows_closed, k_closed, the sparsest choices whose spacing along the
    image's median open curve, across and along its median closed curve, is
    at most max_spacing px."""
    out = []
    for im, a in zip(images, arrs):
        g, rows, k = OPEN_CHOICES[0], ROW_CHOICES[0], K_CHOICES[0]
        if im.n_open:
            P = np.asarray(a["open_ctrl"], dtype=np.float64)
            L = np.linalg.norm(np.diff(P, axis=1), axis=2).sum(1)
            g = _smallest(OPEN_CHOICES, float(np.median(L)), max_spacing)
        if im.n_closed:
            P = np.asarray(a["closed_ctrl"], dtype=np.float64)
            A = P[:, 0:7]                                   # boundary P0..P6
            B = P[:, [0, 11, 10, 9, 8, 7, 6]]               # boundary P0, P11..P7, P6
            across = np.linalg.norm(A[:, 3] - B[:, 3], axis=1)
            along = np.maximum(np.linalg.norm(np.diff(A, axis=1), axis=2).sum(1),
                               np.linalg.norm(np.diff(B, axis=1), axis=2).sum(1))
            rows = _smallest(ROW_CHOICES, float(np.median(across)), max_spacing)
            k = _smallest(K_CHOICES, float(np.median(along)), max_spacing)
        out.append((g, rows, k))
    return out


def with_sampling(images, picks):
    """The images with their sampling replaced: picks[b] = (g_open,
    rows_closed, k_closed) for image b."""
    return [bs.BatchImage(im.width, im.height, im.n_open, im.n_closed,
                          bs.SampleCfg(g_open=g, rows_closed=r, k_closed=k, rho=im.sample.rho,
                                       cov_eps=im.sample.cov_eps), im.bg)
            for im, (g, r, k) in zip(images, picks)]


def _render(images, curves, tile, device):
    r = BatchRasterizer(images, tile=tile, pair_capacity=1 << 22, device=device)
    r.fit_capacity(curves)
    r.forward(curves)
    return r


def pick_sampling(images, curves: bs.CurveSet, psnr_min: float = 35.0, schedule=SCHEDULE, reference=REFERENCE,
                  tile: int = 16, device="cuda"):
    """Per image, the first entry of `schedule` whose render is within
    psnr_min dB (PSNR, peak 1) of the `reference` sampling's render, else
    the last entry.  Returns (images with those samplings, per-image PSNR
    table {entry: [dB per image]})."""
    ref = _render(with_sampling(images, [reference] * len(images)), curves, tile, device)
    table = {}
    picks = [None] * len(images)
    for entry in schedule:
        r = _render(with_sampling(images, [entry] * len(images)), curves, tile, device)
        dbs = []
        for b in range(len(images)):
            d = (r.batch.image(r.img, b) - ref.batch.image(ref.img, b)).double()
            mse = float((d * d).mean())
            db = float("inf") if mse == 0.0 else -10.0 * math.log10(mse)
            dbs.append(db)
            if picks[b] is None and db >= psnr_min:
                picks[b] = entry
        table[entry] = dbs
        del r
    picks = [p if p is not None else schedule[-1] for p in picks]
    return with_sampling(images, picks), table


def pick_tile(images, curves: bs.CurveSet, target: torch.Tensor, tiles=TILES, steps: int = 4, device="cuda"):
    """The tile side whose step (forward with the L2 loss, backward) is
    fastest, and the measured ms per step of each side."""
    ms = {}
    for t in tiles:
        r = BatchRasterizer(images, tile=t, pair_capacity=1 << 22, device=device)
        r.fit_capacity(curves)
        grad = curves.zeros_like()
        r.step(curves, target, grad)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            r.step(curves, target, grad)
        b.record()
        torch.cuda.synchronize()
        ms[t] = a.elapsed_time(b) / steps
        del r
    best = min(ms, key=ms.get)
    return best, ms


def autotune(images, curves: bs.CurveSet, target: torch.Tensor, arrs=None, rule: str = "spacing",
             max_spacing: float = 8.0, psnr_min: float = 35.0, device="cuda"):
    """Sampling per image (rule "spacing" from the host curve arrays `arrs`,
    or "fidelity"), then the tile side for that sampling.  Returns
    (images, tile, report)."""
    if rule == "spacing":
        tuned = with_sampling(images, spacing_sampling(images, arrs, max_spacing))
        table = {}
    else:
        tuned, table = pick_sampling(images, curves, psnr_min, device=device)
    tile, ms = pick_tile(tuned, curves, target, device=device)
    counts = {}
    for im in tuned:
        key = (im.sample.g_open, im.sample.rows_closed, im.sample.k_closed)
        counts[key] = counts.get(key, 0) + 1
    def q(v, f):
        v = sorted(x for x in v if x != float("inf"))
        return round(v[min(len(v) - 1, int(f * len(v)))], 2) if v else None
    report = {"rule": rule, "max_spacing_px": max_spacing if rule == "spacing" else None,
              "psnr_min_db": psnr_min if rule != "spacing" else None,
              "sampling_counts": {f"{g}/{r}x{k}": n for (g, r, k), n in sorted(counts.items())},
              "psnr_vs_reference_db": {f"{g}/{r}x{k}": {"min": q(v, 0.0), "median": q(v, 0.5), "max": q(v, 1.0)}
                                      for (g, r, k), v in table.items()},
              "tile_ms": {str(k): round(v, 4) for k, v in ms.items()}, "tile": tile}
    return tuned, tile, report
