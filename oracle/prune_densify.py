"""Section 3.5 and Algorithm 1 (Appendix B): adaptive pruning and densification.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper (silent, or two passages disagree):
  * opacity threshold tau_op(t) falls linearly from op_start (0.2, the value
    Section 3.5 gives as an example) to op_end (0.02, Section 4.1) at t_end;
  * opacity(b) is the mean of a curve's opacities (three for an open curve);
    area(b) is the draw-order area key (curves.area_keys_f32);
  * a curve is pruned when opacity < tau_op(t), or area < area_min, or when a
    curve drawn in front of it (lower draw rank) has colour distance < 0.03
    and bounding-box IoU > 0.9 (the pair reading of Algorithm 1's overlap
    rule: the later of a redundant pair goes).  Boxes are the control points'
    box, widened by width/2 for open curves;
  * an open curve that is kept and whose middle opacity is more than 0.5
    below both end opacities is split (Appendix B): it keeps its first
    segment, re-parametrised as three segments, and its last segment goes to
    the first free open slot the same way (if no slot is free, that half is
    dropped);
  * error map e = mean over channels of |img - target|; regions are the
    4-connected components of e > err_thresh, sorted by area (descending;
    equal areas by their first pixel in row-major order);
  * the remaining free slots, in index order (open slots first), receive the
    regions in that order; a new curve follows LIVE's circular initialisation:
    control points on the circle through the region's centroid with radius
    sqrt(area / pi) (closed: 12 points at angles 2 pi j / 12; open: 10 points
    at angles 2 pi j / 11), colour = mean target colour over the region,
    opacity new_opacity, width new_width;
  * a free slot left without a region keeps its geometry with opacity 0.

Decisions that floating point makes (the thresholds) are taken in float32
with a fixed operation order, as in the CUDA kernels; sums are fp64.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .curves import area_keys_f32, draw_order, SampleCfg


@dataclass(frozen=True)
class PDCfg:
    op_start: float = 0.2
    op_end: float = 0.02
    step: int = 0
    t_end: int = 1
    area_min: float = 4.0
    color_eps: float = 0.03
    iou_min: float = 0.9
    err_thresh: float = 0.1
    split_drop: float = 0.5
    new_opacity: float = 0.5
    new_width: float = 2.0


F = np.float32


def tau_op(cfg: PDCfg) -> np.float32:
    """op_start (1 - f) + op_end f with f = min(1, step / t_end), in float32
    (the two end points are met exactly)."""
    frac = F(min(1.0, cfg.step / max(1, cfg.t_end)))
    return F(F(F(cfg.op_start) * F(F(1) - frac)) + F(F(cfg.op_end) * frac))


def curve_boxes_f32(open_ctrl, open_width, closed_ctrl):
    """[N, 4] float32 boxes (x0, y0, x1, y1) of the control points; open
    curves widened by width / 2."""
    oc = np.asarray(open_ctrl, F).reshape(-1, 10, 2)
    cc = np.asarray(closed_ctrl, F).reshape(-1, 12, 2)
    hw = np.asarray(open_width, F).reshape(-1) * F(0.5)
    bo = np.stack([oc[..., 0].min(1) - hw, oc[..., 1].min(1) - hw, oc[..., 0].max(1) + hw, oc[..., 1].max(1) + hw], 1)
    bc = np.stack([cc[..., 0].min(1), cc[..., 1].min(1), cc[..., 0].max(1), cc[..., 1].max(1)], 1)
    return np.concatenate([bo, bc]).astype(F)


def iou_f32(a, b):
    """Elementwise IoU of float32 boxes a [..., 4], b [..., 4]: intersection
    over union of the two axis-aligned boxes, each step rounded to float32;
    0 where the union is empty."""
    a = np.asarray(a, F)
    b = np.asarray(b, F)
    iw = np.maximum(F(0), np.minimum(a[..., 2], b[..., 2]) - np.maximum(a[..., 0], b[..., 0]))
    ih = np.maximum(F(0), np.minimum(a[..., 3], b[..., 3]) - np.maximum(a[..., 1], b[..., 1]))
    inter = iw * ih
    area_a = (a[..., 2] - a[..., 0]) * (a[..., 3] - a[..., 1])
    area_b = (b[..., 2] - b[..., 0]) * (b[..., 3] - b[..., 1])
    union = (area_a + area_b) - inter
    with np.errstate(divide="ignore", invalid="ignore"):
        q = inter / union
    return np.where(union > 0, q, F(0)).astype(F)


def color_dist_f32(a, b):
    """Elementwise Euclidean RGB distance of a [..., 3] and b [..., 3] in float32."""
    d = np.asarray(a, F) - np.asarray(b, F)
    return np.sqrt((d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]).astype(F)


def mean_opacity_f32(arr):
    """opacity(b) of Algorithm 1: the mean of an open curve's three segment
    opacities ((o0 + o1) + o2) / 3, a closed curve's single opacity."""
    oo = np.asarray(arr["open_opac"], F).reshape(-1, 3)
    mo = ((oo[:, 0] + oo[:, 1]) + oo[:, 2]) / F(3.0)
    return np.concatenate([mo.astype(F), np.asarray(arr["closed_opac"], F).reshape(-1)])


def prune_flags(arr: dict, cfg: PDCfg, scfg: SampleCfg, rows_per_chunk: int = 512):
    """Pruning phase of Algorithm 1: boolean [N] decision and the masks of
    the three criteria (low opacity, small area, redundant overlap)."""
    oc, ow, cc = arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"]
    keys = area_keys_f32(oc, ow, cc)
    rank, _ = draw_order(oc, ow, cc, scfg)
    low_op = mean_opacity_f32(arr) < tau_op(cfg)
    small = keys < F(cfg.area_min)
    boxes = curve_boxes_f32(oc, ow, cc)
    cols = np.concatenate([np.asarray(arr["open_color"], F).reshape(-1, 3),
                           np.asarray(arr["closed_color"], F).reshape(-1, 3)])
    n = keys.shape[0]
    overlap = np.zeros(n, bool)
    rank = np.asarray(rank)
    for i0 in range(0, n, rows_per_chunk):
        i1 = min(n, i0 + rows_per_chunk)
        # pair (i, j): j is drawn in front of i, similar colour, boxes overlap
        front = rank[None, :] < rank[i0:i1, None]
        similar = color_dist_f32(cols[i0:i1, None, :], cols[None, :, :]) < F(cfg.color_eps)
        iou = iou_f32(boxes[i0:i1, None, :], boxes[None, :, :])
        overlap[i0:i1] = (front & similar & (iou > F(cfg.iou_min))).any(1)
    return low_op | small | overlap, dict(low_op=low_op, small=small, overlap=overlap)


def split_flags(arr: dict, pruned, cfg: PDCfg):
    """Open curves kept whose middle opacity is split_drop below both ends."""
    oo = np.asarray(arr["open_opac"], F).reshape(-1, 3)
    drop = F(cfg.split_drop)
    s = (oo[:, 1] < oo[:, 0] - drop) & (oo[:, 1] < oo[:, 2] - drop)
    return s & ~np.asarray(pruned)[: oo.shape[0]]


def subdivide_thirds(seg):
    """A cubic segment [4, 2] as three chained cubic segments [10, 2]
    covering t in [0, 1/3], [1/3, 2/3], [2/3, 1] (de Casteljau splits)."""
    def split(p, t):
        a = [p[j] * (1 - t) + p[j + 1] * t for j in range(3)]
        b = [a[j] * (1 - t) + a[j + 1] * t for j in range(2)]
        c = b[0] * (1 - t) + b[1] * t
        return np.array([p[0], a[0], b[0], c]), np.array([c, b[1], a[2], p[3]])
    seg = np.asarray(seg, np.float64)
    s0, rest = split(seg, 1.0 / 3.0)
    s1, s2 = split(rest, 0.5)
    return np.concatenate([s0, s1[1:], s2[1:]])


def error_regions(img, target, thresh):
    """4-connected components of mean_c |img - target| > thresh.  Returns the
    per-pixel component root (first pixel of the component in row-major
    order, -1 outside) computed by scipy.ndimage.label."""
    from scipy import ndimage
    img = np.asarray(img, F)
    target = np.asarray(target, F)
    d = np.abs(img - target)
    e = F(F(d[0] + d[1]) + d[2]) / F(3.0)
    mask = e > F(thresh)
    lab, n = ndimage.label(mask, structure=[[0, 1, 0], [1, 1, 1], [0, 1, 0]])
    H, W = mask.shape
    flat = lab.reshape(-1)
    root = np.full(flat.shape, -1, np.int64)
    if n:
        first = np.full(n + 1, np.iinfo(np.int64).max)
        idx = np.nonzero(flat)[0]
        np.minimum.at(first, flat[idx], idx)
        root[idx] = first[flat[idx]]
    return root.reshape(H, W), mask


def region_stats(root, target):
    """Regions sorted by (area descending, root ascending): arrays of root,
    area, centroid (px, pixel centres), mean target colour (fp64)."""
    H, W = root.shape
    flat = root.reshape(-1)
    idx = np.nonzero(flat >= 0)[0]
    roots, inv, area = np.unique(flat[idx], return_inverse=True, return_counts=True)
    xs = (idx % W).astype(np.float64) + 0.5
    ys = (idx // W).astype(np.float64) + 0.5
    tgt = np.asarray(target, np.float64).reshape(3, -1)
    sx = np.bincount(inv, xs, len(roots))
    sy = np.bincount(inv, ys, len(roots))
    col = np.stack([np.bincount(inv, tgt[c, idx], len(roots)) for c in range(3)], 1)
    order = np.lexsort((roots, -area))
    area = area[order]
    return dict(root=roots[order], area=area, cx=sx[order] / area, cy=sy[order] / area,
                color=col[order] / area[:, None])


def circle_points(cx, cy, r, n, span):
    ang = 2.0 * np.pi * np.arange(n) / span
    return np.stack([cx + r * np.cos(ang), cy + r * np.sin(ang)], -1)


def prune_densify(arr: dict, img, target, cfg: PDCfg, scfg: SampleCfg):
    """Apply one prune/densify pass to copies of the curve arrays.  Returns
    (new arrays, changed mask [N], details)."""
    out = {k: np.array(v, dtype=np.float64, copy=True) for k, v in arr.items()}
    n_open = out["open_width"].shape[0]
    n_closed = out["closed_opac"].shape[0]
    n = n_open + n_closed
    pruned, crit = prune_flags(arr, cfg, scfg)
    split = split_flags(arr, pruned, cfg)
    changed = pruned.copy()
    free_open = [i for i in range(n_open) if pruned[i]]
    # splits: keep the first segment; the last segment goes to a free open slot
    for i in np.nonzero(split)[0]:
        ctrl = out["open_ctrl"][i].copy()
        op = out["open_opac"][i].copy()
        out["open_ctrl"][i] = subdivide_thirds(ctrl[0:4])
        out["open_opac"][i] = op[0]
        changed[i] = True
        if free_open:
            j = free_open.pop(0)
            out["open_ctrl"][j] = subdivide_thirds(ctrl[6:10])
            out["open_opac"][j] = op[2]
            out["open_width"][j] = out["open_width"][i]
            out["open_color"][j] = out["open_color"][i]
    free = free_open + [n_open + i for i in range(n_closed) if pruned[n_open + i]]
    root, mask = error_regions(img, target, cfg.err_thresh)
    reg = region_stats(root, target)
    for k, slot in enumerate(free):
        if k < reg["area"].shape[0]:
            cx, cy, a = reg["cx"][k], reg["cy"][k], float(reg["area"][k])
            r = np.sqrt(a / np.pi)
            col = reg["color"][k]
            if slot < n_open:
                out["open_ctrl"][slot] = circle_points(cx, cy, r, 10, 11)
                out["open_color"][slot] = col
                out["open_opac"][slot] = cfg.new_opacity
                out["open_width"][slot] = cfg.new_width
            else:
                j = slot - n_open
                out["closed_ctrl"][j] = circle_points(cx, cy, r, 12, 12)
                out["closed_color"][j] = col
                out["closed_opac"][j] = cfg.new_opacity
        else:
            if slot < n_open:
                out["open_opac"][slot] = 0.0
            else:
                out["closed_opac"][slot - n_open] = 0.0
    return out, changed, dict(pruned=pruned, split=split, regions=reg, root=root, mask=mask, free=free, **crit)
