"""Seeded synthetic inputs: curve sets and procedural target images.

This module draws random numbers and scan-converts plain filled shapes; it
holds none of the rasterizer's arithmetic, so both the CUDA path and the CPU
oracle may consume what it makes.  RNG: numpy PCG64 (default_rng), one
stream per purpose split off with SeedSequence.spawn.

Curve recipes (pixel coordinates, activated attributes):
  "uniform"  every control point uniform over the canvas (the tiny workload)
  "local"    open curves as a random walk from a uniform start point, each
             step uniform in +-5% of the canvas per axis (random stroke
             initialisation); closed curves as jittered circles with the
             centre uniform and the radius log-uniform in 1%..8% of the
             shorter side (the circular initialisation of new curves)
  widths U[1,4] px, colours U[0,1]^3, opacities U[0.3,1] (three per open
  curve, one per closed curve).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CurveArrays:
    open_ctrl: np.ndarray     # [No,10,2] float32
    open_width: np.ndarray    # [No]
    open_color: np.ndarray    # [No,3]
    open_opac: np.ndarray     # [No,3]
    closed_ctrl: np.ndarray   # [Nc,12,2]
    closed_color: np.ndarray  # [Nc,3]
    closed_opac: np.ndarray   # [Nc]

    @property
    def n_open(self) -> int:
        return int(self.open_ctrl.shape[0])

    @property
    def n_closed(self) -> int:
        return int(self.closed_ctrl.shape[0])

    def as_dict(self):
        return dict(open_ctrl=self.open_ctrl, open_width=self.open_width,
                    open_color=self.open_color, open_opac=self.open_opac,
                    closed_ctrl=self.closed_ctrl, closed_color=self.closed_color,
                    closed_opac=self.closed_opac)


def _rngs(seed: int, n: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(n)]


def make_curves(seed: int, W: int, H: int, n_open: int, n_closed: int,
                style: str = "local", width_range=(1.0, 4.0),
                opac_range=(0.3, 1.0)) -> CurveArrays:
    r_geo_o, r_geo_c, r_att = _rngs(seed, 3)
    f = np.float32
    size = np.array([W, H], dtype=np.float64)
    if style == "uniform":
        oc = r_geo_o.uniform(0.0, 1.0, (n_open, 10, 2)) * size
        cc = r_geo_c.uniform(0.0, 1.0, (n_closed, 12, 2)) * size
    elif style == "local":
        start = r_geo_o.uniform(0.0, 1.0, (n_open, 1, 2)) * size
        steps = r_geo_o.uniform(-0.05, 0.05, (n_open, 9, 2)) * size
        oc = np.concatenate([start, start + np.cumsum(steps, axis=1)], axis=1)
        centre = r_geo_c.uniform(0.0, 1.0, (n_closed, 1, 2)) * size
        lo, hi = np.log(0.01 * min(W, H)), np.log(0.08 * min(W, H))
        radius = np.exp(r_geo_c.uniform(lo, hi, (n_closed, 1)))
        phase = r_geo_c.uniform(0.0, 2 * np.pi, (n_closed, 1))
        ang = phase + 2 * np.pi * np.arange(12)[None, :] / 12
        rad = radius * r_geo_c.uniform(0.85, 1.15, (n_closed, 12))
        cc = centre + np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=-1)
    else:
        raise ValueError(style)
    return CurveArrays(
        open_ctrl=oc.astype(f),
        open_width=r_att.uniform(*width_range, n_open).astype(f),
        open_color=r_att.uniform(0.0, 1.0, (n_open, 3)).astype(f),
        open_opac=r_att.uniform(*opac_range, (n_open, 3)).astype(f),
        closed_ctrl=cc.astype(f),
        closed_color=r_att.uniform(0.0, 1.0, (n_closed, 3)).astype(f),
        closed_opac=r_att.uniform(*opac_range, n_closed).astype(f),
    )


def _inside_polygon(xs, ys, vx, vy):
    """Even-odd crossing test of pixel centres against a polygon."""
    inside = np.zeros(xs.shape, dtype=bool)
    n = vx.shape[0]
    for i in range(n):
        j = (i + 1) % n
        crosses = (vy[i] > ys) != (vy[j] > ys)
        with np.errstate(divide="ignore", invalid="ignore"):
            xint = vx[i] + (ys - vy[i]) * (vx[j] - vx[i]) / (vy[j] - vy[i])
        inside ^= crosses & (xs < xint)
    return inside


def procedural_target(seed: int, W: int, H: int, n_shapes: int, noise_std: float = 0.01):
    """Layered filled ellipses and polygons with linear colour gradients,
    quantised to 8 bits, plus N(0, noise_std) noise.  Planar float32 [3,H,W]."""
    r_shape, r_noise = _rngs(seed, 2)
    img = np.empty((H, W, 3), dtype=np.float64)
    img[:] = r_shape.uniform(0.0, 1.0, 3)
    side = min(W, H)
    for _ in range(n_shapes):
        cx, cy = r_shape.uniform(0, W), r_shape.uniform(0, H)
        rad = np.exp(r_shape.uniform(np.log(0.03 * side), np.log(0.3 * side)))
        kind = r_shape.integers(0, 2)
        c0, c1 = r_shape.uniform(0, 1, 3), r_shape.uniform(0, 1, 3)
        gang = r_shape.uniform(0, 2 * np.pi)
        if kind == 0:
            ax, ay = rad, rad * r_shape.uniform(0.3, 1.0)
            rot = r_shape.uniform(0, np.pi)
            ext = max(ax, ay)
        else:
            nv = int(r_shape.integers(3, 9))
            ang = np.sort(r_shape.uniform(0, 2 * np.pi, nv))
            rr = rad * r_shape.uniform(0.4, 1.0, nv)
            vx, vy = cx + rr * np.cos(ang), cy + rr * np.sin(ang)
            ext = rad
        x0, x1 = int(max(0, np.floor(cx - ext))), int(min(W, np.ceil(cx + ext) + 1))
        y0, y1 = int(max(0, np.floor(cy - ext))), int(min(H, np.ceil(cy + ext) + 1))
        if x0 >= x1 or y0 >= y1:
            continue
        ys, xs = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        xs += 0.5
        ys += 0.5
        if kind == 0:
            u = (xs - cx) * np.cos(rot) + (ys - cy) * np.sin(rot)
            v = -(xs - cx) * np.sin(rot) + (ys - cy) * np.cos(rot)
            m = (u / ax) ** 2 + (v / ay) ** 2 <= 1.0
        else:
            m = _inside_polygon(xs, ys, vx, vy)
        proj = ((xs - cx) * np.cos(gang) + (ys - cy) * np.sin(gang)) / (2 * rad) + 0.5
        proj = np.clip(proj, 0.0, 1.0)[..., None]
        col = c0 * (1 - proj) + c1 * proj
        sub = img[y0:y1, x0:x1]
        sub[m] = col[m]
    img = np.round(img * 255.0) / 255.0
    img = img + r_noise.normal(0.0, noise_std, img.shape)
    return np.ascontiguousarray(img.transpose(2, 0, 1)).astype(np.float32)


def lowfreq_noise(seed: int, W: int, H: int, amp: float = 0.1, grid: int = 8):
    """Smooth colour noise: an grid x grid x 3 U[-amp, amp] lattice upsampled
    bilinearly to [3,H,W] float32."""
    (rng,) = _rngs(seed, 1)
    lat = rng.uniform(-amp, amp, (3, grid, grid))
    gy = (np.arange(H) + 0.5) / H * (grid - 1)
    gx = (np.arange(W) + 0.5) / W * (grid - 1)
    y0 = np.clip(np.floor(gy).astype(int), 0, grid - 2)
    x0 = np.clip(np.floor(gx).astype(int), 0, grid - 2)
    fy = (gy - y0)[:, None]
    fx = (gx - x0)[None, :]
    a = lat[:, y0][:, :, x0]
    b = lat[:, y0][:, :, x0 + 1]
    c = lat[:, y0 + 1][:, :, x0]
    d = lat[:, y0 + 1][:, :, x0 + 1]
    out = a * (1 - fy) * (1 - fx) + b * (1 - fy) * fx + c * fy * (1 - fx) + d * fy * fx
    return out.astype(np.float32)


def prune_inputs(seed: int, W: int, H: int, n_open: int, n_closed: int, n_blobs: int = 40,
                 frac: float = 0.06, n_shapes: int = 40):
    """Inputs of a pruning/densification pass: a "local" curve set in which
    about `frac` of the curves each get low opacities, a shrunken outline
    (closed curves), a near-copy of another curve (geometry jittered by
    N(0, 0.2) px, colour by N(0, 0.004)), or a faint middle segment (open
    curves); a procedural target; and an image equal to the target plus
    U[-0.02, 0.02] noise and `n_blobs` filled ellipses offset by U[0.3, 0.6]
    per channel (the error regions).  Returns (curve dict, img, target)."""
    c = make_curves(seed, W, H, n_open, n_closed, style="local").as_dict()
    c = {k: v.copy() for k, v in c.items()}
    r_pick, r_val, r_img = _rngs(seed + 7919, 3)
    oo, co = c["open_opac"], c["closed_opac"]
    low_o = r_pick.random(n_open) < frac
    oo[low_o] = r_val.uniform(0.0, 0.15, (int(low_o.sum()), 3))
    low_c = r_pick.random(n_closed) < frac
    co[low_c] = r_val.uniform(0.0, 0.18, int(low_c.sum()))
    small = r_pick.random(n_closed) < frac
    cc = c["closed_ctrl"]
    ctr = cc[small].mean(1, keepdims=True)
    cc[small] = ctr + (cc[small] - ctr) * np.float32(0.02)
    dip = r_pick.random(n_open) < frac
    k = int(dip.sum())
    oo[dip] = np.stack([r_val.uniform(0.8, 1.0, k), r_val.uniform(0.0, 0.25, k), r_val.uniform(0.8, 1.0, k)], 1)
    for kind, ctrl_key, extra in (("open", "open_ctrl", ("open_width", "open_opac")),
                                  ("closed", "closed_ctrl", ("closed_opac",))):
        n = n_open if kind == "open" else n_closed
        col_key = kind + "_color"
        if n < 2:
            continue
        dst = np.nonzero(r_pick.random(n) < frac)[0]
        src = r_pick.integers(0, n, dst.shape[0])
        keep = src != dst
        dst, src = dst[keep], src[keep]
        c[ctrl_key][dst] = c[ctrl_key][src] + r_val.normal(0, 0.2, c[ctrl_key][src].shape).astype(np.float32)
        c[col_key][dst] = c[col_key][src] + r_val.normal(0, 0.004, (dst.shape[0], 3)).astype(np.float32)
        for e in extra:
            c[e][dst] = c[e][src]
    target = procedural_target(seed, W, H, n_shapes)
    img = target + r_img.uniform(-0.02, 0.02, target.shape).astype(np.float32)
    side = min(W, H)
    for _ in range(n_blobs):
        cx, cy = r_img.uniform(0, W), r_img.uniform(0, H)
        ax, ay = np.exp(r_img.uniform(np.log(0.005 * side + 0.5), np.log(0.06 * side + 1), 2))
        x0, x1 = int(max(0, np.floor(cx - ax))), int(min(W, np.ceil(cx + ax) + 1))
        y0, y1 = int(max(0, np.floor(cy - ay))), int(min(H, np.ceil(cy + ay) + 1))
        off = r_img.uniform(0.3, 0.6, 3) * r_img.choice([-1.0, 1.0], 3)
        if x0 >= x1 or y0 >= y1:
            continue
        ys, xs = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        m = ((xs + 0.5 - cx) / ax) ** 2 + ((ys + 0.5 - cy) / ay) ** 2 <= 1.0
        for ch in range(3):
            img[ch, y0:y1, x0:x1][m] += np.float32(off[ch])
    return c, np.ascontiguousarray(img, dtype=np.float32), target


# The workloads, by what they are.
def batch_layout(seed: int, n_images: int = 64, side=(256, 2048), aspect=(0.5, 2.0), curves=(128, 4096)):
    """A ragged batch: per image W, H, n_open, n_closed and a seed.  The
    side s is log-uniform in `side`, the aspect a = W / H uniform in `aspect`
    (W = s sqrt(a), H = s / sqrt(a), at least 16 px), the curve count
    log-uniform in `curves`, half open (rounded down) and half closed."""
    (rng,) = _rngs(seed, 1)
    out = []
    for i in range(n_images):
        s = float(np.exp(rng.uniform(np.log(side[0]), np.log(side[1]))))
        a = float(rng.uniform(aspect[0], aspect[1]))
        W = max(16, int(round(s * np.sqrt(a))))
        H = max(16, int(round(s / np.sqrt(a))))
        n = int(round(np.exp(rng.uniform(np.log(curves[0]), np.log(curves[1])))))
        out.append(dict(W=W, H=H, n_open=n // 2, n_closed=n - n // 2, seed=seed * 1000 + i))
    return out


def batch_inputs(layout, n_shapes: int = 16, style: str = "local"):
    """Curves (concatenated image after image, the batch layout) and the
    targets (flattened planar images, concatenated) of a batch_layout."""
    arrs = [make_curves(e["seed"], e["W"], e["H"], e["n_open"], e["n_closed"], style=style).as_dict()
            for e in layout]
    cat = {k: np.concatenate([a[k] for a in arrs], 0) for k in arrs[0]} if arrs else {}
    targets = [procedural_target(e["seed"] + 1, e["W"], e["H"], n_shapes) for e in layout]
    return arrs, cat, targets


WORKLOADS = {
    # 256x256, 64 open curves, 16 Gaussians per curve, 16x16 tiles
    "tiny_256_64open": dict(W=256, H=256, n_open=64, n_closed=0, style="uniform",
                            g_open=16, rows_closed=4, k_closed=8, tile=16, seed=1),
    # 1024x1024, 512 open + 256 closed, 32 Gaussians per curve
    "mid_1024_768": dict(W=1024, H=1024, n_open=512, n_closed=256, style="local",
                         g_open=32, rows_closed=4, k_closed=8, tile=16, seed=10,
                         n_shapes=40),
    # 2048x2048, 2048 open + 2048 closed, 64 Gaussians per curve (262,144)
    "hires_2048_4096": dict(W=2048, H=2048, n_open=2048, n_closed=2048, style="local",
                            g_open=64, rows_closed=8, k_closed=8, tile=16, seed=20,
                            n_shapes=200),
    # a quarter of it (1024x1024, 512 + 512 curves, the same sampling): the
    # small case of the kernels' profiler captures
    "hires_1024_1024": dict(W=1024, H=1024, n_open=512, n_closed=512, style="local",
                            g_open=64, rows_closed=8, k_closed=8, tile=16, seed=20,
                            n_shapes=50),
}

# 64 ragged images (sides log-uniform in [256, 2048], aspect in [0.5, 2],
# 128..4096 curves each, half open and half closed), optimised together
BATCH_WORKLOAD = dict(name="batch64_ragged", n_images=64, seed=30, side=(256, 2048), aspect=(0.5, 2.0),
                      curves=(128, 4096), n_shapes=16)
