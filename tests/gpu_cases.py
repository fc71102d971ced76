"""Seeded cases shared by the GPU parity tests: the same synthetic inputs go
to the CUDA library (through the C ABI binding) and to the CPU oracle."""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

import oracle
from oracle.curves import SampleCfg as OCfg, table_to_f32, table_from_f32
from oracle.pipeline import as_curves
from paper_2503_16424_gb300 import synth


@dataclass
class Case:
    name: str
    W: int
    H: int
    n_open: int
    n_closed: int
    style: str
    g_open: int
    rows: int
    kc: int
    seed: int
    bg: tuple = (0.0, 0.0, 0.0)
    dup: int = 0            # duplicate this many curves (equal draw keys)


CASES = {
    # the 256x256, 64-open-curve workload, full size
    "tiny256": Case("tiny256", 256, 256, 64, 0, "uniform", 16, 4, 8, 1),
    # ragged canvas (not a multiple of the tile), open + closed, background
    "ragged": Case("ragged", 100, 73, 12, 6, "local", 12, 5, 7, 2, bg=(0.2, 0.5, 0.1), dup=2),
    # several sort partitions, both curve kinds
    "mixed": Case("mixed", 192, 160, 40, 24, "local", 16, 4, 8, 3, bg=(0.0, 0.3, 0.6), dup=3),
    # curves of 512 samples or more (sampled by the wide CTAs): open curves
    # of 600 samples, closed curves of R = 80 interior rows (82 x 8), whose
    # rows near the boundaries are thin
    "dense": Case("dense", 120, 90, 2, 2, "local", 600, 82, 8, 4, bg=(0.1, 0.1, 0.1)),
}


def arrays(case: Case):
    a = synth.make_curves(case.seed, case.W, case.H, case.n_open, case.n_closed, style=case.style).as_dict()
    if case.dup:
        for k in ("open_ctrl", "open_width", "open_color", "open_opac"):
            if case.n_open > case.dup:
                a[k][-case.dup:] = a[k][:case.dup]
        for k in ("closed_ctrl", "closed_color", "closed_opac"):
            if case.n_closed > case.dup:
                a[k][-case.dup:] = a[k][:case.dup]
    return a


def ocfg(case: Case, tangent_mode: int = 0):
    return OCfg(g_open=case.g_open, rows_closed=case.rows, k_closed=case.kc, tangent_mode=tangent_mode)


def oracle_table(case: Case, arr=None, tangent_mode: int = 0):
    arr = arr if arr is not None else arrays(case)
    cfg = ocfg(case, tangent_mode)
    rank, first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], cfg)
    tab = oracle.gaussian_table(as_curves(arr), cfg, first)
    return tab, rank, first


def target(case: Case):
    return synth.procedural_target(case.seed + 1000, case.W, case.H, 12)


def grad_rel_err(got, exp, floor_frac=1e-6):
    """max_i |got_i - exp_i| / max(|exp_i|, floor_frac * max|exp|)."""
    got = torch.as_tensor(got, dtype=torch.float64).reshape(-1)
    exp = torch.as_tensor(exp, dtype=torch.float64).reshape(-1)
    if exp.numel() == 0:
        return 0.0
    floor = max(float(exp.abs().max()) * floor_frac, 1e-30)
    return float(((got - exp).abs() / torch.clamp(exp.abs(), min=floor)).max())


# Float32 rounding of a gradient entry (see oracle/bounds.py): a sum over
# pixels of per-pixel terms, bounded by gamma_n * sum |terms| with u = 2^-24.
# n = DEPTH + the tiles the Gaussian is listed in: about 12 roundings to
# recompute alpha and its derivative in a term, 3 + 5 + 1 in the in-tile
# reduction (a lane's four pixels, the warp, the shared-memory rows), 4 in
# the conversion from eigen-frame sums, one per tile atomic, and room for the
# transmittance and colour-behind recursions of the reverse walk.
U32 = 2.0 ** -24
DEPTH = 32


def tiles_per_gaussian(rec, W, H, tile=16):
    """Tiles listing each Gaussian of the float32 table (its atomics)."""
    tx0, tx1, ty0, ty1, ok = oracle.tile_rects_f32(rec, W, H, tile)
    return torch.as_tensor(np.where(ok, (tx1 - tx0 + 1) * (ty1 - ty0 + 1), 0), dtype=torch.float64)


def blend_grad_bound(rec, W, H, dC, bg=(0.0, 0.0, 0.0), tile=16, xs=None, ys=None, tab=None):
    """Per field of the table gradient, the float32 error bound of each entry:
    (DEPTH + its tiles) u A, A = oracle.bounds.blend_abs at the pixels
    (xs, ys) (default: the whole W x H canvas) with dL/dC = dC [n, 3]."""
    from oracle.bounds import blend_abs
    tab = table_from_f32(rec) if tab is None else tab
    if xs is None:
        ys_, xs_ = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64),
                                  indexing="ij")
        xs, ys = xs_.reshape(-1), ys_.reshape(-1)
    A = blend_abs(tab, xs, ys, dC, bg)
    c = (DEPTH + tiles_per_gaussian(rec, W, H, tile)) * U32
    return {k: (c[:, None] * v if v.dim() == 2 else c * v) for k, v in A.items()}


def curve_grad_bound(arr, cfg, first, gbound, dtab):
    """The float32 error bound of the curve gradients: the table-gradient
    bound carried through the sampling's Jacobian in absolute value, plus the
    sampling backward's own rounding (DEPTH u |dL/dtable|)."""
    from oracle.bounds import sample_abs_vjp
    from oracle.raster import GRAD_KEYS
    scale = {}
    for k in GRAD_KEYS:
        d = torch.as_tensor(dtab[k], dtype=torch.float64).abs()
        g = gbound[k] if gbound is not None else torch.zeros_like(d)
        scale[k] = g + DEPTH * U32 * d
    return sample_abs_vjp(as_curves(arr), cfg, scale, first)


def grad_check(got, exp, bound=None, rel=1e-3, floor_frac=1e-6):
    """The gradient bar: |got - exp| <= rel max(|exp|, floor_frac max|exp|)
    + bound, entry by entry.  Returns the largest ratio of |got - exp| to
    its allowance (the bar holds when it is <= 1)."""
    got = torch.as_tensor(got, dtype=torch.float64).reshape(-1)
    exp = torch.as_tensor(exp, dtype=torch.float64).reshape(-1)
    if exp.numel() == 0:
        return 0.0
    floor = max(float(exp.abs().max()) * floor_frac, 1e-300)
    allow = rel * torch.clamp(exp.abs(), min=floor)
    if bound is not None:
        allow = allow + torch.as_tensor(bound, dtype=torch.float64).reshape(-1)
    return float(((got - exp).abs() / allow).max())


__all__ = ["CASES", "Case", "arrays", "ocfg", "oracle_table", "target", "grad_rel_err", "grad_check",
           "blend_grad_bound", "curve_grad_bound", "tiles_per_gaussian", "table_to_f32", "table_from_f32"]
