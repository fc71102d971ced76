"""Section 3.4: tile binning with (tile, depth) keys.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper follows the tile pipeline of 3D Gaussian splatting: each Gaussian is
listed in every screen tile its support touches, the (tile, depth) pairs are
sorted, and each tile blends its list in depth order.  Here the depth of a
Gaussian is its index in the draw-ordered table, so a key is

    key = tile_id << gbits | g,   tile_id = ty * tiles_x + tx,

and sorting the keys orders every tile's list front to back.

The tile rectangle of a Gaussian is decided in float32 (the precision the
CUDA kernel decides it in), from the table's own fields, with this fixed
sequence of correctly rounded operations:

    xlo = (mx - ext_x) - 0.5        xhi = (mx + ext_x) - 0.5
    i0  = max(ceil(xlo), 0)         i1  = min(floor(xhi), W - 1)

(same for y); the pixels whose centres x + 0.5 lie in [mx - ext_x, mx + ext_x]
are x = i0..i1, the tiles tx = i0 // T .. i1 // T.  A Gaussian is listed
nowhere if ext_x or ext_y is negative or any bound is not finite, or if the
range is empty.
"""

from __future__ import annotations

import numpy as np


def key_bits(n_gauss: int, n_tiles: int):
    gbits = max(1, int(n_gauss - 1).bit_length())
    tbits = max(1, int(n_tiles - 1).bit_length())
    return gbits, tbits


def tile_rects_f32(rec: np.ndarray, W: int, H: int, tile: int):
    """Per-Gaussian inclusive tile rectangle (tx0, tx1, ty0, ty1) and a
    validity mask, from the float32 table rec [Ng, 12]."""
    f = np.float32
    rec = np.asarray(rec, dtype=f)
    mx, my = rec[:, 0], rec[:, 1]
    ex, ey = rec[:, 10], rec[:, 11]
    half = f(0.5)
    with np.errstate(invalid="ignore", over="ignore"):
        xlo = (mx - ex) - half
        xhi = (mx + ex) - half
        ylo = (my - ey) - half
        yhi = (my + ey) - half
        ok = (ex >= 0) & (ey >= 0)
        ok &= np.isfinite(xlo) & np.isfinite(xhi) & np.isfinite(ylo) & np.isfinite(yhi)
        xlo = np.where(ok, xlo, f(0)); xhi = np.where(ok, xhi, f(0))
        ylo = np.where(ok, ylo, f(0)); yhi = np.where(ok, yhi, f(0))
        i0 = np.maximum(np.ceil(xlo), f(0)); i1 = np.minimum(np.floor(xhi), f(W - 1))
        j0 = np.maximum(np.ceil(ylo), f(0)); j1 = np.minimum(np.floor(yhi), f(H - 1))
        ok &= (i0 <= i1) & (j0 <= j1)
    i0 = np.where(ok, i0, 0).astype(np.int64); i1 = np.where(ok, i1, -1).astype(np.int64)
    j0 = np.where(ok, j0, 0).astype(np.int64); j1 = np.where(ok, j1, -1).astype(np.int64)
    return i0 // tile, i1 // tile, j0 // tile, j1 // tile, ok


def tile_keys(rec: np.ndarray, W: int, H: int, tile: int):
    """All (tile, Gaussian) keys sorted ascending, the tile ranges [n_tiles, 2]
    (start, end) into them (an empty tile has (0, 0)), and the per-Gaussian
    pair counts.  Keys are uint32, or uint64 when tile bits + Gaussian bits
    exceed 32."""
    ng = rec.shape[0]
    tiles_x = -(-W // tile)
    tiles_y = -(-H // tile)
    n_tiles = tiles_x * tiles_y
    gbits, tbits = key_bits(ng, n_tiles)
    wide = gbits + tbits > 32          # then the keys are uint64
    tx0, tx1, ty0, ty1, ok = tile_rects_f32(rec, W, H, tile)
    counts = np.where(ok, (tx1 - tx0 + 1) * (ty1 - ty0 + 1), 0).astype(np.int64)
    # every tile of every rectangle, row by row
    g = np.repeat(np.arange(ng, dtype=np.int64), counts)
    start = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    local = np.arange(g.shape[0], dtype=np.int64) - start[g]
    width = (tx1 - tx0 + 1)[g]
    tx = tx0[g] + local % width
    ty = ty0[g] + local // width
    tid = (ty * tiles_x + tx).astype(np.uint64)
    keys = np.sort((tid << np.uint64(gbits)) | g.astype(np.uint64))
    if not wide:
        keys = keys.astype(np.uint32)
    tile_of = keys >> keys.dtype.type(gbits)
    t = np.arange(n_tiles, dtype=keys.dtype)
    ranges = np.stack([np.searchsorted(tile_of, t, side="left"),
                       np.searchsorted(tile_of, t, side="right")], axis=1).astype(np.uint32)
    ranges[ranges[:, 0] == ranges[:, 1]] = 0       # an empty tile is (0, 0)
    return keys, ranges, counts
