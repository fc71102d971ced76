"""Pins of the oracle's tile binning (Section 3.4): per-pixel enumeration,
exact culling against the brute-force alpha rule, key and range structure."""

import numpy as np
import pytest
import torch

import oracle
from oracle.curves import SampleCfg, table_to_f32, table_from_f32
from oracle.binning import key_bits, tile_keys, tile_rects_f32
from paper_2503_16424_gb300 import synth


def _table_f32(seed, W, H, n_open, n_closed, cfg, style="local"):
    c = synth.make_curves(seed, W, H, n_open, n_closed, style=style)
    curves = {k: torch.as_tensor(v, dtype=torch.float64) for k, v in c.as_dict().items()}
    tab = oracle.gaussian_table(curves, cfg)
    return table_to_f32(tab)


def test_rects_equal_per_pixel_enumeration():
    """Tile set of a Gaussian = tiles of the pixels x whose index lies in
    [xlo, xhi] (float32 bounds), enumerated pixel by pixel."""
    W, H, T = 53, 37, 8
    rec = _table_f32(1, W, H, 4, 2, SampleCfg(g_open=9, rows_closed=3, k_closed=4))
    rec[0, 10] = -1.0                    # culled
    rec[1, 0] = np.float32(np.nan)       # non-finite
    rec[2, 0] = 1e30                     # far away
    tx0, tx1, ty0, ty1, ok = tile_rects_f32(rec, W, H, T)
    f = np.float32
    for g in range(rec.shape[0]):
        mx, my, ex, ey = rec[g, 0], rec[g, 1], rec[g, 10], rec[g, 11]
        with np.errstate(invalid="ignore", over="ignore"):
            xlo, xhi = (mx - ex) - f(0.5), (mx + ex) - f(0.5)
            ylo, yhi = (my - ey) - f(0.5), (my + ey) - f(0.5)
        tiles = set()
        if ex >= 0 and ey >= 0 and np.isfinite([xlo, xhi, ylo, yhi]).all():
            for y in range(H):
                for x in range(W):
                    if xlo <= x <= xhi and ylo <= y <= yhi:
                        tiles.add((y // T, x // T))
        got = set()
        if ok[g]:
            got = {(ty, tx) for ty in range(ty0[g], ty1[g] + 1) for tx in range(tx0[g], tx1[g] + 1)}
        assert got == tiles, g


@pytest.mark.parametrize("W,H,T", [(64, 48, 16), (45, 29, 8)])
def test_culling_is_exact(W, H, T):
    """Every (pixel, Gaussian) with alpha >= 1/255 (fp64 rule on the float32
    table) lies in a tile listed for that Gaussian."""
    rec = _table_f32(2, W, H, 6, 3, SampleCfg(g_open=10, rows_closed=4, k_closed=5))
    keys, ranges, counts = tile_keys(rec, W, H, T)
    tab = table_from_f32(rec)
    gbits, _ = key_bits(rec.shape[0], ranges.shape[0])
    listed = {(int(k) >> gbits, int(k) & ((1 << gbits) - 1)) for k in keys}
    tiles_x = -(-W // T)
    ys, xs = np.mgrid[0:H, 0:W]
    px, py = torch.as_tensor(xs.ravel() + 0.5), torch.as_tensor(ys.ravel() + 0.5)
    from oracle.raster import _alpha_raw
    a = _alpha_raw(tab, px, py)
    hit = torch.nonzero(a >= 1 / 255)
    assert hit.shape[0] > 100
    for p, g in hit.tolist():
        t = (int(ys.ravel()[p]) // T) * tiles_x + int(xs.ravel()[p]) // T
        assert (t, g) in listed


def test_keys_sorted_and_ranges_consistent():
    W, H, T = 70, 50, 16
    rec = _table_f32(3, W, H, 8, 4, SampleCfg(g_open=12, rows_closed=4, k_closed=6))
    keys, ranges, counts = tile_keys(rec, W, H, T)
    assert keys.dtype == np.uint32 and np.all(np.diff(keys.astype(np.int64)) > 0)
    assert keys.shape[0] == counts.sum()
    gbits, tbits = key_bits(rec.shape[0], ranges.shape[0])
    for t, (s, e) in enumerate(ranges):
        seg = keys[s:e]
        assert np.all((seg >> gbits) == t)
        g = seg & ((1 << gbits) - 1)
        assert np.all(np.diff(g.astype(np.int64)) > 0)      # front to back
    assert ranges[:, 1].max() == keys.shape[0]
    assert np.bincount(keys & ((1 << gbits) - 1), minlength=rec.shape[0]).tolist() == counts.tolist()


def test_key_bits():
    assert key_bits(262144, 16384) == (18, 14)
    assert key_bits(1024, 256) == (10, 8)
    assert key_bits(1, 1) == (1, 1)
    assert key_bits(24576, 4096) == (15, 12)
