"""The single-canvas binning has two ways to put the (tile, Gaussian) keys in
(tile, depth) order: a two-level stable counting sort over the rectangles
(32-bit keys, at most 512 x 512 tiles; Section 3.4's order from the tile
rows, then the columns of each row) and the LSD radix passes over the tile
bits (wider grids, 64-bit keys, and bs_bin_tiles_static, whose fixed
scratch is sized for them).  Both must give the oracle's keys, ranges and
pair counts bit for bit: at the two-level path's largest grid, with row
lists of many level-2 chunks and tiles of about a thousand pairs, just past its
limits, against each other on the same inputs, and with the graph-safe
call (grids sized by the capacity, nothing read back)."""

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def _table(seed, W, H, n, ext=(0.0, 40.0), y_band=None):
    """A seeded float32 Gaussian table: means over and around the canvas (or
    in a horizontal band), support boxes of ext px, a few culled records."""
    rng = np.random.default_rng(seed)
    rec = np.zeros((n, 12), dtype=np.float32)
    rec[:, 0] = rng.uniform(-30, W + 30, n)
    rec[:, 1] = rng.uniform(-30, H + 30, n) if y_band is None else rng.uniform(*y_band, n)
    rec[:, 10] = rng.uniform(*ext, n)
    rec[:, 11] = rng.uniform(*ext, n)
    rec[::61, 10] = -1.0
    return rec


def _check_against_oracle(bs, rec, W, H, tile):
    """Keys, ranges and pair count of bs_bin_tiles against the oracle's (32-bit
    keys: the cases here all fit them)."""
    keys, ranges, _ = oracle.tile_keys(rec, W, H, tile)
    assert keys.dtype == np.uint32
    gauss = torch.as_tensor(rec, device="cuda")
    b = bs.Binning(bs.Canvas(W, H, tile), "cuda", pair_capacity=keys.shape[0] + 64).run(gauss)
    assert b.device_status() == 0
    assert b.n_pairs == keys.shape[0]
    assert np.array_equal(b.keys[:b.n_pairs].cpu().numpy().view(np.uint32), keys)
    assert np.array_equal(b.ranges.cpu().numpy().view(np.uint32), ranges)
    return gauss, b


def test_two_level_at_its_largest_grid(bs):
    """4096 x 4096 at 8 px tiles: 512 x 512 tiles, the largest grid the
    two-level sort takes; 16,000 Gaussians (63 level-1 chunks; 14 + 18 key
    bits), about half a million pairs; the radix passes of
    bs_bin_tiles_static give the same keys."""
    W = H = 4096
    rec = _table(7, W, H, 16000)
    gauss, b = _check_against_oracle(bs, rec, W, H, 8)
    assert b.n_pairs > 400_000
    canvas = bs.Canvas(W, H, 8)
    keys = torch.full((b.n_pairs + 64,), -1, dtype=torch.int32, device="cuda")
    ranges = torch.full((canvas.n_tiles, 2), -1, dtype=torch.int32, device="cuda")
    n_pairs = bs.bin_tiles_static(gauss, canvas, keys, ranges)
    torch.cuda.synchronize()
    assert n_pairs == b.n_pairs
    assert torch.equal(keys[:n_pairs], b.keys[:n_pairs])
    assert torch.equal(ranges, b.ranges)


def test_two_level_with_long_row_lists(bs):
    """A 2048 x 48 canvas (128 x 3 tiles of 16 px) with 6,000 Gaussians in
    its band: each row list holds about 6,000 entries (47 level-2 chunks) and
    a tile up to about a thousand pairs."""
    W, H = 2048, 48
    rec = _table(8, W, H, 6000, ext=(10.0, 300.0), y_band=(0.0, 48.0))
    _, b = _check_against_oracle(bs, rec, W, H, 16)
    counts = (b.ranges[:, 1] - b.ranges[:, 0]).cpu().numpy()
    assert counts.max() > 800


@pytest.mark.parametrize("W,H", [(4104, 64), (64, 4104)])
def test_past_the_two_level_limits(bs, W, H):
    """513 tile columns or rows of 8 px: the radix passes."""
    rec = _table(9, W, H, 6000, ext=(0.0, 30.0))
    _check_against_oracle(bs, rec, W, H, 8)


def test_two_level_graph_safe_call_matches_the_synchronising_one(bs):
    """bs_bin_tiles_async with a capacity well above the pairs (its grids are
    sized by the capacity, and the level-2 kernels read their chunk count on
    the device) gives the keys and ranges of bs_bin_tiles."""
    W, H = 1536, 1024
    rec = _table(10, W, H, 20000)
    gauss, b = _check_against_oracle(bs, rec, W, H, 16)
    a = bs.Binning(bs.Canvas(W, H, 16), "cuda").prepare(rec.shape[0], 3 * b.n_pairs)
    a.run_async(gauss)
    st, n = a.result()
    assert st == bs.BS_OK and n == b.n_pairs
    assert torch.equal(a.keys[:n], b.keys[:n])
    assert torch.equal(a.ranges, b.ranges)
