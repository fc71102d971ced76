"""Tile sides 8 and 32 (the 16 x 16 tiling is covered by the other parity
tests): tile keys bit-exact against the oracle's binning at that side,
forward pixels against the oracle's brute force, gradients against the
oracle, on one canvas and on a batch.

The tiling decides only which Gaussians a pixel's list holds; those left
out cannot reach the pixel (alpha < 1/255, culling is exact), so every pixel
blends the same Gaussians in the same order whatever the tile side: images
and final transmittances equal the 16 x 16 results bit for bit."""

import numpy as np
import pytest
import torch

import oracle
from oracle.pipeline import as_curves, sample_vjp
from tests.gpu_cases import CASES, arrays, blend_grad_bound, curve_grad_bound, grad_check, ocfg, table_from_f32
from tests.test_gpu_batch import KEYS, OPEN_KEYS, SPECS, make_batch, ocfg_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def _plain(bs, case, tile):
    from paper_2503_16424_gb300.raster import Rasterizer
    arr = arrays(case)
    cfg = bs.SampleCfg(g_open=case.g_open, rows_closed=case.rows, k_closed=case.kc)
    curves = bs.CurveSet.from_arrays(arr, device="cuda")
    r = Rasterizer(bs.Canvas(case.W, case.H, tile, case.bg), cfg, curves.n_open, curves.n_closed, pair_capacity=1024)
    r.forward(curves)
    torch.cuda.synchronize()
    return arr, curves, r


@pytest.mark.parametrize("tile", [8, 32])
@pytest.mark.parametrize("name", ["ragged", "mixed", "dense"])
def test_plain_path_at_tile_side(bs, name, tile):
    case = CASES[name]
    arr, curves, r = _plain(bs, case, tile)
    rec = r.gauss.cpu().numpy()
    keys, ranges, counts = oracle.tile_keys(rec, case.W, case.H, tile)
    n = r.binning.n_pairs
    assert n == keys.shape[0]
    assert np.array_equal(r.binning.keys[:n].cpu().numpy().view(np.uint32), keys)
    assert np.array_equal(r.binning.ranges.cpu().numpy().view(np.uint32), ranges)
    ref = oracle.render_image(table_from_f32(rec), case.W, case.H, bg=case.bg, margin=1e-5)
    ok = ~ref["flag"]
    err = (r.img.cpu().double() - ref["img"]).abs().amax(0)
    assert float(err[ok].max()) <= 1e-5
    assert float(((~ok) & (err > 1e-5)).double().mean()) < 1e-4
    _, _, r16 = _plain(bs, case, 16)
    assert torch.equal(r.img, r16.img)
    assert torch.equal(r.T, r16.T)
    # gradients of a loss on the unflagged pixels, against the oracle
    ok_g = ~oracle.render_image(table_from_f32(rec), case.W, case.H, bg=case.bg, margin=1e-4)["flag"]
    rng = np.random.default_rng(tile)
    dimg = torch.as_tensor(rng.normal(0, 1e-3, (3, case.H, case.W)).astype(np.float32), device="cuda")
    dimg *= ok_g.to("cuda")[None].float()
    grad = r.backward(curves, dimg)
    ys, xs = torch.meshgrid(torch.arange(case.H, dtype=torch.float64), torch.arange(case.W, dtype=torch.float64),
                            indexing="ij")
    dC = dimg.cpu().double().permute(1, 2, 0).reshape(-1, 3)
    dtab = oracle.render_grads(table_from_f32(rec), xs.reshape(-1), ys.reshape(-1), dC, bg=case.bg)
    _, o_first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], ocfg(case))
    dref = sample_vjp(as_curves(arr), ocfg(case), dtab, o_first)
    cb = curve_grad_bound(arr, ocfg(case), o_first, blend_grad_bound(rec, case.W, case.H, dC, case.bg, tile), dtab)
    for k in KEYS:
        if getattr(grad, k).numel():
            assert grad_check(getattr(grad, k).cpu(), dref[k], cb[k]) <= 1.0, k


@pytest.mark.parametrize("tile", [8, 32])
def test_batch_at_tile_side(bs, tile):
    from paper_2503_16424_gb300.batch import BatchRasterizer
    images, arrs, targets, curves, target = make_batch(bs, SPECS)
    rs = {}
    for t in (16, tile):
        r = BatchRasterizer(images, tile=t, pair_capacity=1 << 16)
        r.fit_capacity(curves)
        r.forward(curves, target)
        torch.cuda.synchronize()
        assert r.batch.status()[0] == bs.BS_OK
        rs[t] = r
    r, r16 = rs[tile], rs[16]
    assert torch.equal(r.img, r16.img)
    assert torch.equal(r.T, r16.T)
    assert torch.equal(r.dimg, r16.dimg)
    # per-tile float partial sums of the loss: equal up to their order
    assert np.allclose(r.loss.cpu().numpy(), r16.loss.cpu().numpy(), rtol=1e-6, atol=0)
    gauss = r.gauss.cpu().numpy()
    vals = r.vals.cpu().numpy().view(np.uint32)
    ranges = r.ranges.cpu().numpy().view(np.uint32)
    for b, im in enumerate(images):
        g0, n = r.batch.gauss0[b], r.batch.n_gauss_of[b]
        if n == 0:
            continue
        keys, oranges, _ = oracle.tile_keys(gauss[g0:g0 + n], im.width, im.height, tile)
        nt = (-(-im.width // tile)) * (-(-im.height // tile))
        gbits, _ = oracle.key_bits(n, nt)
        local = keys & np.uint32((1 << gbits) - 1)
        for t in range(nt):
            s, e = ranges[r.batch.tile0[b] + t]
            assert np.array_equal(vals[s:e].astype(np.int64) - g0, local[oranges[t, 0]:oranges[t, 1]].astype(np.int64))
    # backward: the same curve gradients as the 16 x 16 tiling up to the
    # order of the per-Gaussian float sums: within 1e-4 relative plus twice
    # each image's float32 rounding bound (one for either tiling)
    g = curves.zeros_like()
    g16 = curves.zeros_like()
    r.backward(curves, r.dimg, g)
    r16.backward(curves, r16.dimg, g16)
    for b, (im, arr) in enumerate(zip(images, arrs)):
        g0, n = r.batch.gauss0[b], r.batch.n_gauss_of[b]
        if n == 0:
            continue
        oc = ocfg_of(im)
        _, o_first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], oc)
        ys, xs = torch.meshgrid(torch.arange(im.height, dtype=torch.float64),
                                torch.arange(im.width, dtype=torch.float64), indexing="ij")
        dC = r16.batch.image(r16.dimg, b).cpu().double().permute(1, 2, 0).reshape(-1, 3)
        dtab = oracle.render_grads(table_from_f32(gauss[g0:g0 + n]), xs.reshape(-1), ys.reshape(-1), dC, bg=im.bg)
        gb = blend_grad_bound(gauss[g0:g0 + n], im.width, im.height, dC, im.bg, min(tile, 16))
        cb = curve_grad_bound(arr, oc, o_first, gb, dtab)
        for k in KEYS:
            sl = (slice(r.batch.open0[b], r.batch.open0[b] + im.n_open) if k in OPEN_KEYS else
                  slice(r.batch.closed0[b], r.batch.closed0[b] + im.n_closed))
            a, c = getattr(g, k)[sl], getattr(g16, k)[sl]
            if a.numel():
                assert grad_check(a.cpu(), c.cpu(), 2 * cb[k], rel=1e-4) <= 1.0, (b, k)


def test_autotuner_picks_first_sampling_within_threshold_and_fastest_tile(bs):
    from paper_2503_16424_gb300 import autotune
    images, arrs, targets, curves, target = make_batch(bs, SPECS[:3] + SPECS[5:])
    tuned, table = autotune.pick_sampling(images, curves, psnr_min=35.0)
    for b, im in enumerate(tuned):
        entry = (im.sample.g_open, im.sample.rows_closed, im.sample.k_closed)
        i = autotune.SCHEDULE.index(entry)
        earlier = [table[e][b] for e in autotune.SCHEDULE[:i]]
        assert all(db < 35.0 for db in earlier), b
        assert table[entry][b] >= 35.0 or entry == autotune.SCHEDULE[-1], b
        assert (im.width, im.height, im.n_open, im.n_closed) == (images[b].width, images[b].height,
                                                                 images[b].n_open, images[b].n_closed)
    tile, ms = autotune.pick_tile(tuned, curves, target, steps=2)
    assert set(ms) == {8, 16, 32} and ms[tile] == min(ms.values())


def test_plain_binning_with_wide_keys(bs):
    """18 tile bits (a 4100 x 4100 canvas in 8 x 8 tiles) + 16 Gaussian bits
    > 32: 64-bit keys, tile_keys holds each tile's Gaussian indices front to
    back; lists bit-exact against the oracle, sampled pixels against its
    brute force."""
    from paper_2503_16424_gb300 import synth
    from paper_2503_16424_gb300.raster import Rasterizer
    W = H = 4100
    arr = synth.make_curves(41, W, H, 600, 400, style="local").as_dict()
    cfg = bs.SampleCfg(g_open=32, rows_closed=4, k_closed=8)
    curves = bs.CurveSet.from_arrays(arr, device="cuda")
    r = Rasterizer(bs.Canvas(W, H, 8, (0.1, 0.2, 0.3)), cfg, curves.n_open, curves.n_closed, pair_capacity=1 << 20)
    assert r.n_gauss == 600 * 32 + 400 * 32 and (r.n_gauss - 1).bit_length() + (513 * 513 - 1).bit_length() > 32
    r.forward(curves)
    torch.cuda.synchronize()
    rec = r.gauss.cpu().numpy()
    keys, ranges, counts = oracle.tile_keys(rec, W, H, 8)
    assert keys.dtype == np.uint64
    n = r.binning.n_pairs
    assert n == keys.shape[0]
    gbits, _ = oracle.key_bits(rec.shape[0], ranges.shape[0])
    assert np.array_equal(r.binning.keys[:n].cpu().numpy().view(np.uint32).astype(np.uint64),
                          keys & np.uint64((1 << gbits) - 1))
    assert np.array_equal(r.binning.ranges.cpu().numpy().view(np.uint32), ranges.astype(np.uint32))
    rng = np.random.default_rng(7)
    xs, ys = rng.integers(0, W, 96), rng.integers(0, H, 96)
    px = oracle.render_pixels(table_from_f32(rec), xs, ys, bg=(0.1, 0.2, 0.3))
    got = r.img.cpu().double()[:, torch.as_tensor(ys), torch.as_tensor(xs)].T
    ok = ~px["flag"]
    assert float((got - px["C"]).abs().amax(1)[ok].max()) <= 1e-5
    # the same image as 16 x 16 tiles with 32-bit keys
    r16 = Rasterizer(bs.Canvas(W, H, 16, (0.1, 0.2, 0.3)), cfg, curves.n_open, curves.n_closed, pair_capacity=1 << 20)
    r16.forward(curves)
    assert torch.equal(r.img, r16.img)
