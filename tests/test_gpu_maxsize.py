"""The largest canvas side the calls accept (32768 px, bs_canvas), on thin
canvases 32768 x 48 and 48 x 32768 (2048 x 3 tiles of 16 px): draw order
and sampling against the oracle, every tile key and range bit-exact,
sampled pixels of the blend within 1e-5 of the oracle's brute force, and
the per-Gaussian gradients of a loss on a crop within the gradient bar (as
tests/test_gpu_fullsize.py does at 2048 x 2048).  A 32768 x 32768 canvas
(4.2 M tiles, 64-bit keys, the unfused tile scan) renders a few curves with
the oracle's pixels near them and the background everywhere else."""

import numpy as np
import pytest
import torch

import oracle
from oracle.curves import SampleCfg as OCfg, table_from_f32
from oracle.pipeline import as_curves
from paper_2503_16424_gb300 import synth
from tests.gpu_cases import blend_grad_bound, grad_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def _near(tab, x0, y0, w, h):
    ex, ey = tab["ext_x"], tab["ext_y"]
    return ((ex >= 0) & (tab["mx"] + ex >= x0 + 0.5) & (tab["mx"] - ex <= x0 + w - 0.5)
            & (tab["my"] + ey >= y0 + 0.5) & (tab["my"] - ey <= y0 + h - 0.5))


@pytest.mark.parametrize("W,H,seed", [(32768, 48, 31), (48, 32768, 32)])
def test_thin_canvas_at_the_largest_side(bs, W, H, seed):
    from paper_2503_16424_gb300.raster import Rasterizer
    arr = synth.make_curves(seed, W, H, 24, 12, style="local").as_dict()
    cfg = bs.SampleCfg(g_open=32, rows_closed=4, k_closed=8)
    ocfg = OCfg(g_open=32, rows_closed=4, k_closed=8)
    bg = (0.1, 0.2, 0.3)
    curves = bs.CurveSet.from_arrays(arr, device="cuda")
    r = Rasterizer(bs.Canvas(W, H, 16, bg), cfg, curves.n_open, curves.n_closed, pair_capacity=1 << 16)
    img = r.forward(curves)
    torch.cuda.synchronize()
    rank, first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], ocfg)
    assert np.array_equal(r.rank.cpu().numpy(), rank) and np.array_equal(r.first.cpu().numpy(), first)
    with torch.no_grad():
        tab64 = oracle.gaussian_table(as_curves(arr), ocfg, first)
    rec = r.gauss.cpu().numpy()
    ref = np.stack([tab64[k].numpy() for k in ("mx", "my", "ux", "uy", "isx", "isy")], 1)
    got = rec[:, :6].astype(np.float64)
    assert np.abs(got[:, 0:2] - ref[:, 0:2]).max() / max(W, H) <= 1e-5
    assert np.abs(got[:, 2:4] - ref[:, 2:4]).max() <= 1e-5
    assert (np.abs(got[:, 4:6] - ref[:, 4:6]) / ref[:, 4:6]).max() <= 1e-5
    # binning on the GPU's own table, bit for bit
    keys, ranges, _ = oracle.tile_keys(rec, W, H, 16)
    assert r.binning.n_pairs == keys.shape[0] > 0
    assert np.array_equal(r.binning.keys[:r.binning.n_pairs].cpu().numpy().view(np.uint32), keys)
    assert np.array_equal(r.binning.ranges.cpu().numpy().view(np.uint32), ranges)
    # sampled pixels: random ones and those at Gaussian means
    tab = table_from_f32(rec)
    rng = np.random.default_rng(seed)
    pick = rng.choice(rec.shape[0], 96, replace=False)
    xs = np.concatenate([rng.integers(0, W, 96), np.clip(rec[pick, 0].astype(np.int64), 0, W - 1)])
    ys = np.concatenate([rng.integers(0, H, 96), np.clip(rec[pick, 1].astype(np.int64), 0, H - 1)])
    pf = oracle.render_pixels(tab, xs.astype(np.float64), ys.astype(np.float64), bg=bg, margin=1e-5)
    got_px = img.cpu().numpy()[:, ys, xs].T.astype(np.float64)
    err = np.abs(got_px - pf["C"].numpy()).max(1)
    flag = pf["flag"].numpy()
    print(f"{W}x{H}: {keys.shape[0]} pairs; {xs.size} pixels, max err {err[~flag].max():.1e}, flagged {flag.sum()}")
    assert err[~flag].max() <= 1e-5 and int((flag & (err > 1e-5)).sum()) == 0
    # backward of a loss on a 32 x 32 crop around the middle curve's first Gaussian
    cx, cy = int(rec[pick[0], 0]), int(rec[pick[0], 1])
    side_x, side_y = min(32, W), min(32, H)
    x0, y0 = int(np.clip(cx - 16, 0, W - side_x)), int(np.clip(cy - 16, 0, H - side_y))
    yy, xx = torch.meshgrid(torch.arange(y0, y0 + side_y, dtype=torch.float64),
                            torch.arange(x0, x0 + side_x, dtype=torch.float64), indexing="ij")
    cxs, cys = xx.reshape(-1), yy.reshape(-1)
    idx = torch.nonzero(_near(tab, x0, y0, side_x, side_y))[:, 0]
    sub = {k: v[idx] for k, v in tab.items()}
    pc = oracle.render_pixels(sub, cxs, cys, bg=bg, margin=1e-4)
    dC = torch.as_tensor(rng.normal(0, 1e-6, (side_x * side_y, 3)))
    dC[pc["flag"]] = 0.0
    dimg = torch.zeros(3, H, W, dtype=torch.float32)
    dimg[:, y0:y0 + side_y, x0:x0 + side_x] = dC.float().reshape(side_y, side_x, 3).permute(2, 0, 1)
    dgauss, _ = bs.render_bwd(r.gauss, r.canvas, r.binning, r.T, r.nc, dimg.cuda())
    g = dgauss.cpu().double()
    others = torch.ones(g.shape[0], dtype=torch.bool)
    others[idx] = False
    assert float(g[others].abs().max()) == 0.0
    refg = oracle.render_grads(sub, cxs, cys, dC.float().double(), bg=bg)
    bound = blend_grad_bound(rec[idx.numpy()], W, H, dC.float().double(), bg, xs=cxs, ys=cys, tab=sub)
    cols = {"mx": 0, "my": 1, "ux": 2, "uy": 3, "isx": 4, "isy": 5, "o": 6, "col": slice(7, 10)}
    for k, c in cols.items():
        assert grad_check(g[idx][:, c], refg[k], bound[k]) <= 1.0, k


def test_square_canvas_at_the_largest_side(bs):
    """32768 x 32768 with twelve small curves (1,536 Gaussians): the tile
    scan runs unfused over 4.2 M tiles and the keys are 64-bit (22 tile
    bits + 11 Gaussian bits); every tile range is bit-exact, pixels at the
    curves match the oracle and a sample of the rest is the background."""
    from paper_2503_16424_gb300.raster import Rasterizer
    W = H = 32768
    rng = np.random.default_rng(33)
    arr = synth.make_curves(34, 512, 512, 6, 6, style="local").as_dict()
    shift = rng.uniform(0, W - 512, (12, 2)).astype(np.float32)   # one place per curve across the canvas
    arr["open_ctrl"] = arr["open_ctrl"] + shift[:6, None, :]
    arr["closed_ctrl"] = arr["closed_ctrl"] + shift[6:, None, :]
    cfg = bs.SampleCfg(g_open=128, rows_closed=8, k_closed=16)
    ocfg = OCfg(g_open=128, rows_closed=8, k_closed=16)
    bg = (0.25, 0.5, 0.75)
    curves = bs.CurveSet.from_arrays(arr, device="cuda")
    r = Rasterizer(bs.Canvas(W, H, 16, bg), cfg, 6, 6, pair_capacity=1 << 16)
    img = r.forward(curves)
    torch.cuda.synchronize()
    assert r.binning.device_status() == 0
    _, first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], ocfg)
    assert np.array_equal(r.first.cpu().numpy(), first)
    rec = r.gauss.cpu().numpy()
    assert rec.shape[0] == 1536
    keys, ranges, _ = oracle.tile_keys(rec, W, H, 16)
    assert keys.dtype == np.uint64                         # the wide-key path
    assert r.binning.n_pairs == keys.shape[0]
    assert np.array_equal(r.binning.ranges.cpu().numpy().view(np.uint32), ranges)
    gbits, _ = oracle.key_bits(rec.shape[0], (W // 16) * (H // 16))
    assert np.array_equal(r.binning.keys[:r.binning.n_pairs].cpu().numpy().view(np.uint32),
                          (keys & np.uint64((1 << gbits) - 1)).astype(np.uint32))
    tab = table_from_f32(rec)
    pick = rng.choice(rec.shape[0], 64, replace=False)
    xs = np.clip(rec[pick, 0].astype(np.int64), 0, W - 1)
    ys = np.clip(rec[pick, 1].astype(np.int64), 0, H - 1)
    pf = oracle.render_pixels(tab, xs.astype(np.float64), ys.astype(np.float64), bg=bg, margin=1e-5)
    got_px = img[:, torch.as_tensor(ys, device="cuda"), torch.as_tensor(xs, device="cuda")].T.cpu().double().numpy()
    err = np.abs(got_px - pf["C"].numpy()).max(1)
    flag = pf["flag"].numpy()
    assert err[~flag].max() <= 1e-5
    # a sample of pixels away from every Gaussian's box: the background
    fx = rng.integers(0, W, 4096)
    fy = rng.integers(0, H, 4096)
    far = np.ones(fx.size, bool)
    for g in range(rec.shape[0]):
        far &= ~((np.abs(fx + 0.5 - rec[g, 0]) <= rec[g, 10] + 1) & (np.abs(fy + 0.5 - rec[g, 1]) <= rec[g, 11] + 1))
    vals = img[:, torch.as_tensor(fy[far], device="cuda"), torch.as_tensor(fx[far], device="cuda")].cpu().numpy()
    assert np.array_equal(vals, np.broadcast_to(np.array(bg, np.float32)[:, None], vals.shape))
