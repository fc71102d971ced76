"""End-to-end step on the GPU against the fp64 oracle and finite differences,
the autograd wrapper, edge cases, and the bounded-wait fault path."""

import numpy as np
import pytest
import torch

import oracle
from oracle.curves import SampleCfg as OCfg, table_to_f32, table_from_f32
from oracle.pipeline import as_curves, loss_only, sample_vjp
from paper_2503_16424_gb300 import synth
from tests.gpu_cases import blend_grad_bound, curve_grad_bound, grad_check, grad_rel_err

pytestmark = pytest.mark.gpu

KEYS = ("open_ctrl", "open_width", "open_color", "open_opac", "closed_ctrl", "closed_color", "closed_opac")


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def _setup(bs, W, H, arr, g_open, rows, kc, bg=(0.0, 0.0, 0.0), tangent_mode=0):
    from paper_2503_16424_gb300.raster import Rasterizer
    cfg = bs.SampleCfg(g_open=g_open, rows_closed=rows, k_closed=kc, tangent_mode=tangent_mode)
    curves = bs.CurveSet.from_arrays(arr, device="cuda")
    r = Rasterizer(bs.Canvas(W, H, 16, bg), cfg, curves.n_open, curves.n_closed, pair_capacity=2048)
    return cfg, curves, r


@pytest.mark.parametrize("seed,W,H,no,nc,tmode", [(5, 64, 48, 6, 3, 0), (6, 96, 80, 10, 5, 0),
                                                   (7, 80, 64, 8, 4, 1)])
def test_step_matches_oracle_and_fd(bs, seed, W, H, no, nc, tmode):
    bg = (0.1, 0.2, 0.3)
    arr = synth.make_curves(seed, W, H, no, nc, style="local").as_dict()
    g_open, rows, kc = 10, 4, 6
    cfg, curves, r = _setup(bs, W, H, arr, g_open, rows, kc, bg, tangent_mode=tmode)
    ocfg = OCfg(g_open=g_open, rows_closed=rows, k_closed=kc, tangent_mode=tmode)
    tgt_np = synth.procedural_target(seed, W, H, 6)
    tgt = torch.as_tensor(tgt_np, device="cuda")
    img = r.forward(curves)
    # oracle: its own sampling (fp64) of the same curves
    oc = as_curves(arr)
    _, first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], ocfg)
    tab = oracle.gaussian_table(oc, ocfg, first)
    ref = oracle.render_image({k: v.detach() for k, v in tab.items()}, W, H, bg=bg, margin=1e-5)
    err = (img.cpu().double() - ref["img"]).abs().amax(0)
    excused = ref["flag"] & (err > 1e-5)
    print(f"step {W}x{H}: flagged {float(ref['flag'].double().mean()):.1e}, "
          f"pixel err {float(err[~ref['flag']].max()):.1e}, excused {int(excused.sum())}")
    assert float(err[~ref["flag"]].max()) <= 1e-5
    assert float(excused.double().mean()) < 1e-4
    # gradients of the L2 loss restricted to pixels with no threshold
    # decision within 1e-4 (a kink of the blend), on both sides
    ok = ~oracle.render_image({k: v.detach() for k, v in tab.items()}, W, H, bg=bg, margin=1e-4)["flag"]
    _, dimg = bs.l2_loss_grad(img, tgt)
    dimg = dimg * ok.to("cuda")[None].float()
    grad = r.backward(curves, dimg)
    ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64),
                            indexing="ij")
    dC = dimg.cpu().double().permute(1, 2, 0).reshape(-1, 3)
    dtab = oracle.render_grads({k: v.detach() for k, v in tab.items()}, xs.reshape(-1), ys.reshape(-1), dC, bg=bg)
    dref = sample_vjp(oc, ocfg, dtab, first)
    gb = blend_grad_bound(r.gauss.cpu().numpy(), W, H, dC, bg, tab={k: v.detach() for k, v in tab.items()})
    cb = curve_grad_bound(arr, ocfg, first, gb, dtab)
    errs = {k: grad_rel_err(getattr(grad, k).cpu(), dref[k]) for k in KEYS}
    ratio = {k: grad_check(getattr(grad, k).cpu(), dref[k], cb[k]) for k in KEYS}
    print("  curve grad rel errs: " + ", ".join(f"{k} {v:.1e}" for k, v in errs.items()) +
          "; of the bar: " + ", ".join(f"{k} {v:.2f}" for k, v in ratio.items()))
    for k, e in ratio.items():
        assert e <= 1.0, k
    # central finite differences of the oracle loss (same mask) for a few parameters
    mask = ok.double()

    def masked_loss(cv):
        with torch.no_grad():
            t = oracle.gaussian_table(cv, ocfg, first)
            im = oracle.render_image(t, W, H, bg=bg)["img"]
            d = (im - torch.as_tensor(tgt_np, dtype=torch.float64)) * mask[None]
            return float((d * d).sum() / d.numel())
    def central(k, i, h):
        plus = {kk: v.clone() for kk, v in oc.items()}
        minus = {kk: v.clone() for kk, v in oc.items()}
        plus[k].view(-1)[i] += h
        minus[k].view(-1)[i] -= h
        return (masked_loss(plus) - masked_loss(minus)) / (2 * h)

    # the bar of the curve gradients, with the finite difference's own error
    # estimated from a second step (central differences err ~ h^2, so
    # |fd(h) - fd(2h)| / 3 estimates the error of fd(h))
    rng = np.random.default_rng(seed)
    for k in ("open_ctrl", "closed_ctrl", "open_width", "closed_color"):
        g = getattr(grad, k).cpu().double().reshape(-1)
        gmax = float(g.abs().max())
        bnd = cb[k].reshape(-1)
        for i in rng.choice(g.numel(), size=4, replace=False):
            h = 1e-5 * max(1.0, abs(float(oc[k].reshape(-1)[i])))
            fd, fd2 = central(k, i, h), central(k, i, 2 * h)
            allow = 1e-3 * max(abs(fd), 1e-6 * gmax) + float(bnd[i]) + abs(fd - fd2) / 3
            assert abs(float(g[i]) - fd) <= allow, (k, i, float(g[i]), fd, fd2)


def test_autograd_function_matches_rasterizer(bs):
    from paper_2503_16424_gb300.raster import rasterize
    W, H = 80, 64
    arr = synth.make_curves(8, W, H, 5, 3, style="local").as_dict()
    cfg, curves, r = _setup(bs, W, H, arr, 8, 4, 5)
    params = bs.CurveSet(**{k: getattr(curves, k).clone().requires_grad_(True) for k in KEYS})
    img = rasterize(r, params)
    tgt = torch.as_tensor(synth.procedural_target(8, W, H, 4), device="cuda")
    loss = ((img - tgt) ** 2).mean()
    loss.backward()
    loss2, grad = r.step(curves, tgt)
    assert abs(loss.item() - loss2.item()) <= 1e-6 * loss2.item()
    for k in KEYS:
        a, b = getattr(params, k).grad, getattr(grad, k)
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * float(b.abs().max()) + 1e-12), k


def test_empty_and_offscreen(bs):
    # no curves at all
    W, H = 40, 24
    empty = synth.make_curves(0, W, H, 0, 0).as_dict()
    cfg, curves, r = _setup(bs, W, H, empty, 8, 3, 4, bg=(0.25, 0.5, 0.75))
    img = r.forward(curves)
    assert r.binning.n_pairs == 0
    assert torch.allclose(img, torch.tensor([0.25, 0.5, 0.75], device="cuda")[:, None, None].expand(3, H, W))
    assert torch.all(r.T == 1) and torch.all(r.nc == 0)
    # every curve far outside the canvas
    arr = synth.make_curves(1, W, H, 4, 2, style="local").as_dict()
    arr["open_ctrl"] += 1000.0
    arr["closed_ctrl"] -= 1000.0
    cfg, curves, r = _setup(bs, W, H, arr, 8, 3, 4)
    img = r.forward(curves)
    assert r.binning.n_pairs == 0 and float(img.abs().max()) == 0.0
    loss, grad = r.step(curves, torch.ones(3, H, W, device="cuda"))
    for k in KEYS:
        assert float(getattr(grad, k).abs().max()) == 0.0


def test_degenerate_curves_match_oracle(bs):
    """Coincident control points (zero-length differences: theta = 0, sigma
    from eps only), a 1x1 canvas, and closed curves collapsed to a segment."""
    W, H = 33, 17
    arr = synth.make_curves(2, W, H, 3, 2, style="local").as_dict()
    arr["open_ctrl"][0] = arr["open_ctrl"][0, :1]          # all 10 points equal
    arr["closed_ctrl"][0] = arr["closed_ctrl"][0, :1]      # all 12 points equal
    arr["closed_ctrl"][1, 7:12] = arr["closed_ctrl"][1, 5:0:-1]  # B == A: zero-area fill
    ocfg = OCfg(g_open=7, rows_closed=3, k_closed=5)
    cfg, curves, r = _setup(bs, W, H, arr, 7, 3, 5)
    r.forward(curves)
    _, first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], ocfg)
    tab = oracle.gaussian_table(as_curves(arr), ocfg, first)
    got = r.gauss.cpu().numpy().astype(np.float64)
    ref = table_to_f32(tab).astype(np.float64)
    assert np.isfinite(got).all()
    assert np.abs(got[:, 0:2] - ref[:, 0:2]).max() <= 1e-4
    assert np.abs(got[:, 2:4] - ref[:, 2:4]).max() <= 1e-5
    assert (np.abs(got[:, 4:6] - ref[:, 4:6]) / ref[:, 4:6]).max() <= 1e-5
    refi = oracle.render_image(table_from_f32(r.gauss.cpu().numpy()), W, H, margin=1e-5)
    ok = ~refi["flag"]
    err = (r.img.cpu().double() - refi["img"]).abs().amax(0)
    assert float(err[ok].max()) <= 1e-5
    assert float(((~ok) & (err > 1e-5)).double().mean()) < 1e-4
    # 1x1 canvas
    cfg, curves, r1 = _setup(bs, 1, 1, arr, 7, 3, 5)
    img = r1.forward(curves)
    ref1 = oracle.render_image(table_from_f32(r1.gauss.cpu().numpy()), 1, 1)
    assert float((img.cpu().double() - ref1["img"]).abs().max()) <= 1e-5


def test_tile_with_more_than_1e4_gaussians(bs):
    """200 curves x 64 samples piled into one 16x16 tile."""
    W, H = 48, 48
    rng = np.random.default_rng(3)
    n = 200
    arr = synth.make_curves(4, W, H, n, 0, style="uniform").as_dict()
    arr["open_ctrl"] = (20 + rng.uniform(0, 8, (n, 10, 2))).astype(np.float32)
    arr["open_width"] = rng.uniform(0.3, 0.8, n).astype(np.float32)
    arr["open_opac"] = rng.uniform(0.01, 0.05, (n, 3)).astype(np.float32)   # keep T above 1e-4
    cfg, curves, r = _setup(bs, W, H, arr, 64, 3, 4)
    r.forward(curves)
    ranges = r.binning.ranges.cpu().numpy()
    assert (ranges[:, 1] - ranges[:, 0]).max() > 10000
    # the float32 transmittance after n factors carries a relative rounding
    # error that grows with n (about sqrt(n) u in practice, 2 n u at worst:
    # 1.5e-3 after 12,800 factors), so with lists this long the stop decision
    # is flagged at 1e-4 relative instead of 1e-5
    refi = oracle.render_image(table_from_f32(r.gauss.cpu().numpy()), W, H, margin=1e-5, margin_T=1e-4)
    ok = ~refi["flag"]
    err = (r.img.cpu().double() - refi["img"]).abs().amax(0)
    print(f"pile: list max {(ranges[:, 1] - ranges[:, 0]).max()}, err {float(err[ok].max()):.1e}, "
          f"flagged {float((~ok).double().mean()):.1e}")
    assert float(err[ok].max()) <= 1e-5
    assert float(((~ok) & (err > 1e-5)).double().mean()) < 1e-4


def test_sort_over_many_partitions_is_exact(bs):
    """More than three sort partitions of 4096 keys, keys spread over every
    digit of both passes: keys and ranges bit-exact against the oracle, on a
    fresh workspace and again on the reused one; the status word stays 0."""
    rng = np.random.default_rng(9)
    W, H, n = 256, 256, 3000
    rec = np.zeros((n, 12), dtype=np.float32)
    rec[:, 0] = rng.uniform(0, W, n)
    rec[:, 1] = rng.uniform(0, H, n)
    rec[:, 10:12] = rng.uniform(5, 30, (n, 2))
    keys, ranges, _ = oracle.tile_keys(rec, W, H, 16)
    assert keys.shape[0] > 3 * 4096
    gauss = torch.as_tensor(rec, device="cuda")
    canvas = bs.Canvas(W, H)
    b = bs.Binning(canvas, "cuda", pair_capacity=keys.shape[0] + 16)
    for _ in range(2):
        b.run(gauss)
        assert b.device_status() == 0
        assert np.array_equal(b.keys[:b.n_pairs].cpu().numpy().view(np.uint32), keys)
        assert np.array_equal(b.ranges.cpu().numpy().view(np.uint32), ranges)


def test_capacity_growth(bs):
    rng = np.random.default_rng(10)
    rec = np.zeros((500, 12), dtype=np.float32)
    rec[:, 0:2] = rng.uniform(0, 128, (500, 2))
    rec[:, 10:12] = 20.0
    gauss = torch.as_tensor(rec, device="cuda")
    b = bs.Binning(bs.Canvas(128, 128), "cuda", pair_capacity=16)
    b.run(gauss)
    keys, _, _ = oracle.tile_keys(rec, 128, 128, 16)
    assert b.n_pairs == keys.shape[0] and b.capacity >= keys.shape[0]
