"""Pins of the oracle's gradients: autograd of the brute-force definition
against central finite differences in fp64 (8x8 and 12x10 images, few
curves, parameters away from the threshold decisions)."""

import numpy as np
import pytest
import torch

import oracle
from oracle.curves import SampleCfg
from oracle.pipeline import CURVE_KEYS, as_curves, loss_only, step
from paper_2503_16424_gb300 import synth


def _case(seed, W, H, n_open, n_closed, cfg):
    c = synth.make_curves(seed, W, H, n_open, n_closed, style="uniform",
                          width_range=(1.5, 3.0), opac_range=(0.3, 0.85))
    curves = as_curves(c.as_dict())
    target = torch.as_tensor(np.random.default_rng(seed + 100).uniform(0, 1, (3, H, W)))
    return curves, target


@pytest.mark.parametrize("seed,W,H,n_open,n_closed", [(0, 8, 8, 2, 0), (1, 8, 8, 0, 1),
                                                      (2, 12, 10, 2, 1)])
def test_autograd_equals_central_fd(seed, W, H, n_open, n_closed):
    cfg = SampleCfg(g_open=6, rows_closed=3, k_closed=4, eps=0.3)
    curves, target = _case(seed, W, H, n_open, n_closed, cfg)
    bg = (0.2, 0.1, 0.4)
    res = step(curves, cfg, W, H, target, bg)
    # no pixel close to a threshold decision, so the loss is smooth here
    from oracle.raster import render_pixels
    ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64),
                            indexing="ij")
    fl = render_pixels(res["table"], xs.reshape(-1), ys.reshape(-1), bg, margin=1e-4)["flag"]
    assert not bool(fl.any())
    checked = 0
    for key in CURVE_KEYS:
        base = curves[key]
        g_auto = res["dcurves"][key].reshape(-1)
        flat = base.reshape(-1)
        gmax = float(g_auto.abs().max()) if g_auto.numel() else 0.0
        for i in range(flat.numel()):
            h = 1e-6 * max(1.0, abs(float(flat[i])))
            plus = {k: v.clone() for k, v in curves.items()}
            minus = {k: v.clone() for k, v in curves.items()}
            plus[key].view(-1)[i] += h
            minus[key].view(-1)[i] -= h
            fd = (loss_only(plus, cfg, W, H, target, bg) - loss_only(minus, cfg, W, H, target, bg)) / (2 * h)
            err = abs(fd - float(g_auto[i]))
            # FD rounding error is about eps * L / h; allow 50x that
            fd_round = 50 * 2.2e-16 * res["loss"] / h
            assert err <= 1e-5 * max(abs(fd), 1e-3 * gmax) + fd_round, (key, i, fd, float(g_auto[i]))
            checked += 1
    assert checked > 20


def test_per_gaussian_grads_fd():
    """dL/d(table) of render_grads against FD in the table entries."""
    cfg = SampleCfg(g_open=5, rows_closed=3, k_closed=4)
    curves, target = _case(3, 8, 8, 2, 1, cfg)
    res = step(curves, cfg, 8, 8, target)
    tab = {k: v.detach().clone() for k, v in res["table"].items() if k in
           ("mx", "my", "ux", "uy", "isx", "isy", "o", "col")}

    def loss_of(t):
        img = oracle.render_image(t, 8, 8)["img"]
        return float(oracle.l2_loss(img, target)[0])

    rng = np.random.default_rng(0)
    for key in ("mx", "my", "ux", "uy", "isx", "isy", "o", "col"):
        g = res["dtable"][key].reshape(-1)
        for i in rng.choice(g.numel(), size=min(6, g.numel()), replace=False):
            h = 1e-6 * max(1.0, abs(float(tab[key].reshape(-1)[i])))
            tp = {k: v.clone() for k, v in tab.items()}
            tm = {k: v.clone() for k, v in tab.items()}
            tp[key].view(-1)[i] += h
            tm[key].view(-1)[i] -= h
            fd = (loss_of(tp) - loss_of(tm)) / (2 * h)
            fd_round = 50 * 2.2e-16 * res["loss"] / h
            assert abs(fd - float(g[i])) <= 1e-5 * max(abs(fd), 1e-3 * float(g.abs().max())) + fd_round


def test_l2_loss_gradient():
    rng = np.random.default_rng(1)
    a, b = rng.uniform(0, 1, (3, 4, 5)), rng.uniform(0, 1, (3, 4, 5))
    L, g = oracle.l2_loss(a, b)
    assert abs(float(L) - ((a - b) ** 2).sum() / 60) < 1e-15
    i = (1, 2, 3)
    h = 1e-7
    ap = a.copy(); ap[i] += h
    am = a.copy(); am[i] -= h
    fd = (float(oracle.l2_loss(ap, b)[0]) - float(oracle.l2_loss(am, b)[0])) / (2 * h)
    assert abs(fd - float(g[i])) < 1e-8


def _conic_blend_loss(curves, cfg, W, H, target, bg):
    """The loss through a blend written in the conic form of Eq. 11-12,
    alpha = min(0.99, o exp(-0.5 d^T Sigma^-1 d)) with Sigma^-1 from
    torch.linalg.inv, walked Gaussian by Gaussian in draw order with the
    three thresholds (skip below 1/255, stop before T < 1e-4): no use of the
    eigen-frame fields of the table."""
    tab = oracle.gaussian_table(curves, cfg)
    P = torch.linalg.inv(tab["Sigma"])
    ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64),
                            indexing="ij")
    px, py = xs.reshape(-1) + 0.5, ys.reshape(-1) + 0.5
    T = torch.ones_like(px)
    C = torch.zeros(px.shape[0], 3, dtype=torch.float64)
    alive = torch.ones_like(px, dtype=torch.bool)
    for i in range(tab["mx"].shape[0]):
        dx, dy = px - tab["mx"][i], py - tab["my"][i]
        q = P[i, 0, 0] * dx * dx + (P[i, 0, 1] + P[i, 1, 0]) * dx * dy + P[i, 1, 1] * dy * dy
        a = torch.clamp(tab["o"][i] * torch.exp(-0.5 * q), max=0.99)
        Tn = T * (1.0 - a)
        use = alive & (a >= 1.0 / 255.0) & (Tn >= 1e-4)
        alive = alive & ~((a >= 1.0 / 255.0) & (Tn < 1e-4))
        w = torch.where(use, a * T, torch.zeros_like(a))
        C = C + w[:, None] * tab["col"][i][None, :]
        T = torch.where(use, Tn, T)
    img = (C + T[:, None] * torch.as_tensor(bg, dtype=torch.float64)[None, :]).T.reshape(3, H, W)
    return ((img - target) ** 2).mean()


@pytest.mark.parametrize("seed,W,H,n_open,n_closed", [(3, 10, 9, 2, 1), (4, 12, 8, 1, 2)])
def test_curve_gradients_match_a_conic_form_blend(seed, W, H, n_open, n_closed):
    """The oracle stores Gaussians in the eigen-frame (R, S^-1) and takes its
    table gradients there; the curve gradients must equal those of the
    conic form of Eq. 11-12 through autograd, which shares none of that
    parameterisation (the same thresholds, no pixel near one)."""
    cfg = SampleCfg(g_open=6, rows_closed=3, k_closed=4, eps=0.3)
    curves, target = _case(seed, W, H, n_open, n_closed, cfg)
    bg = (0.2, 0.1, 0.4)
    res = step(curves, cfg, W, H, target, bg)
    assert not bool(res["flag"].any())
    leaves = as_curves({k: v.detach().numpy() for k, v in curves.items()}, requires_grad=True)
    L = _conic_blend_loss(leaves, cfg, W, H, target, bg)
    assert abs(float(L.detach()) - res["loss"]) <= 1e-12 * abs(res["loss"])
    gs = torch.autograd.grad(L, [leaves[k] for k in CURVE_KEYS], allow_unused=True)
    for k, g in zip(CURVE_KEYS, gs):
        ref = res["dcurves"][k]
        g = torch.zeros_like(ref) if g is None else g
        scale = float(ref.abs().max()) if ref.numel() else 0.0
        if scale == 0.0:
            assert float(g.abs().max()) == 0.0 if g.numel() else True, k
            continue
        assert float((g - ref).abs().max()) <= 1e-9 * scale, k
    assert float(res["dcurves"]["open_ctrl"].abs().max()) > 0.0


def test_colour_gradient_is_the_sum_of_alpha_t():
    """With dL/dC = 1 in every channel, dL/dc_i = sum over pixels of
    alpha_i T_i (Eq. 9 is linear in the colours), written out from the
    forward's alphas in draw order."""
    cfg = SampleCfg(g_open=6, rows_closed=3, k_closed=4, eps=0.3)
    curves, _ = _case(7, 10, 9, 2, 1, cfg)
    with torch.no_grad():
        tab = oracle.gaussian_table({k: v.detach() for k, v in curves.items()}, cfg)
    ys, xs = torch.meshgrid(torch.arange(9, dtype=torch.float64), torch.arange(10, dtype=torch.float64), indexing="ij")
    xs, ys = xs.reshape(-1), ys.reshape(-1)
    g = oracle.render_grads(tab, xs, ys, torch.ones(xs.shape[0], 3, dtype=torch.float64))
    # alpha_i T_i per pixel, the walk written out with the three thresholds
    from oracle.raster import ALPHA_MAX, ALPHA_MIN, T_MIN
    w = torch.zeros(xs.shape[0], tab["mx"].shape[0], dtype=torch.float64)
    for p in range(xs.shape[0]):
        T = 1.0
        for i in range(tab["mx"].shape[0]):
            dx, dy = float(xs[p]) + 0.5 - float(tab["mx"][i]), float(ys[p]) + 0.5 - float(tab["my"][i])
            a1 = float(tab["isx"][i]) * (float(tab["ux"][i]) * dx + float(tab["uy"][i]) * dy)
            a2 = float(tab["isy"][i]) * (-float(tab["uy"][i]) * dx + float(tab["ux"][i]) * dy)
            a = min(ALPHA_MAX, float(tab["o"][i]) * np.exp(-0.5 * (a1 * a1 + a2 * a2)))
            if a < ALPHA_MIN:
                continue
            if T * (1 - a) < T_MIN:
                break
            w[p, i] = a * T
            T *= 1 - a
    exp = w.sum(0)
    assert float(exp.max()) > 0.1
    for ch in range(3):
        assert torch.allclose(g["col"][:, ch], exp, atol=1e-12)


def test_curve_gradients_rotate_with_the_scene():
    """Rotating the curves and the target by 90 degrees rotates the image,
    so the control-point gradients rotate with it: g'(x, y) = (g_y, -g_x)
    at the rotated points (x, y) -> (y, W - x); the other gradients are
    unchanged.  Catches a transposed or sign-flipped conic in the backward."""
    cfg = SampleCfg(g_open=6, rows_closed=3, k_closed=4, eps=0.3)
    W = 10
    curves, target = _case(8, W, W, 2, 1, cfg)
    rot = dict(curves)
    for k in ("open_ctrl", "closed_ctrl"):
        P = curves[k].detach()
        rot[k] = torch.stack([P[..., 1], W - P[..., 0]], -1)
    rot = as_curves({k: v.detach().numpy() for k, v in rot.items()})
    # image pixel (x, y) moves to (y, W - 1 - x): rotate the target alike
    target_r = torch.rot90(target, k=1, dims=(1, 2))
    bg = (0.2, 0.1, 0.4)
    a = step(curves, cfg, W, W, target, bg)
    b = step(rot, cfg, W, W, target_r, bg)
    assert abs(a["loss"] - b["loss"]) < 1e-12
    for k in ("open_ctrl", "closed_ctrl"):
        ga, gb = a["dcurves"][k], b["dcurves"][k]
        assert torch.allclose(gb[..., 0], ga[..., 1], atol=1e-10)
        assert torch.allclose(gb[..., 1], -ga[..., 0], atol=1e-10)
    for k in ("open_width", "open_color", "open_opac", "closed_color", "closed_opac"):
        assert torch.allclose(a["dcurves"][k], b["dcurves"][k], atol=1e-10), k
