"""Pins of oracle.bounds (the absolute-term scales of the float32 error bound
on the gradients) against brute force and closed forms, on the CPU."""

import numpy as np
import pytest
import torch

import oracle
from oracle.bounds import blend_abs, sample_abs_vjp
from oracle.curves import SampleCfg, gaussian_table
from oracle.pipeline import as_curves, sample_vjp
from oracle.raster import GRAD_KEYS, render_grads
from paper_2503_16424_gb300 import synth

F64 = torch.float64


def _case(seed=3, W=14, H=11, no=2, nc=1):
    arr = synth.make_curves(seed, W, H, no, nc, style="local").as_dict()
    cfg = SampleCfg(g_open=5, rows_closed=3, k_closed=4)
    _, first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], cfg)
    tab = {k: v.detach() for k, v in gaussian_table(as_curves(arr), cfg, first).items()}
    return arr, cfg, first, tab


def _pixels(W, H):
    ys, xs = torch.meshgrid(torch.arange(H, dtype=F64), torch.arange(W, dtype=F64), indexing="ij")
    return xs.reshape(-1), ys.reshape(-1)


def test_blend_abs_dominates_the_per_pixel_absolute_sum():
    """Brute force: the gradient of every pixel on its own (one autograd
    call per pixel), summed in absolute value, is at most blend_abs; the
    colour field has no inner sum, so there the two are equal."""
    W, H = 14, 11
    arr, cfg, first, tab = _case(W=W, H=H)
    xs, ys = _pixels(W, H)
    rng = np.random.default_rng(0)
    dC = torch.as_tensor(rng.normal(0, 1, (W * H, 3)))
    bg = (0.2, 0.1, 0.4)
    A = blend_abs(tab, xs, ys, dC, bg)
    brute = {k: torch.zeros_like(A[k]) for k in GRAD_KEYS}
    for p in range(W * H):
        g = render_grads(tab, xs[p:p + 1], ys[p:p + 1], dC[p:p + 1], bg)
        for k in GRAD_KEYS:
            brute[k] += g[k].abs()
    for k in GRAD_KEYS:
        assert torch.all(A[k] >= brute[k] * (1 - 1e-12) - 1e-300), k
    assert torch.allclose(A["col"], brute["col"], rtol=1e-12, atol=0)
    total = render_grads(tab, xs, ys, dC, bg)
    for k in GRAD_KEYS:          # and so the triangle inequality
        assert torch.all(A[k] >= total[k].abs() * (1 - 1e-12)), k
    assert float(A["mx"].max()) > 0 and float(A["isx"].max()) > 0


def test_blend_abs_is_exact_without_cancellation():
    """One Gaussian, no background, dL/dC > 0 at every pixel: every
    per-pixel term of isx, isy and o has one sign (dalpha/disx = -alpha a^2
    / isx, dalpha/do = alpha / o), so the bound equals |gradient|."""
    W, H = 9, 7
    tab = dict(mx=torch.tensor([4.3], dtype=F64), my=torch.tensor([3.1], dtype=F64),
               ux=torch.tensor([0.8], dtype=F64), uy=torch.tensor([0.6], dtype=F64),
               isx=torch.tensor([0.7], dtype=F64), isy=torch.tensor([0.45], dtype=F64),
               o=torch.tensor([0.6], dtype=F64), col=torch.tensor([[0.3, 0.5, 0.9]], dtype=F64))
    xs, ys = _pixels(W, H)
    dC = torch.as_tensor(np.random.default_rng(1).uniform(0.1, 1.0, (W * H, 3)))
    A = blend_abs(tab, xs, ys, dC)
    g = render_grads(tab, xs, ys, dC)
    for k in ("isx", "isy", "o", "col"):
        assert torch.allclose(A[k], g[k].abs(), rtol=1e-12, atol=0), k


def test_blend_abs_zero_where_nothing_blends():
    """o = 0 blends nothing: no term, a zero scale."""
    W, H = 6, 5
    arr, cfg, first, tab = _case(W=W, H=H)
    tab = dict(tab, o=torch.zeros_like(tab["o"]))
    xs, ys = _pixels(W, H)
    A = blend_abs(tab, xs, ys, torch.ones(W * H, 3, dtype=F64))
    for k in GRAD_KEYS:
        assert float(A[k].abs().max()) == 0.0, k


def test_sample_abs_vjp_equals_the_dense_jacobian():
    """Brute force: the full Jacobian of the table with respect to the curve
    parameters (torch.autograd.functional.jacobian), contracted in absolute
    value with the scales, equals sample_abs_vjp."""
    arr, cfg, first, tab = _case(seed=5, no=1, nc=1)
    cv = as_curves(arr)
    ng = tab["mx"].shape[0]
    rng = np.random.default_rng(2)
    scale = {k: torch.as_tensor(rng.uniform(0, 1, tuple(tab[k].shape))) for k in GRAD_KEYS}
    got = sample_abs_vjp(cv, cfg, scale, first)
    keys = list(cv)

    def flat(*vals):
        t = gaussian_table(dict(zip(keys, vals)), cfg, first)
        return torch.cat([t[k].reshape(ng, -1) for k in GRAD_KEYS], 1)

    jac = torch.autograd.functional.jacobian(flat, tuple(cv[k] for k in keys))
    s = torch.cat([scale[k].reshape(ng, -1) for k in GRAD_KEYS], 1)
    for k, J in zip(keys, jac):
        ref = (J.abs() * s[:, :, *([None] * cv[k].dim())]).sum((0, 1))
        assert torch.allclose(got[k], ref, rtol=1e-12, atol=1e-300), k


def test_sample_abs_vjp_dominates_the_vjp():
    arr, cfg, first, tab = _case(seed=6, no=3, nc=2)
    cv = as_curves(arr)
    rng = np.random.default_rng(4)
    dtab = {k: torch.as_tensor(rng.normal(0, 1, tuple(tab[k].shape))) for k in GRAD_KEYS}
    vjp = sample_vjp(cv, cfg, dtab, first)
    bound = sample_abs_vjp(cv, cfg, {k: v.abs() for k, v in dtab.items()}, first)
    for k in vjp:
        assert torch.all(bound[k] >= vjp[k].abs() * (1 - 1e-12)), k
