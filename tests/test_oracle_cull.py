"""Pins of oracle/cull.c (the multi-core, box-culled fp64 blend and its
hand-derived backward) against the brute-force blend of raster.py (every
Gaussian at every pixel) and its autograd gradient, on the CPU."""

import numpy as np
import pytest
import torch

import oracle
from oracle import cull
from oracle.curves import SampleCfg
from oracle.pipeline import as_curves
from paper_2503_16424_gb300 import synth


def _case(seed, W, H, no, nc, g=9, rows=4, kc=6):
    arr = synth.make_curves(seed, W, H, no, nc, style="local").as_dict()
    cfg = SampleCfg(g_open=g, rows_closed=rows, k_closed=kc)
    _, first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], cfg)
    with torch.no_grad():
        return {k: v.detach() for k, v in oracle.gaussian_table(as_curves(arr), cfg, first).items()}


@pytest.mark.parametrize("seed,W,H,no,nc,bg", [(1, 37, 29, 5, 3, (0.2, 0.3, 0.1)), (2, 64, 48, 10, 6, (0.0, 0.0, 0.0)),
                                              (3, 1, 23, 2, 2, (0.5, 0.5, 0.5))])
def test_culled_blend_equals_the_brute_force_blend(seed, W, H, no, nc, bg):
    tab = _case(seed, W, H, no, nc)
    img, T, used = cull.forward(tab, W, H, bg)
    ref = oracle.render_image(tab, W, H, bg=bg)
    assert np.abs(img - ref["img"].numpy()).max() <= 1e-12
    assert np.abs(T - ref["T"].numpy()).max() <= 1e-12
    # the walk length: up to the last blended Gaussian (0 for none)
    assert np.array_equal(used > 0, ref["last"].numpy() >= 0)


@pytest.mark.parametrize("seed,W,H,no,nc,bg", [(4, 40, 30, 6, 3, (0.1, 0.2, 0.3)), (5, 33, 51, 8, 4, (0.0, 0.0, 0.0))])
def test_hand_derived_backward_equals_autograd(seed, W, H, no, nc, bg):
    tab = _case(seed, W, H, no, nc)
    rng = np.random.default_rng(seed)
    dimg = rng.normal(0, 1, (3, H, W))
    img, T, used = cull.forward(tab, W, H, bg)
    got = cull.backward(tab, W, H, dimg, T, used, bg)
    ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64),
                            indexing="ij")
    dC = torch.as_tensor(dimg).permute(1, 2, 0).reshape(-1, 3)
    ref = oracle.render_grads(tab, xs.reshape(-1), ys.reshape(-1), dC, bg=bg)
    for k in ref:
        r, g = ref[k].reshape(-1), got[k].reshape(-1)
        scale = float(r.abs().max())
        assert float((g - r).abs().max()) <= 1e-10 * scale + 1e-300, k
    assert float(ref["mx"].abs().max()) > 0


def test_empty_table_and_invisible_gaussians():
    tab = _case(6, 20, 20, 3, 1)
    tab = dict(tab, o=torch.zeros_like(tab["o"]), ext_x=-torch.ones_like(tab["ext_x"]))
    img, T, used = cull.forward(tab, 20, 20, (0.3, 0.2, 0.1))
    assert np.allclose(img, np.array([0.3, 0.2, 0.1])[:, None, None]) and np.all(T == 1) and np.all(used == 0)
    g = cull.backward(tab, 20, 20, np.ones((3, 20, 20)), T, used, (0.3, 0.2, 0.1))
    assert all(float(v.abs().max()) == 0.0 for v in g.values())
    assert cull.threads() >= 1
