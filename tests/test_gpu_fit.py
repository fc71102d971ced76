"""Optimisation runs through the library (paper_2503_16424_gb300.fit): the
captured step with Adam and the periodic pruning and densification pass of
Section 3.5 (Algorithm 1) on a reduced schedule of the 2048 x 2048 run
(256 x 256, 120 steps, a pass every 30).

Bars: the PSNR rises; every pass's changed mask and counts are bit-exact
against the oracle on the same curves, image and target, with the edited
values within 2 float32 ulps (the bars of tests/test_gpu_prune.py); the
loss of the first step after each pass equals the oracle's loss of the new
curves within the error the 1e-5 pixel bar allows, 2e-5 mean|C - I| +
1e-10 (|d(C - I)^2| <= 2 |C - I| |dC| + dC^2)."""

import numpy as np
import pytest
import torch

import oracle
from oracle.curves import SampleCfg as OCfg
from oracle.pipeline import as_curves
from oracle.prune_densify import PDCfg as OPD, prune_densify as oracle_pd
from paper_2503_16424_gb300 import synth
from tests.test_gpu_prune import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def test_fit_with_passes_rises_and_every_pass_matches_the_oracle(bs):
    from paper_2503_16424_gb300.fit import FitCfg, fit
    from paper_2503_16424_gb300.raster import Rasterizer
    W = H = 256
    iters, every = 120, 30
    arr = synth.make_curves(42, W, H, 48, 24, style="local").as_dict()
    tgt_np = synth.procedural_target(43, W, H, 12)
    target = torch.as_tensor(tgt_np, device="cuda")
    cfg = bs.SampleCfg(g_open=16, rows_closed=4, k_closed=8)
    ocfg = OCfg(g_open=16, rows_closed=4, k_closed=8)
    curves = bs.CurveSet.from_arrays(arr, device="cuda")
    r = Rasterizer(bs.Canvas(W, H, 16), cfg, curves.n_open, curves.n_closed, pair_capacity=1 << 16)
    passes = []

    def hook(step, before, img, changed, stats, after):
        passes.append((step, before, img, changed, stats, after))

    res = fit(r, curves, target, FitCfg(iters=iters, prune_every=every), pass_hook=hook)
    loss = res["loss"]
    psnr = -10.0 * np.log10(loss)
    print(f"fit: psnr {psnr[0]:.2f} -> {psnr[-1]:.2f} dB, passes {res['passes']}")
    assert np.all(np.isfinite(loss))
    assert psnr[-10:].mean() > psnr[:10].mean() + 1.0
    assert [p[0] for p in passes] == [30, 60, 90]
    for step, before, img, changed, stats, after in passes:
        o_out, o_changed, info = oracle_pd(before, img, tgt_np, OPD(step=step, t_end=iters), ocfg)
        compare(before, bs.CurveSet.from_arrays(after), changed.astype(bool), stats, o_out, o_changed, info)
        # the first step after the pass renders the new curves
        with torch.no_grad():
            cv = as_curves(after)
            _, first = oracle.draw_order(after["open_ctrl"], after["open_width"], after["closed_ctrl"], ocfg)
            tab = oracle.gaussian_table(cv, ocfg, first)
            img_o = oracle.render_image(tab, W, H)["img"]
        d = img_o - torch.as_tensor(tgt_np, dtype=torch.float64)
        l_ref = float((d * d).mean())
        allow = 2e-5 * float(d.abs().mean()) + 1e-10
        print(f"  pass at {step}: {stats}; next loss {loss[step]:.8f} vs oracle {l_ref:.8f}")
        assert abs(float(loss[step]) - l_ref) <= allow, (step, float(loss[step]), l_ref)
    assert sum(p[4]["pruned"] for p in passes) > 0


def test_fit_without_passes_matches_eager_steps(bs):
    """The captured step with Adam replays the eager step with Adam: the
    same loss curve up to the order of the float atomics."""
    from paper_2503_16424_gb300.batch import AdamCfg, CurveAdam
    from paper_2503_16424_gb300.fit import FitCfg, fit
    from paper_2503_16424_gb300.raster import Rasterizer
    W, H = 120, 96
    arr = synth.make_curves(44, W, H, 12, 6, style="local").as_dict()
    target = torch.as_tensor(synth.procedural_target(45, W, H, 8), device="cuda")
    cfg = bs.SampleCfg(g_open=12, rows_closed=4, k_closed=6)
    c1 = bs.CurveSet.from_arrays(arr, device="cuda")
    r1 = Rasterizer(bs.Canvas(W, H, 16), cfg, c1.n_open, c1.n_closed, pair_capacity=4096)
    res = fit(r1, c1, target, FitCfg(iters=12))
    c2 = bs.CurveSet.from_arrays(arr, device="cuda")
    r2 = Rasterizer(bs.Canvas(W, H, 16), cfg, c2.n_open, c2.n_closed, pair_capacity=4096)
    g2 = c2.zeros_like()
    adam = CurveAdam(c2, g2, [bs.BatchImage(W, H, c2.n_open, c2.n_closed, cfg)], AdamCfg(), "cuda")
    eager = []
    for _ in range(12):
        loss, _ = r2.step(c2, target, g2)
        eager.append(float(loss))
        adam.step()
    assert np.allclose(res["loss"], eager, rtol=1e-4, atol=0)
    for k in bs.CURVE_FIELDS:
        a, b = getattr(c1, k), getattr(c2, k)
        assert float((a - b).abs().max()) <= 1e-3 * max(1.0, float(b.abs().max())), k
