"""Host-side set-up of the batched optimiser (no GPU): the per-curve
control-point step sizes follow each curve's image (Section 4.1's 2e-4 in
[-1, 1] coordinates is 2e-4 x half the longer side in pixels), and the Adam
groups carry the rates and boxes of AdamCfg."""

import numpy as np
import pytest
import torch

from paper_2503_16424_gb300 import bs
from paper_2503_16424_gb300.batch import AdamCfg, CurveAdam, _curve_scales
from paper_2503_16424_gb300 import synth


def _images():
    cfg = bs.SampleCfg()
    return [bs.BatchImage(300, 200, 2, 1, cfg), bs.BatchImage(64, 640, 0, 3, cfg), bs.BatchImage(50, 50, 4, 0, cfg)]


def test_control_point_scales_follow_each_curves_image():
    images = _images()
    s_open = _curve_scales(images, "open", "cpu").numpy()
    s_closed = _curve_scales(images, "closed", "cpu").numpy()
    assert np.array_equal(s_open, [150.0, 150.0, 25.0, 25.0, 25.0, 25.0])
    assert np.array_equal(s_closed, [150.0, 320.0, 320.0, 320.0])


def test_adam_groups_carry_the_rates_and_boxes():
    images = _images()
    n_open, n_closed = 6, 4
    arrs = synth.make_curves(5, 300, 300, n_open, n_closed, style="local").as_dict()
    curves = bs.CurveSet.from_arrays(arrs, device="cpu")
    cfg = AdamCfg()
    adam = CurveAdam(curves, curves.zeros_like(), images, cfg, "cpu")
    by_param = {id(g.param): g for g in adam.groups}
    want = {
        "open_ctrl": (cfg.lr_ctrl, 20), "closed_ctrl": (cfg.lr_ctrl, 24),
        "open_width": (cfg.lr_width, 1), "open_color": (cfg.lr_color, 1), "open_opac": (cfg.lr_opac, 1),
        "closed_color": (cfg.lr_color, 1), "closed_opac": (cfg.lr_opac, 1),
    }
    for field, (lr, row_len) in want.items():
        g = by_param[id(getattr(curves, field))]
        assert g.lr == pytest.approx(lr) and g.row_len == row_len
        assert g.param.numel() == g.grad.numel() == g.m.numel() == g.v.numel()
        if field.endswith("ctrl"):
            assert g.row_scale is not None and g.row_scale.numel() * row_len == g.param.numel()
            assert (g.lo, g.hi) == (-3.0e38, 3.0e38)
        else:
            assert g.row_scale is None
    assert by_param[id(curves.open_width)].lo == pytest.approx(cfg.width_min)
    for field in ("open_color", "open_opac", "closed_color", "closed_opac"):
        g = by_param[id(getattr(curves, field))]
        assert (g.lo, g.hi) == (0.0, 1.0)
    # no gradient-fill fields: no groups for them
    assert len(adam.groups) == len(want)
    # the step counter starts at 0 (bias corrections use t = counter + 1)
    assert int(adam.t.item()) == 0
    assert adam.t.dtype == torch.int32
