"""Host-side helpers of the learned initialiser (no GPU): the baseline
initialisation (per 32 x 32 cell the circle of Section 4.1, radius 10 px, and
a horizontal stroke through the centre, 20 px long and 2 px wide, both in the
cell's mean target colour at opacity 0.8), the head bias that proposes it,
and the cutting of a large target into 256 x 256 patches whose proposals are
put back in place."""

import numpy as np
import torch

from oracle import net as onet
from paper_2503_16424_gb300 import learned


def test_circle_points_lie_on_the_circle_from_angle_zero():
    P = learned.circle_points(np.array([40.0]), np.array([-7.0]), 10.0)[0]
    assert P.shape == (12, 2)
    assert np.allclose(np.hypot(P[:, 0] - 40.0, P[:, 1] + 7.0), 10.0)
    assert np.allclose(P[0], [50.0, -7.0])
    ang = np.arctan2(P[:, 1] + 7.0, P[:, 0] - 40.0) % (2 * np.pi)
    assert np.allclose(np.diff(ang[:7]), np.pi / 6)


def test_stroke_points_are_evenly_spaced_on_the_horizontal_segment():
    Q = learned.stroke_points(np.array([40.0]), np.array([-7.0]), 9.0)[0]
    assert Q.shape == (10, 2)
    assert np.allclose(Q[:, 1], -7.0)
    assert np.allclose(Q[:, 0], 40.0 + np.arange(-9.0, 10.0, 2.0))


def test_baseline_init_centres_colours_widths_and_opacity():
    rng = np.random.default_rng(0)
    target = rng.uniform(0, 1, (2, 3, 256, 256)).astype(np.float32)
    b = learned.baseline_init(2, 256, target)
    shapes = dict(ctrl=(128, 12, 2), color=(128, 3), opac=(128,), open_ctrl=(128, 10, 2), open_width=(128,),
                  open_color=(128, 3), open_opac=(128, 3))
    assert {k: v.shape for k, v in b.items()} == shapes
    for kind in ("ctrl", "open_ctrl"):
        centres = b[kind].mean(axis=1)
        for p in range(2):
            for cy in range(8):
                for cx in range(8):
                    i = p * 64 + cy * 8 + cx
                    assert np.allclose(centres[i], [(cx + 0.5) * 32, (cy + 0.5) * 32], atol=1e-4)
                    cell = target[p, :, cy * 32:(cy + 1) * 32, cx * 32:(cx + 1) * 32]
                    assert np.allclose(b["color"][i], cell.mean(axis=(1, 2)), atol=1e-6)
    assert np.array_equal(b["open_color"], b["color"])
    assert np.all(b["opac"] == np.float32(learned.OPACITY)) and np.all(b["open_opac"] == np.float32(learned.OPACITY))
    assert np.all(b["open_width"] == np.float32(learned.STROKE_WIDTH))
    assert np.allclose(np.ptp(b["open_ctrl"][:, :, 0], axis=1), 2 * learned.STROKE_HALF)
    grey = learned.baseline_init(1, 256, None)
    assert np.all(grey["color"] == 0.5) and np.all(grey["open_color"] == 0.5)


def test_head_bias_proposes_the_baseline_curves():
    """With a zero feature map the head's output is its bias; the oracle's
    mapping of that bias gives the baseline curves with colour 0.5."""
    head_w = learned.initial_weights(0)[5]
    bias = torch.as_tensor(head_w[-64:], dtype=torch.float64)
    side = 64
    p = onet.head_curves(bias.expand(1, (side // 32) ** 2, 64), side)
    b = learned.baseline_init(1, side, None)
    for k in onet.CURVE_KEYS:
        assert np.allclose(p[k][0].numpy(), b[k], atol=1e-5), k


def test_patches_and_proposals_go_back_in_place():
    rng = np.random.default_rng(1)
    H, W = 512, 768
    target = torch.as_tensor(rng.uniform(0, 1, (3, H, W)).astype(np.float32))
    patches = learned.image_patches(target)
    assert patches.shape == (6, 3, 256, 256)
    for i in range(6):
        py, px = divmod(i, 3)
        assert torch.equal(patches[i], target[:, py * 256:(py + 1) * 256, px * 256:(px + 1) * 256])
    # the baseline curves of the whole image: every 32 x 32 cell once per
    # kind, at its centre, with its mean colour
    curves = learned.initial_curves(target)
    for ctrl, color in ((curves.closed_ctrl, curves.closed_color), (curves.open_ctrl, curves.open_color)):
        centres = ctrl.numpy().mean(axis=1)
        assert centres.shape == (H // 32 * W // 32, 2)
        seen = set()
        for c, col in zip(centres, color.numpy()):
            gx, gy = int(c[0] // 32), int(c[1] // 32)
            assert np.allclose(c, [(gx + 0.5) * 32, (gy + 0.5) * 32], atol=1e-3)
            cell = target[:, gy * 32:(gy + 1) * 32, gx * 32:(gx + 1) * 32].numpy()
            assert np.allclose(col, cell.mean(axis=(1, 2)), atol=1e-6)
            seen.add((gx, gy))
        assert len(seen) == centres.shape[0]
