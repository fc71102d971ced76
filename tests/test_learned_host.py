"""Host-side helpers of the learned initialiser (no GPU): the circular
initialisation of Section 4.1 (one circle of radius 10 px per 32 x 32 cell,
the cell's mean target colour, opacity 0.8) and the cutting of a large
target into 256 x 256 patches whose proposals are put back in place."""

import numpy as np
import torch

from paper_2503_16424_gb300 import learned


def test_circle_points_lie_on_the_circle_from_angle_zero():
    P = learned.circle_points(np.array([40.0]), np.array([-7.0]), 10.0)[0]
    assert P.shape == (12, 2)
    assert np.allclose(np.hypot(P[:, 0] - 40.0, P[:, 1] + 7.0), 10.0)
    assert np.allclose(P[0], [50.0, -7.0])
    ang = np.arctan2(P[:, 1] + 7.0, P[:, 0] - 40.0) % (2 * np.pi)
    assert np.allclose(np.diff(ang[:7]), np.pi / 6)


def test_circle_init_centres_colours_and_opacity():
    rng = np.random.default_rng(0)
    target = rng.uniform(0, 1, (2, 3, 256, 256)).astype(np.float32)
    ctrl, color, opac = learned.circle_init(2, 256, target)
    assert ctrl.shape == (2 * 64, 12, 2) and color.shape == (128, 3) and opac.shape == (128,)
    centres = ctrl.mean(axis=1)
    for p in range(2):
        for cy in range(8):
            for cx in range(8):
                i = p * 64 + cy * 8 + cx
                assert np.allclose(centres[i], [(cx + 0.5) * 32, (cy + 0.5) * 32], atol=1e-4)
                cell = target[p, :, cy * 32:(cy + 1) * 32, cx * 32:(cx + 1) * 32]
                assert np.allclose(color[i], cell.mean(axis=(1, 2)), atol=1e-6)
    assert np.all(opac == np.float32(learned.OPACITY))
    _, grey, _ = learned.circle_init(1, 256, None)
    assert np.all(grey == 0.5)


def test_patches_and_proposals_go_back_in_place():
    rng = np.random.default_rng(1)
    H, W = 512, 768
    target = torch.as_tensor(rng.uniform(0, 1, (3, H, W)).astype(np.float32))
    patches = learned.image_patches(target)
    assert patches.shape == (6, 3, 256, 256)
    for i in range(6):
        py, px = divmod(i, 3)
        assert torch.equal(patches[i], target[:, py * 256:(py + 1) * 256, px * 256:(px + 1) * 256])
    # the circles of the whole image: every 32 x 32 cell once, at its centre,
    # with its mean colour
    curves = learned.initial_curves(target)
    centres = curves.closed_ctrl.numpy().mean(axis=1)
    colors = curves.closed_color.numpy()
    assert centres.shape == (H // 32 * W // 32, 2)
    seen = set()
    for c, col in zip(centres, colors):
        gx, gy = int(c[0] // 32), int(c[1] // 32)
        assert np.allclose(c, [(gx + 0.5) * 32, (gy + 0.5) * 32], atol=1e-3)
        cell = target[:, gy * 32:(gy + 1) * 32, gx * 32:(gx + 1) * 32].numpy()
        assert np.allclose(col, cell.mean(axis=(1, 2)), atol=1e-6)
        seen.add((gx, gy))
    assert len(seen) == centres.shape[0]
