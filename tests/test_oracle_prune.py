"""Pins of the oracle's pruning and densification (Section 3.5, Algorithm 1,
Appendix B): closed-form thresholds, constructed curves whose fate is known,
brute-force pair tests and flood fills, and geometric identities of the new
curves."""

from collections import deque

import numpy as np
import pytest
import torch

from oracle.curves import SampleCfg, area_keys_f32, bezier
from oracle.prune_densify import (
    PDCfg, tau_op, prune_flags, split_flags, subdivide_thirds, error_regions,
    region_stats, circle_points, prune_densify, curve_boxes_f32,
)

SCFG = SampleCfg(g_open=8, rows_closed=3, k_closed=4)
F = np.float32


def rect_closed(x0, y0, x1, y1):
    """12 control points around an axis-aligned rectangle (3 per side)."""
    pts = []
    for (ax, ay), (bx, by) in [((x0, y0), (x1, y0)), ((x1, y0), (x1, y1)),
                               ((x1, y1), (x0, y1)), ((x0, y1), (x0, y0))]:
        for s in range(3):
            t = s / 3.0
            pts.append((ax + t * (bx - ax), ay + t * (by - ay)))
    return np.array(pts)


def line_open(x0, y0, x1, y1):
    t = np.arange(10) / 9.0
    return np.stack([x0 + t * (x1 - x0), y0 + t * (y1 - y0)], 1)


def curve_set(opens=(), closeds=()):
    """opens: (ctrl [10,2], width, colour, opac[3]); closeds: (ctrl, colour, opac)."""
    oc = np.array([o[0] for o in opens], F).reshape(-1, 10, 2)
    return dict(
        open_ctrl=oc,
        open_width=np.array([o[1] for o in opens], F).reshape(-1),
        open_color=np.array([o[2] for o in opens], F).reshape(-1, 3),
        open_opac=np.array([o[3] for o in opens], F).reshape(-1, 3),
        closed_ctrl=np.array([c[0] for c in closeds], F).reshape(-1, 12, 2),
        closed_color=np.array([c[1] for c in closeds], F).reshape(-1, 3),
        closed_opac=np.array([c[2] for c in closeds], F).reshape(-1),
    )


def test_tau_op_schedule():
    assert tau_op(PDCfg(step=0, t_end=1000)) == F(0.2)
    assert abs(float(tau_op(PDCfg(step=500, t_end=1000))) - 0.11) < 1e-7
    assert tau_op(PDCfg(step=1000, t_end=1000)) == F(0.02)
    assert tau_op(PDCfg(step=5000, t_end=1000)) == F(0.02)


def test_low_opacity_rule():
    big = rect_closed(0, 0, 20, 20)
    arr = curve_set(
        opens=[(line_open(0, 0, 30, 0), 3.0, (1, 0, 0), (0.1, 0.1, 0.3)),    # mean 1/6
               (line_open(0, 5, 30, 5), 3.0, (0, 1, 0), (0.2, 0.2, 0.23))],  # mean 0.21
        closeds=[(big + 40, (0, 0, 1), 0.15), (big + 80, (1, 1, 0), 0.25)])
    p0, c0 = prune_flags(arr, PDCfg(step=0, t_end=100), SCFG)
    assert c0["low_op"].tolist() == [True, False, True, False]
    p1, c1 = prune_flags(arr, PDCfg(step=50, t_end=100), SCFG)      # tau 0.11
    assert c1["low_op"].tolist() == [False, False, False, False]
    assert p0.tolist() == [True, False, True, False] and not p1.any()


def test_small_area_rule():
    arr = curve_set(
        opens=[(line_open(0, 0, 1, 0), 3.0, (1, 0, 0), (1, 1, 1)),      # key 3
               (line_open(0, 9, 2, 9), 3.0, (0, 1, 0), (1, 1, 1))],     # key 6
        closeds=[(rect_closed(10, 10, 11.9, 11.9), (0, 0, 1), 1.0),    # 3.61
                 (rect_closed(20, 20, 22.1, 22.1), (1, 1, 0), 1.0)])   # 4.41
    keys = area_keys_f32(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"])
    np.testing.assert_allclose(keys, [3.0, 6.0, 3.61, 4.41], rtol=1e-5)
    _, crit = prune_flags(arr, PDCfg(), SCFG)
    assert crit["small"].tolist() == [True, False, True, False]


@pytest.mark.parametrize("dcol,expect", [(0.029, True), (0.031, False)])
def test_overlap_colour_threshold(dcol, expect):
    sq = rect_closed(0, 0, 10, 10)
    arr = curve_set(closeds=[(sq, (0.5, 0.5, 0.5), 1.0), (sq, (0.5 + dcol, 0.5, 0.5), 1.0)])
    _, crit = prune_flags(arr, PDCfg(), SCFG)
    # equal areas: curve 0 is drawn in front, so only curve 1 can go
    assert crit["overlap"].tolist() == [False, expect]


@pytest.mark.parametrize("h,iou,expect", [(9.5, 0.95, True), (8.5, 0.85, False)])
def test_overlap_iou_threshold_and_direction(h, iou, expect):
    big = rect_closed(0, 0, 10, 10)
    small = rect_closed(0, 0, 10, h)      # smaller area: drawn in front of `big`
    arr = curve_set(closeds=[(big, (0.2, 0.3, 0.4), 1.0), (small, (0.2, 0.3, 0.4), 1.0)])
    boxes = curve_boxes_f32(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"])
    np.testing.assert_allclose(boxes, [[0, 0, 10, 10], [0, 0, 10, h]])
    _, crit = prune_flags(arr, PDCfg(), SCFG)
    assert crit["overlap"].tolist() == [expect, False]
    assert abs(h * 10 / 100 - iou) < 1e-12


def test_open_box_includes_half_width():
    arr = curve_set(opens=[(line_open(5, 7, 25, 7), 4.0, (0, 0, 0), (1, 1, 1))])
    np.testing.assert_array_equal(curve_boxes_f32(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"]),
                                  [[3, 5, 27, 9]])


def _brute_overlap(arr, cfg):
    """Scalar float32 pair loop written from the rule, independent of the
    vectorised oracle: later curve of a (similar colour, IoU > min) pair."""
    f = np.float32
    oc = arr["open_ctrl"].astype(f)
    boxes, cols = [], []
    for i in range(oc.shape[0]):
        hw = f(arr["open_width"][i]) * f(0.5)
        xs, ys = oc[i, :, 0], oc[i, :, 1]
        boxes.append((f(xs.min() - hw), f(ys.min() - hw), f(xs.max() + hw), f(ys.max() + hw)))
        cols.append(arr["open_color"][i])
    for j in range(arr["closed_ctrl"].shape[0]):
        xs, ys = arr["closed_ctrl"][j, :, 0], arr["closed_ctrl"][j, :, 1]
        boxes.append((xs.min(), ys.min(), xs.max(), ys.max()))
        cols.append(arr["closed_color"][j])
    keys = area_keys_f32(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"])
    n = len(boxes)
    out = [False] * n
    for i in range(n):
        for j in range(n):
            if not (keys[j] < keys[i] or (keys[j] == keys[i] and j < i)):
                continue
            d = [f(cols[i][c]) - f(cols[j][c]) for c in range(3)]
            dist = np.sqrt(f(f(d[0] * d[0]) + f(d[1] * d[1])) + f(d[2] * d[2]))
            if not dist < f(cfg.color_eps):
                continue
            a, b = boxes[i], boxes[j]
            iw = max(f(0), f(min(a[2], b[2]) - max(a[0], b[0])))
            ih = max(f(0), f(min(a[3], b[3]) - max(a[1], b[1])))
            inter = f(iw * ih)
            uni = f(f(f(a[2] - a[0]) * f(a[3] - a[1])) + f(f(b[2] - b[0]) * f(b[3] - b[1]))) - inter
            if uni > 0 and f(inter / uni) > f(cfg.iou_min):
                out[i] = True
                break
    return np.array(out)


def test_overlap_matches_brute_force():
    rng = np.random.default_rng(5)
    n_o, n_c = 24, 24
    base_o = rng.uniform(0, 60, (4, 10, 2))
    base_c = np.stack([rect_closed(x, y, x + w, y + w) for x, y, w in rng.uniform(5, 40, (4, 3))])
    opens = [(base_o[i % 4] + rng.normal(0, 0.3, (10, 2)), rng.uniform(1, 3),
              (0.5, 0.5, 0.5) + rng.normal(0, 0.02, 3), (1, 1, 1)) for i in range(n_o)]
    closeds = [(base_c[i % 4] + rng.normal(0, 0.3, (12, 2)),
                (0.3, 0.6, 0.2) + rng.normal(0, 0.02, 3), 1.0) for i in range(n_c)]
    arr = curve_set(opens, closeds)
    cfg = PDCfg()
    _, crit = prune_flags(arr, cfg, SCFG, rows_per_chunk=7)
    ref = _brute_overlap(arr, cfg)
    assert ref.sum() > 5 and (~ref).sum() > 5
    assert crit["overlap"].tolist() == ref.tolist()


def test_split_rule():
    opac = [(0.9, 0.3, 0.9), (0.9, 0.45, 0.9), (0.9, 0.3, 0.7), (0.3, 0.9, 0.3), (0.95, 0.2, 0.8)]
    arr = curve_set(opens=[(line_open(0, i, 50, i), 2.0, (0, 0, 0), o) for i, o in enumerate(opac)])
    pruned = np.array([False, False, False, False, True])
    assert split_flags(arr, pruned, PDCfg()).tolist() == [True, False, False, False, False]
    assert split_flags(arr, np.zeros(5, bool), PDCfg(split_drop=0.1)).tolist() == [True, True, True, False, True]


def test_subdivide_thirds_traces_the_segment():
    rng = np.random.default_rng(2)
    seg = rng.uniform(-50, 50, (4, 2))
    out = subdivide_thirds(seg)
    assert out.shape == (10, 2)
    np.testing.assert_array_equal(out[0], seg[0])
    np.testing.assert_allclose(out[9], seg[3], atol=1e-12)
    t = torch.linspace(0, 1, 17, dtype=torch.float64)
    P = torch.as_tensor(seg)
    for s in range(3):
        sub = torch.as_tensor(out[3 * s: 3 * s + 4])
        np.testing.assert_allclose(bezier(sub, t).numpy(), bezier(P, (s + t) / 3).numpy(), atol=1e-11)


def _flood_roots(mask):
    """Breadth-first 4-connected flood fill; root = first pixel in row-major order."""
    H, W = mask.shape
    root = np.full((H, W), -1, np.int64)
    for y in range(H):
        for x in range(W):
            if mask[y, x] and root[y, x] < 0:
                r = y * W + x
                q = deque([(y, x)])
                root[y, x] = r
                while q:
                    cy, cx = q.popleft()
                    for ny, nx in ((cy - 1, cx), (cy + 1, cx), (cy, cx - 1), (cy, cx + 1)):
                        if 0 <= ny < H and 0 <= nx < W and mask[ny, nx] and root[ny, nx] < 0:
                            root[ny, nx] = r
                            q.append((ny, nx))
    return root


@pytest.mark.parametrize("seed,p", [(0, 0.45), (1, 0.6), (2, 0.3)])
def test_error_regions_match_flood_fill(seed, p):
    rng = np.random.default_rng(seed)
    H, W = 23, 31
    mask = rng.random((H, W)) < p
    target = rng.random((3, H, W)).astype(F)
    img = target.copy()
    img[:, mask] += F(0.5)            # error 0.5 on the masked pixels, 0 elsewhere
    root, m = error_regions(img, target, 0.1)
    assert (m == mask).all()
    assert (root == _flood_roots(mask)).all()


def test_error_map_is_channel_mean():
    target = np.zeros((3, 1, 4), F)
    img = np.zeros((3, 1, 4), F)
    img[0, 0, 0] = 0.35       # mean 0.1167 > 0.1
    img[0, 0, 1] = 0.29       # mean 0.0967 < 0.1
    img[:, 0, 2] = -0.11      # |.| mean 0.11 > 0.1
    img[1, 0, 3] = 0.31       # one channel: mean 0.1033 > 0.1
    _, m = error_regions(img, target, 0.1)
    assert m[0].tolist() == [True, False, True, True]


def test_diagonal_pixels_are_separate_regions():
    mask = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], bool)
    t = np.zeros((3, 3, 3), F)
    root, _ = error_regions(t + mask * F(1), t, 0.1)
    assert sorted(set(root[mask].tolist())) == [0, 4, 8]


def test_region_stats_closed_form():
    H, W = 10, 12
    mask = np.zeros((H, W), bool)
    mask[2:4, 3:6] = True          # area 6, centre (4.5, 3.0) in pixel-centre coords
    mask[7, 0:6] = True            # area 6, later root
    mask[0, 11] = True             # area 1
    mask[5:9, 9:11] = True         # area 8
    target = np.zeros((3, H, W), F)
    target[0, 2:4, 3:6] = 0.25
    target[1, 2, 3:6] = 1.0
    root, _ = error_regions(target * 0 + mask * F(1), target * 0, 0.1)
    st = region_stats(root, target)
    assert st["area"].tolist() == [8, 6, 6, 1]
    assert st["root"].tolist() == [5 * W + 9, 2 * W + 3, 7 * W + 0, 11]
    np.testing.assert_allclose([st["cx"][1], st["cy"][1]], [4.5, 3.0])
    np.testing.assert_allclose([st["cx"][0], st["cy"][0]], [10.0, 7.0])
    np.testing.assert_allclose(st["color"][1], [0.25, 0.5, 0.0])
    np.testing.assert_allclose(st["color"][2], [0, 0, 0])


def test_circle_curve_geometry():
    cx, cy, A = 37.25, 11.5, 200.0
    r = np.sqrt(A / np.pi)
    pc = circle_points(cx, cy, r, 12, 12)
    np.testing.assert_allclose(np.hypot(pc[:, 0] - cx, pc[:, 1] - cy), r)
    # regular 12-gon inscribed in radius r: area 3 r^2 = 3 A / pi
    key = area_keys_f32(np.zeros((0, 10, 2)), np.zeros(0), pc[None])
    np.testing.assert_allclose(key, [3 * A / np.pi], rtol=1e-6)
    po = circle_points(cx, cy, r, 10, 11)
    ang = np.arctan2(po[:, 1] - cy, po[:, 0] - cx) % (2 * np.pi)
    np.testing.assert_allclose(np.diff(ang), 2 * np.pi / 11, atol=1e-12)


def _op(y, o):
    return (line_open(0, y, 40, y), 2.0, (0.1, 0.2, 0.3), o)


def test_prune_densify_slot_assignment():
    """Split half to the first free open slot, then regions by area into the
    remaining free slots (open first), leftovers made transparent."""
    opens = [_op(0, (0.9, 0.2, 0.8)),         # 0: split
             _op(3, (0.05, 0.05, 0.05)),      # 1: pruned (low opacity) -> split half
             _op(6, (1, 1, 1)),               # 2: untouched
             _op(9, (0.01, 0.01, 0.01))]      # 3: pruned -> largest region
    closeds = [(rect_closed(50, 50, 60, 60), (0.5, 0.5, 0.5), 0.01),   # 4: pruned -> 1st area-20
               (rect_closed(70, 70, 80, 80), (0.5, 0.5, 0.5), 1.0),    # 5: untouched
               (rect_closed(0, 60, 1, 61), (0.9, 0.9, 0.9), 1.0),      # 6: small -> 2nd area-20
               (rect_closed(90, 0, 99, 9), (0.2, 0.2, 0.2), 0.0)]      # 7: pruned -> transparent
    arr = curve_set(opens, closeds)
    H, W = 32, 40
    target = np.full((3, H, W), 0.25, F)
    img = target.copy()
    img[:, 2:10, 2:12] = 1.0        # area 80
    img[:, 20:25, 30:34] = 1.0      # area 20, root 20*W+30
    img[:, 28:30, 0:10] = 1.0       # area 20, later root
    out, changed, info = prune_densify(arr, img, target, PDCfg(), SCFG)
    assert info["pruned"].tolist() == [False, True, False, True, True, False, True, True]
    assert info["split"].tolist() == [True, False, False, False]
    assert changed.tolist() == [True, True, False, True, True, False, True, True]
    assert info["free"] == [3, 4, 6, 7]
    # curve 0 keeps its first segment, curve 1 receives the last one
    np.testing.assert_allclose(out["open_ctrl"][0], subdivide_thirds(arr["open_ctrl"][0][0:4]))
    np.testing.assert_allclose(out["open_ctrl"][1], subdivide_thirds(arr["open_ctrl"][0][6:10]))
    np.testing.assert_allclose(out["open_opac"][0], [0.9] * 3, rtol=1e-7)
    np.testing.assert_allclose(out["open_opac"][1], [0.8] * 3, rtol=1e-7)
    np.testing.assert_allclose(out["open_color"][1], arr["open_color"][0])
    np.testing.assert_allclose(out["open_width"][1], arr["open_width"][0])
    # untouched curves
    for k in ("open_ctrl", "open_opac", "open_color", "open_width"):
        np.testing.assert_array_equal(out[k][2], arr[k][2])
    np.testing.assert_array_equal(out["closed_ctrl"][1], arr["closed_ctrl"][1])
    # open slot 3 <- area 80 centred at (7, 6) in pixel-centre coordinates
    np.testing.assert_allclose(out["open_ctrl"][3][0], [7.0 + np.sqrt(80 / np.pi), 6.0])
    np.testing.assert_allclose(out["open_opac"][3], [0.5] * 3)
    np.testing.assert_allclose(out["open_width"][3], 2.0)
    np.testing.assert_allclose(out["open_color"][3], [0.25] * 3)
    # closed 4 <- the area-20 region with the lower first pixel, closed 6 <- the other
    np.testing.assert_allclose(out["closed_ctrl"][0].mean(0), [32.0, 22.5])
    np.testing.assert_allclose(out["closed_ctrl"][2].mean(0), [5.0, 29.0])
    np.testing.assert_allclose(out["closed_opac"], [0.5, 1.0, 0.5, 0.0])
    np.testing.assert_array_equal(out["closed_ctrl"][3], arr["closed_ctrl"][3])
    for k in arr:
        assert out[k].shape == arr[k].shape       # the curve budget is constant


def test_split_without_free_open_slot_drops_the_second_half():
    arr = curve_set([_op(0, (0.9, 0.1, 0.9)), _op(5, (1, 1, 1))],
                    [(rect_closed(50, 50, 60, 60), (0.5, 0.5, 0.5), 0.01)])
    target = np.zeros((3, 8, 8), F)
    img = target.copy()
    img[:, 1:3, 1:3] = 1.0
    out, changed, info = prune_densify(arr, img, target, PDCfg(), SCFG)
    assert changed.tolist() == [True, False, True]
    np.testing.assert_allclose(out["open_ctrl"][0], subdivide_thirds(arr["open_ctrl"][0][0:4]))
    np.testing.assert_array_equal(out["open_ctrl"][1], arr["open_ctrl"][1])
    np.testing.assert_allclose(out["closed_ctrl"][0].mean(0), [2.0, 2.0], atol=1e-12)
    np.testing.assert_allclose(np.hypot(*(out["closed_ctrl"][0] - 2.0).T), np.sqrt(4 / np.pi))
