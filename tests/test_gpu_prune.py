"""Parity of bs_prune_densify (Section 3.5, Algorithm 1, Appendix B) with the
CPU oracle on the same seeded inputs.

Bars: the changed mask and every count bit-exact; curves the pass leaves
alone bit-identical to the input; edited values within 2 float32 ulps of the
oracle's fp64 result (the two differ only in the last double bits of a
cosine or of a differently ordered colour sum before the float32 cast)."""

import numpy as np
import pytest
import torch

from oracle.curves import SampleCfg as OCfg
from oracle.prune_densify import PDCfg as OPD, prune_densify as oracle_pd
from paper_2503_16424_gb300 import synth

pytestmark = pytest.mark.gpu

FIELDS = ("open_ctrl", "open_width", "open_color", "open_opac", "closed_ctrl", "closed_color", "closed_opac")
OCFG = OCfg(g_open=16, rows_closed=4, k_closed=8)


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def expected_stats(info):
    n_open = info["split"].shape[0]
    free_open = int(info["pruned"][:n_open].sum())
    split = int(info["split"].sum())
    regions = int(info["regions"]["area"].shape[0])
    slots = len(info["free"])
    return dict(pruned=int(info["pruned"].sum()), low_opacity=int(info["low_op"].sum()),
                small_area=int(info["small"].sum()), overlap=int(info["overlap"].sum()), split=split,
                split_placed=min(split, free_open), regions=regions, inserted=min(slots, regions),
                transparent=slots - min(slots, regions))


def run_both(bs, arr, img, tgt, W, H, **kw):
    o_out, o_changed, info = oracle_pd(arr, img, tgt, OPD(**kw), OCFG)
    curves = bs.CurveSet.from_arrays(arr)
    changed, st = bs.prune_densify(curves, torch.as_tensor(img).cuda(), torch.as_tensor(tgt).cuda(),
                                   bs.PDCfg(**kw), bs.Canvas(W, H))
    torch.cuda.synchronize()
    return curves, changed.cpu().numpy().astype(bool), st, o_out, o_changed, info


def compare(arr, curves, changed, st, o_out, o_changed, info):
    assert st == expected_stats(info)
    assert changed.tolist() == o_changed.tolist()
    n_open = arr["open_ctrl"].shape[0]
    for k in FIELDS:
        g = getattr(curves, k).cpu().numpy()
        o = o_out[k].astype(np.float32)
        rows = o_changed[:n_open] if k.startswith("open") else o_changed[n_open:]
        np.testing.assert_array_equal(g[~rows], np.asarray(arr[k], np.float32)[~rows], err_msg=k)
        tol = 2 * np.spacing(np.abs(o))
        bad = np.abs(g.astype(np.float64) - o) > tol
        assert not bad.any(), (k, np.argwhere(bad)[:5], g[bad][:5], o[bad][:5])


@pytest.mark.parametrize("seed,W,H,n_open,n_closed,n_blobs", [
    (3, 300, 211, 200, 150, 40),     # ragged canvas, more regions than freed slots
    (4, 300, 211, 200, 150, 2),      # few regions: leftover slots made transparent
    (5, 97, 61, 120, 0, 12),         # open curves only
    (6, 97, 61, 0, 90, 12),          # closed curves only
    (7, 1, 97, 30, 20, 6),           # one-pixel-wide canvas
    (8, 131, 1, 30, 20, 6),          # one-row canvas
])
def test_prune_densify_matches_oracle(bs, seed, W, H, n_open, n_closed, n_blobs):
    arr, img, tgt = synth.prune_inputs(seed, W, H, n_open, n_closed, n_blobs=n_blobs)
    res = run_both(bs, arr, img, tgt, W, H, step=10, t_end=100)
    compare(arr, *res)
    assert res[2]["pruned"] > 0


def test_schedule_and_thresholds_are_honoured(bs):
    W, H = 160, 120
    arr, img, tgt = synth.prune_inputs(11, W, H, 150, 100, n_blobs=30)
    for kw in (dict(step=0, t_end=50), dict(step=50, t_end=50), dict(step=25, t_end=50, area_min=40.0),
               dict(color_eps=0.2, iou_min=0.5, split_drop=0.3, err_thresh=0.25, new_opacity=0.7, new_width=3.5)):
        compare(arr, *run_both(bs, arr, img, tgt, W, H, **kw))


def test_checkerboard_errors_give_the_most_regions(bs):
    W, H = 67, 45
    arr, _, tgt = synth.prune_inputs(12, W, H, 60, 40, n_blobs=0)
    ys, xs = np.mgrid[0:H, 0:W]
    img = tgt + np.float32(0.5) * ((xs + ys) % 2 == 0)[None].astype(np.float32)
    res = run_both(bs, arr, img.astype(np.float32), tgt, W, H)
    assert res[2]["regions"] == (W * H + 1) // 2
    compare(arr, *res)


@pytest.mark.parametrize("mode", ["none", "all"])
def test_no_error_and_all_error(bs, mode):
    W, H = 90, 70
    arr, _, tgt = synth.prune_inputs(13, W, H, 80, 60, n_blobs=0)
    img = tgt.copy() if mode == "none" else tgt + np.float32(0.4)
    res = run_both(bs, arr, img.astype(np.float32), tgt, W, H)
    assert res[2]["regions"] == (0 if mode == "none" else 1)
    compare(arr, *res)


def test_nothing_to_prune_leaves_curves_alone(bs):
    W, H = 64, 48
    c = synth.make_curves(14, W, H, 20, 10, style="uniform", opac_range=(0.9, 1.0)).as_dict()
    tgt = synth.procedural_target(14, W, H, 5)
    res = run_both(bs, c, tgt + np.float32(0.3), tgt, W, H, area_min=0.0)
    curves, changed, st = res[:3]
    assert st["pruned"] == 0 and st["split"] == 0 and not changed.any()
    compare(c, *res)


def test_two_passes_in_a_row(bs):
    """The second pass reads the first pass's output and reuses its workspace."""
    W, H = 200, 150
    arr, img, tgt = synth.prune_inputs(15, W, H, 120, 90, n_blobs=25)
    o1, _, _ = oracle_pd(arr, img, tgt, OPD(step=0, t_end=10), OCFG)
    o1 = {k: v.astype(np.float32) for k, v in o1.items()}
    curves = bs.CurveSet.from_arrays(arr)
    i_d, t_d = torch.as_tensor(img).cuda(), torch.as_tensor(tgt).cuda()
    nbytes = bs.prune_densify_workspace(curves.n_open, curves.n_closed, bs.Canvas(W, H))
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    bs.prune_densify(curves, i_d, t_d, bs.PDCfg(step=0, t_end=10), bs.Canvas(W, H), ws=ws)
    g1 = {k: getattr(curves, k).cpu().numpy() for k in FIELDS}
    for k in FIELDS:   # the first pass agrees to 2 ulps; continue from the GPU's own result
        assert np.all(np.abs(g1[k].astype(np.float64) - o1[k]) <= 2 * np.spacing(np.abs(o1[k])))
    o2, o2_changed, info2 = oracle_pd(g1, img, tgt, OPD(step=10, t_end=10, err_thresh=0.2), OCFG)
    changed, st = bs.prune_densify(curves, i_d, t_d, bs.PDCfg(step=10, t_end=10, err_thresh=0.2), bs.Canvas(W, H),
                                   ws=ws)
    compare(g1, curves, changed.cpu().numpy().astype(bool), st, o2, o2_changed, info2)


def test_full_size_workload(bs):
    """2048 x 2048 canvas, 2048 open + 2048 closed curves."""
    W = H = 2048
    arr, img, tgt = synth.prune_inputs(20, W, H, 2048, 2048, n_blobs=300)
    res = run_both(bs, arr, img, tgt, W, H, step=200, t_end=1000)
    assert res[2]["pruned"] > 100 and res[2]["regions"] > 100
    compare(arr, *res)


def test_pruned_curves_render_through_the_pipeline(bs):
    """After a pass the curve set goes straight back into the rasterizer."""
    from paper_2503_16424_gb300.raster import Rasterizer
    W, H = 128, 96
    arr, img, tgt = synth.prune_inputs(16, W, H, 40, 30, n_blobs=10)
    curves = bs.CurveSet.from_arrays(arr)
    r = Rasterizer(bs.Canvas(W, H), bs.SampleCfg(g_open=16, rows_closed=4, k_closed=8), 40, 30)
    t_d = torch.as_tensor(tgt).cuda()
    loss0, _ = r.step(curves, t_d)
    changed, st = r.prune_densify(curves, t_d, bs.PDCfg(), img=torch.as_tensor(img).cuda())
    assert st["pruned"] > 0 and changed.any()
    loss1, grad = r.step(curves, t_d)
    assert torch.isfinite(loss1) and all(torch.isfinite(getattr(grad, k)).all() for k in FIELDS)


def test_bounded_retry_gives_up_and_recovers(bs):
    """With no linking attempt allowed, the union step gives up: the call
    reports BS_ERR_TIMEOUT and returns (nothing waits).  With the default
    bound restored the next call matches the oracle."""
    W, H = 120, 90
    arr, img, tgt = synth.prune_inputs(17, W, H, 60, 40, n_blobs=12)
    curves = bs.CurveSet.from_arrays(arr)
    i_d, t_d = torch.as_tensor(img).cuda(), torch.as_tensor(tgt).cuda()
    try:
        bs.debug_retry_limit(0)
        with pytest.raises(bs.BSError) as e:
            bs.prune_densify(curves, i_d, t_d, bs.PDCfg(), bs.Canvas(W, H))
        assert e.value.status == bs.BS_ERR_TIMEOUT
    finally:
        bs.debug_retry_limit(-1)
    compare(arr, *run_both(bs, arr, img, tgt, W, H))
