"""The seeded synthetic inputs (no GPU): the same seed gives the same
arrays, the ragged batch follows its recipe (sides log-uniform in [256,
2048], aspect W / H in [0.5, 2], curve counts in [128, 4096], half open and
half closed), and the curve and target generators stay in range."""

import numpy as np

from paper_2503_16424_gb300 import synth


def test_generators_are_seeded():
    a = synth.make_curves(7, 300, 200, 5, 4, style="local").as_dict()
    b = synth.make_curves(7, 300, 200, 5, 4, style="local").as_dict()
    c = synth.make_curves(8, 300, 200, 5, 4, style="local").as_dict()
    for k in a:
        assert np.array_equal(a[k], b[k])
    assert not np.array_equal(a["open_ctrl"], c["open_ctrl"])
    assert np.array_equal(synth.procedural_target(3, 64, 48, 5), synth.procedural_target(3, 64, 48, 5))


def test_curve_attributes_in_their_ranges():
    a = synth.make_curves(11, 512, 384, 40, 30, style="local").as_dict()
    assert a["open_ctrl"].shape == (40, 10, 2) and a["closed_ctrl"].shape == (30, 12, 2)
    assert np.all((a["open_width"] >= 1.0) & (a["open_width"] <= 4.0))
    for k in ("open_color", "closed_color"):
        assert np.all((a[k] >= 0.0) & (a[k] <= 1.0))
    for k in ("open_opac", "closed_opac"):
        assert np.all((a[k] >= 0.3) & (a[k] <= 1.0))
    for k in a:
        assert a[k].dtype == np.float32


def test_target_is_planar_and_in_range():
    t = synth.procedural_target(5, 96, 64, 12)
    assert t.shape == (3, 64, 96) and t.dtype == np.float32
    assert np.all(np.isfinite(t))
    assert t.min() > -0.1 and t.max() < 1.1   # 8-bit shapes plus N(0, 0.01) noise


def test_batch_layout_follows_its_recipe():
    W = synth.BATCH_WORKLOAD
    lay = synth.batch_layout(W["seed"], W["n_images"], W["side"], W["aspect"], W["curves"])
    assert lay == synth.batch_layout(W["seed"], W["n_images"], W["side"], W["aspect"], W["curves"])
    assert len(lay) == 64
    sides = np.array([np.sqrt(e["W"] * e["H"]) for e in lay])
    aspects = np.array([e["W"] / e["H"] for e in lay])
    counts = np.array([e["n_open"] + e["n_closed"] for e in lay])
    assert np.all((sides >= 256 * 0.99) & (sides <= 2048 * 1.01))
    assert np.all((aspects >= 0.5 * 0.99) & (aspects <= 2.0 * 1.01))
    assert np.all((counts >= 128) & (counts <= 4096))
    assert all(e["n_open"] == (e["n_open"] + e["n_closed"]) // 2 for e in lay)
    # log-uniform sides: the median sits near the geometric mean of the range
    assert 0.6 * np.sqrt(256 * 2048) < np.median(sides) < 1.6 * np.sqrt(256 * 2048)
    assert len({e["seed"] for e in lay}) == 64
