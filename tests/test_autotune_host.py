"""The autotuner's host-side rules (no GPU): the spacing rule picks, per
image, the sparsest sampling whose spacing along the median open curve, and
across and along the median closed curve, is at most max_spacing px; the
image list keeps everything but its sampling."""

import numpy as np
import pytest

from paper_2503_16424_gb300 import autotune, bs


def _line(x0, x1, y=50.0):
    """Open-curve control points on a straight line: polygon length x1 - x0."""
    xs = np.linspace(x0, x1, 10)
    return np.stack([xs, np.full(10, y)], 1)


def _closed(cx, cy, half_w, half_h):
    """Closed-curve control points: boundary A = P0..P6 along the top, B =
    P0, P11..P7, P6 along the bottom, both from (cx - half_w, cy) to
    (cx + half_w, cy); their middles P3 and P9 are 2 half_h apart."""
    xs = np.linspace(cx - half_w, cx + half_w, 7)
    top = np.stack([xs, np.full(7, cy - half_h)], 1)
    bot = np.stack([xs, np.full(7, cy + half_h)], 1)
    top[0] = bot[0] = (cx - half_w, cy)
    top[6] = bot[6] = (cx + half_w, cy)
    P = np.zeros((12, 2))
    P[0:7] = top
    P[7:12] = bot[5:0:-1]   # P7..P11 = B_5..B_1
    return P


def _expected(choices, length, max_spacing):
    for c in choices:
        if length / (c - 1) <= max_spacing:
            return c
    return choices[-1]


def _polyline(P):
    return float(np.linalg.norm(np.diff(P, axis=0), axis=1).sum())


@pytest.mark.parametrize("max_spacing", [4.0, 8.0, 12.0])
def test_open_curves_take_the_sparsest_sampling_of_the_median_length(max_spacing):
    lengths = [40.0, 300.0, 900.0]          # median 300
    arr = {"open_ctrl": np.stack([_line(10, 10 + L) for L in lengths])}
    im = bs.BatchImage(1024, 256, 3, 0, bs.SampleCfg())
    (g, rows, k), = autotune.spacing_sampling([im], [arr], max_spacing)
    assert g == _expected(autotune.OPEN_CHOICES, 300.0, max_spacing)
    assert 300.0 / (g - 1) <= max_spacing or g == autotune.OPEN_CHOICES[-1]
    if g != autotune.OPEN_CHOICES[0]:
        smaller = autotune.OPEN_CHOICES[autotune.OPEN_CHOICES.index(g) - 1]
        assert 300.0 / (smaller - 1) > max_spacing          # the sparsest that qualifies
    # no closed curves: their sampling stays at the sparsest choice
    assert (rows, k) == (autotune.ROW_CHOICES[0], autotune.K_CHOICES[0])


def test_closed_curves_take_rows_from_the_width_and_samples_from_the_boundary_length():
    shapes = [(200, 200, 30, 10), (200, 200, 60, 25), (200, 200, 150, 80)]   # median: 60 x 25
    P = np.stack([_closed(*s) for s in shapes])
    arr = {"closed_ctrl": P}
    im = bs.BatchImage(400, 400, 0, 3, bs.SampleCfg())
    (g, rows, k), = autotune.spacing_sampling([im], [arr], 8.0)
    across = 2 * 25.0
    along = max(_polyline(P[1, 0:7]), _polyline(P[1][[0, 11, 10, 9, 8, 7, 6]]))
    assert rows == _expected(autotune.ROW_CHOICES, across, 8.0)
    assert k == _expected(autotune.K_CHOICES, along, 8.0)
    assert g == autotune.OPEN_CHOICES[0]


def test_huge_curves_saturate_at_the_densest_choice():
    arr = {"open_ctrl": _line(0, 1e5)[None], "closed_ctrl": _closed(0, 0, 1e5, 1e5)[None]}
    im = bs.BatchImage(64, 64, 1, 1, bs.SampleCfg())
    (g, rows, k), = autotune.spacing_sampling([im], [arr], 8.0)
    assert (g, rows, k) == (autotune.OPEN_CHOICES[-1], autotune.ROW_CHOICES[-1], autotune.K_CHOICES[-1])


def test_with_sampling_keeps_everything_but_the_sampling():
    cfg = bs.SampleCfg(g_open=16, rows_closed=4, k_closed=4, rho=0.7, cov_eps=1e-3)
    images = [bs.BatchImage(300, 200, 5, 3, cfg, (0.1, 0.2, 0.3)), bs.BatchImage(64, 90, 0, 2, cfg)]
    out = autotune.with_sampling(images, [(32, 8, 16), (64, 16, 32)])
    for a, b, pick in zip(images, out, [(32, 8, 16), (64, 16, 32)]):
        assert (b.width, b.height, b.n_open, b.n_closed, tuple(b.bg)) == \
            (a.width, a.height, a.n_open, a.n_closed, tuple(a.bg))
        assert (b.sample.g_open, b.sample.rows_closed, b.sample.k_closed) == pick
        assert (b.sample.rho, b.sample.cov_eps) == (a.sample.rho, a.sample.cov_eps)
