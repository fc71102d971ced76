"""Pins of the Xing-loss oracle by closed forms and finite differences."""

import numpy as np
import torch

from oracle.xing import xing_loss


def _ring(cx, cy, r, n=1):
    a = 2 * np.pi * np.arange(12) / 12
    return np.tile(np.stack([cx + r * np.cos(a), cy + r * np.sin(a)], -1)[None], (n, 1, 1))


def test_convex_curves_cost_nothing():
    assert float(xing_loss(_ring(10, 20, 7, 3))) == 0.0
    # the same ring walked the other way round is still convex
    assert float(xing_loss(_ring(10, 20, 7)[:, ::-1].copy())) == 0.0


def test_a_crossing_segment_in_closed_form():
    # A = (0,0), B = (1,1), C = (1,0), D = (0,1): u x v = -1 (D1 = 0),
    # u x w = 2, |u| |w| = 2, so D2 = 1 and L = 1; the other three segments
    # of this curve are straight and cost nothing
    P = np.zeros((1, 12, 2))
    P[0, 0:4] = [[0, 0], [1, 1], [1, 0], [0, 1]]
    for j in range(4, 12):                  # back to P0 along a straight path
        t = (j - 3) / 9.0
        P[0, j] = (1 - t) * np.array([0.0, 1.0])
    assert abs(float(xing_loss(P, lam=2.0)) - 2.0 * 1.0 / 4.0) < 1e-12


def test_degenerate_legs_cost_nothing():
    P = _ring(0, 0, 5)
    P[0, 1] = P[0, 0]                       # |u| = 0 for segment 0
    assert float(xing_loss(P)) == 0.0


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    P = _ring(0, 0, 10, 6) + rng.normal(0, 6, (6, 12, 2))
    t = torch.tensor(P, requires_grad=True)
    L = xing_loss(t, lam=0.7)
    assert float(L.detach()) > 0.0
    (g,) = torch.autograd.grad(L, t)
    g = g.numpy()
    for (c, j, k) in [tuple(int(x) for x in np.unravel_index(i, P.shape)) for i in np.argsort(-np.abs(g).ravel())[:8]]:
        h = 1e-7
        Pp, Pm = P.copy(), P.copy()
        Pp[c, j, k] += h
        Pm[c, j, k] -= h
        fd = (float(xing_loss(Pp, 0.7)) - float(xing_loss(Pm, 0.7))) / (2 * h)
        assert abs(fd - g[c, j, k]) <= 1e-6 * max(1.0, abs(fd))
