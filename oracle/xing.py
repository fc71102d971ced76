"""The Xing loss of Eq. 13 (the convexity term the paper adopts from LIVE).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading (the paper does not restate the term; this follows LIVE's published
definition): for each cubic segment with control points A, B, C, D, with
u = B - A, v = C - B, w = D - C,
    D1 = 1 if u x v >= 0 else 0      (the turn at B)
    D2 = (u x w) / (|u| |w|)          (sine of the angle from AB to CD)
    L  = D1 relu(-D2) + (1 - D1) relu(D2),
which is positive when the segment's end legs turn against its first turn,
as a self-intersecting segment does.  Applied to the four segments of every
closed curve (segment s: P_3s .. P_3s+3 with P_12 = P_0); the loss is
lambda times the mean over all segments.  D1 is a step function and carries
no gradient; a segment with |u| = 0 or |w| = 0 contributes 0.
"""

from __future__ import annotations

import torch


def cross(a, b):
    return a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]


def xing_loss(closed_ctrl, lam: float = 1.0):
    P = torch.as_tensor(closed_ctrl, dtype=torch.float64)
    n = P.shape[0]
    if n == 0:
        return P.sum() * 0.0
    idx = torch.arange(4)[:, None] * 3 + torch.arange(4)[None, :]          # [4 segments, 4 points]
    seg = P[:, idx % 12]                                                    # [Nc, 4, 4, 2]
    A, B, C, D = seg[..., 0, :], seg[..., 1, :], seg[..., 2, :], seg[..., 3, :]
    u, v, w = B - A, C - B, D - C
    nu, nw = torch.linalg.norm(u, dim=-1), torch.linalg.norm(w, dim=-1)
    ok = (nu > 0) & (nw > 0)
    d1 = (cross(u, v) >= 0).double().detach()
    d2 = torch.where(ok, cross(u, w) / torch.where(ok, nu * nw, torch.ones_like(nu)), torch.zeros_like(nu))
    L = d1 * torch.relu(-d2) + (1.0 - d1) * torch.relu(d2)
    return lam * L.sum() / (4 * n)
