"""Section 3.5, Eq. 13: the L2 reconstruction term.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading: lambda_1 = 1 and the squared norm is averaged over the 3HW entries
(the paper gives no value for lambda_1 and no normalisation); the Xing term
of Eq. 13 is off (lambda_2 = 0).
"""

from __future__ import annotations

import torch


def l2_loss(img, target):
    """L = mean((img - target)^2) and dL/dimg = 2 (img - target) / (3HW)."""
    img = torch.as_tensor(img, dtype=torch.float64)
    target = torch.as_tensor(target, dtype=torch.float64)
    diff = img - target
    n = diff.numel()
    return (diff * diff).sum() / n, 2.0 * diff / n
