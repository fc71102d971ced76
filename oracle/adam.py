"""Adam, the optimiser of Section 4.1 (Kingma and Ba, "Adam: A Method for
Stochastic Optimization", Algorithm 1), followed by a projection onto a box.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Per parameter, at step t = 1, 2, ...:
  m_t   = beta1 m_{t-1} + (1 - beta1) g_t
  v_t   = beta2 v_{t-1} + (1 - beta2) g_t^2
  m_hat = m_t / (1 - beta1^t),  v_hat = v_t / (1 - beta2^t)
  p_t   = p_{t-1} - lr m_hat / (sqrt(v_hat) + eps)
and then p_t is clamped to [lo, hi] (reading: the rasterizer's parameters
are activated values, colours and opacities in [0, 1], so the update is
projected onto their box).  All arithmetic in float64.
"""

from __future__ import annotations

import numpy as np


def adam_step(p, g, m, v, t: int, lr, beta1=0.9, beta2=0.999, eps=1e-8, lo=-np.inf, hi=np.inf):
    """One step at step number t (>= 1).  lr may be an array broadcastable
    to p (per-parameter learning rates).  Returns (p, m, v), new arrays."""
    p = np.asarray(p, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    p = p - np.asarray(lr, dtype=np.float64) * m_hat / (np.sqrt(v_hat) + eps)
    return np.clip(p, lo, hi), m, v
