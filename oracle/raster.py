"""Section 3.4: front-to-back alpha blending, by brute force.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For every requested pixel and EVERY Gaussian, in draw order (no culling):
  d     = p - mu,  p = (x + 0.5, y + 0.5) the pixel centre
  s     = 0.5 d^T Sigma^-1 d                      (Eq. 10, Sigma from Eq. 11-12)
  alpha = min(0.99, o exp(-s))                    (Eq. 10 with the clamp below)
  C     = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j) + T_final bg      (Eq. 9)

Readings (the paper says only that it follows the 3D Gaussian splatting
tile rasterizer, whose thresholds it does not restate):
  * alpha is clamped to 0.99;
  * a Gaussian with alpha < 1/255 is skipped (contributes nothing);
  * the pixel stops at the first Gaussian that would bring its
    transmittance below 1e-4; that Gaussian is not blended;
  * the background colour bg is added with the final transmittance.

The product over j<i is torch.cumprod over the draw-ordered Gaussians, which
is Eq. 9's product written as a scan.
"""

from __future__ import annotations

import torch

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4


def _alpha_raw(tab, px, py):
    """o exp(-0.5 d^T Sigma^-1 d) with Sigma^-1 = R diag(isx^2, isy^2) R^T,
    R = [[ux, -uy], [uy, ux]] (Eq. 10-12), so d^T Sigma^-1 d = |S^-1 R^T d|^2."""
    dx = px[:, None] - tab["mx"][None, :]
    dy = py[:, None] - tab["my"][None, :]
    a = (tab["ux"][None] * dx + tab["uy"][None] * dy) * tab["isx"][None]      # along the curve
    b = (-tab["uy"][None] * dx + tab["ux"][None] * dy) * tab["isy"][None]     # across it
    s = 0.5 * (a * a + b * b)
    return tab["o"][None] * torch.exp(-s)


def render_pixels(tab: dict, xs, ys, bg=(0.0, 0.0, 0.0), margin: float = 1e-4, margin_T=None):
    """Blend all Gaussians of ``tab`` at pixels (xs[i], ys[i]).

    Returns dict(C [n,3], T [n] final transmittance, last [n] index of the
    last blended Gaussian or -1, n_blend [n], flag [n], stop [n] index of the
    Gaussian at which the pixel stops, or the number of Gaussians).  ``flag`` marks a
    pixel where some threshold decision (the 1/255 skip, the 1e-4 stop, the
    0.99 clamp) lies within a relative ``margin`` of its threshold (``margin_T``
    for the transmittance stop, default ``margin``), so that an fp32
    evaluation may legitimately decide it the other way.
    Differentiable in the table entries."""
    xs = torch.as_tensor(xs, dtype=torch.float64)
    ys = torch.as_tensor(ys, dtype=torch.float64)
    px, py = xs + 0.5, ys + 0.5
    n = px.shape[0]
    a_raw = _alpha_raw(tab, px, py)                               # [n, Ng]
    alpha = torch.clamp(a_raw, max=ALPHA_MAX)
    alpha = torch.where(a_raw >= ALPHA_MIN, alpha, torch.zeros_like(alpha))
    one_minus = 1.0 - alpha
    T_after = torch.cumprod(one_minus, dim=1)                     # prod_{j<=i}
    T_before = torch.cat([torch.ones(n, 1, dtype=alpha.dtype), T_after[:, :-1]], dim=1)
    ng = alpha.shape[1]
    stop = (alpha > 0) & (T_after < T_MIN)
    idx = torch.arange(ng)[None, :].expand(n, -1)
    first_stop = torch.where(stop, idx, torch.full_like(idx, ng)).min(dim=1).values
    keep = (idx < first_stop[:, None]) & (alpha > 0)
    w = torch.where(keep, alpha * T_before, torch.zeros_like(alpha))
    C = w @ tab["col"]
    T_ext = torch.cat([T_before, T_after[:, -1:]], dim=1)          # T_before[ng] = T_after[-1]
    T_final = T_ext.gather(1, first_stop[:, None])[:, 0]
    bg_t = torch.as_tensor(bg, dtype=torch.float64)
    C = C + T_final[:, None] * bg_t[None, :]
    with torch.no_grad():
        last = torch.where(keep, idx, torch.full_like(idx, -1)).max(dim=1).values
        n_blend = keep.sum(dim=1)
        considered = idx <= first_stop[:, None]
        near_skip = (torch.abs(a_raw - ALPHA_MIN) <= margin * ALPHA_MIN) & considered
        near_clamp = (torch.abs(a_raw - ALPHA_MAX) <= margin) & considered & (a_raw >= ALPHA_MIN)
        mT = margin if margin_T is None else margin_T
        near_stop = (torch.abs(T_after - T_MIN) <= mT * T_MIN) & considered & (alpha > 0)
        flag = (near_skip | near_clamp | near_stop).any(dim=1)
    return dict(C=C, T=T_final, last=last, n_blend=n_blend, flag=flag, stop=first_stop)


def _chunks(n, size):
    for s in range(0, n, size):
        yield s, min(n, s + size)


def render_image(tab: dict, W: int, H: int, bg=(0.0, 0.0, 0.0), margin=1e-4, margin_T=None,
                 max_entries: int = 1 << 22):
    """Brute-force render of a W x H image.  Returns planar img [3,H,W],
    T [H,W], last [H,W], flag [H,W], stop [H,W], n_blend [H,W] (no autograd)."""
    ng = max(1, tab["mx"].shape[0])
    chunk = max(1, max_entries // ng)
    ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64),
                            torch.arange(W, dtype=torch.float64), indexing="ij")
    xs, ys = xs.reshape(-1), ys.reshape(-1)
    C, T, last, flag, stop, nb = [], [], [], [], [], []
    with torch.no_grad():
        for s, e in _chunks(xs.shape[0], chunk):
            r = render_pixels(tab, xs[s:e], ys[s:e], bg, margin, margin_T)
            C.append(r["C"]); T.append(r["T"]); last.append(r["last"]); flag.append(r["flag"])
            stop.append(r["stop"]); nb.append(r["n_blend"])
    C = torch.cat(C).reshape(H, W, 3).permute(2, 0, 1).contiguous()
    return dict(img=C, T=torch.cat(T).reshape(H, W), last=torch.cat(last).reshape(H, W),
                flag=torch.cat(flag).reshape(H, W), stop=torch.cat(stop).reshape(H, W),
                n_blend=torch.cat(nb).reshape(H, W))


GRAD_KEYS = ("mx", "my", "ux", "uy", "isx", "isy", "o", "col")


def render_grads(tab: dict, xs, ys, dC, bg=(0.0, 0.0, 0.0), max_entries: int = 1 << 21):
    """Vector-Jacobian product of render_pixels: given dL/dC [n,3] at pixels
    (xs, ys), return dL/d(table field) for every field of GRAD_KEYS, by
    autograd through the brute-force definition, accumulated over pixel
    chunks (the loss is a sum over pixels)."""
    leaves = {k: tab[k].detach().clone().requires_grad_(True) for k in GRAD_KEYS}
    grads = {k: torch.zeros_like(v) for k, v in leaves.items()}
    xs = torch.as_tensor(xs, dtype=torch.float64)
    ys = torch.as_tensor(ys, dtype=torch.float64)
    dC = torch.as_tensor(dC, dtype=torch.float64)
    ng = max(1, leaves["mx"].shape[0])
    chunk = max(1, max_entries // ng)
    for s, e in _chunks(xs.shape[0], chunk):
        r = render_pixels(leaves, xs[s:e], ys[s:e], bg)
        gs = torch.autograd.grad(r["C"], [leaves[k] for k in GRAD_KEYS], grad_outputs=dC[s:e],
                                 allow_unused=True)
        for k, g in zip(GRAD_KEYS, gs):
            if g is not None:
                grads[k] += g
    return grads
