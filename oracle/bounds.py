"""Error scales of the gradients: the sums of ABSOLUTE per-pixel terms.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A gradient entry of the blend backward (Section 3.4, the reverse walk of
Eq. 9-10) is a sum over pixels p of a per-pixel term
    term[p, g, k] = dL/dalpha[p, g] * dalpha[p, g] / dtheta[g, k]
(colour: dL/dC[p] * w[p, g], w = alpha T the blend weight).  Evaluated in
float32, such a sum carries a rounding error bounded by
    |fl(sum) - sum| <= gamma_n * sum_p |term[p, g, k]|,   gamma_n ~ n u,
with u = 2^-24 and n the longest chain of roundings from a term to the
result (the standard forward error bound of recursive summation, Higham,
"Accuracy and Stability of Numerical Algorithms", Section 4.2).  When the
terms cancel, that bound is far above 1e-3 |gradient|, and no float32
evaluation can reach a relative bar there.

``blend_abs`` returns, per Gaussian and field, A = sum_p |term| with every
sum INSIDE a term also replaced by the sum of its absolute values (the
running-error form of the bound): dL/dalpha is bounded by
    sum_c |dL/dC_c| (T_g c_g + S_g / (1 - alpha_g)),
S_g = sum_{i > g} w_i c_i + T_final bg the colour behind g (all colours and
the background are >= 0), and dalpha/dtheta by the absolute values of its
two eigen-frame parts (d = p - mu, a = isx (ux dx + uy dy), b = isy (-uy dx
+ ux dy), alpha = o exp(-(a^2 + b^2) / 2)):
    mx: alpha (|a| isx |ux| + |b| isy |uy|)   my: alpha (|a| isx |uy| + |b| isy |ux|)
    ux: alpha (|a| isx |dx| + |b| isy |dy|)   uy: alpha (|a| isx |dy| + |b| isy |dx|)
    isx: alpha a^2 / isx    isy: alpha b^2 / isy    o: alpha / o.
Pixels past their stop point, Gaussians skipped (alpha < 1/255) or clamped
(alpha = 0.99, where dalpha/dtheta = 0) contribute nothing, as in the
definition.

``sample_abs_vjp`` carries such per-field scales through the sampling of
Section 3.3: sum over a curve's Gaussians and fields of
|d table[g, k] / d curve parameter| * scale[g, k], with the Jacobian entries
taken exactly by forward-mode differentiation of ``curves.gaussian_table``.
"""

from __future__ import annotations

import torch

from .curves import SampleCfg, gaussian_table
from .raster import ALPHA_MAX, ALPHA_MIN, GRAD_KEYS, T_MIN

F64 = torch.float64
GEOM_KEYS = ("mx", "my", "ux", "uy", "isx", "isy", "o")


def blend_abs(tab: dict, xs, ys, dC, bg=(0.0, 0.0, 0.0), chunk: int = 1 << 20) -> dict:
    """Per field of GRAD_KEYS, sum over the pixels (xs[i], ys[i]) of the
    absolute per-pixel terms of the blend's gradient (see the module
    docstring).  dC [n, 3] is dL/dC at those pixels.  [Ng] per field, the
    colour [Ng, 3]."""
    xs = torch.as_tensor(xs, dtype=F64)
    ys = torch.as_tensor(ys, dtype=F64)
    dC = torch.as_tensor(dC, dtype=F64)
    ng = tab["mx"].shape[0]
    out = {k: torch.zeros(ng, dtype=F64) for k in GEOM_KEYS}
    out["col"] = torch.zeros(ng, 3, dtype=F64)
    if ng == 0:
        return out
    bg_t = torch.as_tensor(bg, dtype=F64)
    col = tab["col"].detach()
    f = {k: tab[k].detach()[None, :] for k in ("mx", "my", "ux", "uy", "isx", "isy", "o")}
    step = max(1, chunk // ng)
    for s in range(0, xs.shape[0], step):
        e = min(xs.shape[0], s + step)
        n = e - s
        dx = xs[s:e, None] + 0.5 - f["mx"]
        dy = ys[s:e, None] + 0.5 - f["my"]
        a = (f["ux"] * dx + f["uy"] * dy) * f["isx"]
        b = (-f["uy"] * dx + f["ux"] * dy) * f["isy"]
        a_raw = f["o"] * torch.exp(-0.5 * (a * a + b * b))
        alpha = torch.where(a_raw >= ALPHA_MIN, torch.clamp(a_raw, max=ALPHA_MAX), torch.zeros_like(a_raw))
        one_minus = 1.0 - alpha
        T_after = torch.cumprod(one_minus, dim=1)
        T_before = torch.cat([torch.ones(n, 1, dtype=F64), T_after[:, :-1]], dim=1)
        idx = torch.arange(ng)[None, :].expand(n, -1)
        stop = (alpha > 0) & (T_after < T_MIN)
        first_stop = torch.where(stop, idx, torch.full_like(idx, ng)).min(dim=1).values
        keep = (idx < first_stop[:, None]) & (alpha > 0)
        w = torch.where(keep, alpha * T_before, torch.zeros_like(alpha))
        T_final = torch.cat([T_before, T_after[:, -1:]], dim=1).gather(1, first_stop[:, None])[:, 0]
        adC = dC[s:e].abs()
        wc = w[:, :, None] * col[None]                                     # [n, Ng, 3]
        total = wc.sum(1) + T_final[:, None] * bg_t[None, :]
        behind = total[:, None, :] - torch.cumsum(wc, dim=1)              # S_g T_{g+1}
        dl_da = (adC[:, None, :] * (T_before[:, :, None] * col[None] + behind / one_minus[:, :, None])).sum(2)
        live = keep & (a_raw < ALPHA_MAX)                                  # the clamp has no slope
        dl_da = torch.where(live, dl_da, torch.zeros_like(dl_da))
        aa, ab = a.abs(), b.abs()
        jac = dict(mx=alpha * (aa * f["isx"] * f["ux"].abs() + ab * f["isy"] * f["uy"].abs()),
                   my=alpha * (aa * f["isx"] * f["uy"].abs() + ab * f["isy"] * f["ux"].abs()),
                   ux=alpha * (aa * f["isx"] * dx.abs() + ab * f["isy"] * dy.abs()),
                   uy=alpha * (aa * f["isx"] * dy.abs() + ab * f["isy"] * dx.abs()),
                   isx=alpha * a * a / f["isx"], isy=alpha * b * b / f["isy"],
                   o=alpha / torch.clamp(f["o"], min=1e-300))
        for k, j in jac.items():
            out[k] += (dl_da * j).sum(0)
        out["col"] += torch.einsum("pc,pg->gc", adC, w)
    return out


def sample_abs_vjp(curves: dict, cfg: SampleCfg, scale: dict, first=None) -> dict:
    """Per curve parameter theta: sum over its curve's Gaussians g and the
    fields k of GRAD_KEYS of |d table[g, k] / d theta| * scale[k][g]
    (scale[k] >= 0, [Ng], the colour [Ng, 3]).  A Gaussian depends on its
    own curve only, so one forward-mode derivative per parameter slot, with
    the tangent set at that slot of every curve at once, gives every
    Gaussian's derivative with respect to its own curve's parameter; the
    slots' derivatives are taken together (torch.func.vmap over the
    tangents)."""
    keys = [k for k in curves]
    vals = tuple(curves[k].detach().to(F64) for k in keys)

    def table(*v):
        t = gaussian_table(dict(zip(keys, v)), cfg, first)
        return tuple(t[k] for k in GRAD_KEYS)

    slots = []          # (input index, slot index within a curve's row)
    for vi, v in enumerate(vals):
        if v.shape[0]:
            slots += [(vi, j) for j in range(v[0].numel())]
    out = {k: torch.zeros_like(v) for k, v in zip(keys, vals)}
    if not slots:
        return out
    tangents = []
    for vi, v in enumerate(vals):
        t = torch.zeros((len(slots),) + tuple(v.shape), dtype=F64)
        for si, (vj, j) in enumerate(slots):
            if vj == vi:
                t[si].reshape(v.shape[0], -1)[:, j] = 1.0
        tangents.append(t)
    jvps = torch.func.vmap(lambda *tt: torch.func.jvp(table, vals, tt)[1])(*tangents)
    sc = [torch.as_tensor(scale[k], dtype=F64) for k in GRAD_KEYS]
    for si, (vi, j) in enumerate(slots):
        contrib = sum((d[si].abs() * s).reshape(d.shape[1], -1).sum(1) for d, s in zip(jvps, sc))
        k = keys[vi]
        n = vals[vi].shape[0]
        # Gaussian g belongs to one curve: sum its contributions per curve
        out[k].reshape(n, -1)[:, j] = _per_curve(contrib, k, curves, cfg, first)
    return out


def _per_curve(contrib: torch.Tensor, key: str, curves: dict, cfg: SampleCfg, first) -> torch.Tensor:
    """Sum a per-Gaussian [Ng] vector over each curve of the kind of `key`
    (the curves' Gaussians are draw-ordered runs starting at first[i])."""
    n_open = curves["open_ctrl"].shape[0]
    n_closed = curves["closed_ctrl"].shape[0]
    if first is None:
        from .curves import draw_order
        _, first = draw_order(curves["open_ctrl"].detach().numpy(), curves["open_width"].detach().numpy(),
                              curves["closed_ctrl"].detach().numpy(), cfg)
    first = torch.as_tensor(first, dtype=torch.int64)
    if key.startswith("open"):
        start, per, n = first[:n_open], cfg.g_open, n_open
    else:
        start, per, n = first[n_open:n_open + n_closed], cfg.per_closed, n_closed
    idx = start[:, None] + torch.arange(per)[None, :]
    return contrib[idx.reshape(-1)].reshape(n, per).sum(1)
