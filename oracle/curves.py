"""Section 3.2-3.3: Bezier curves, Gaussians sampled on them, draw order.

TEST INFRASTRUCTURE ONLY (see the package docstring).

All geometry is fp64 torch (differentiable).  Curves are in pixel
coordinates with activated attributes:
  open curves   ctrl [No,10,2] (3 chained cubic segments, Section 3.2 / 3.3
                "open curves"), width [No], color [No,3], opac [No,3]
                (one opacity per segment, Section 3.2 and Appendix D)
  closed curves ctrl [Nc,12,2] (4 chained cubic segments, the 13th point is
                the first one again), color [Nc,3], opac [Nc] (one uniform
                opacity, Appendix D)

Readings of the paper used here (the paper is silent or garbled):
  * cubic segments (M = 3): "10 control points" for 3 chained segments fixes
    1 + 3*3 points, so the "degree of 4" of Section 3.3 counts points.
  * K samples per chain are uniform in a global parameter u_k = k/(K-1) over
    the whole chain (Eq. 3); sample k lies on segment s_k = floor(S k/(K-1))
    (clamped to S-1) at local parameter t_k = S u_k - s_k, both computed from
    integers so that the segment decision is exact.
  * closed curve = the paired structure of Section 3.3 with 2 segments per
    group: boundary A = P0..P6, boundary B = P0,P11,P10,...,P6 (the last two
    segments walked backwards); both run from P0 to P6.
  * interior rows: tau_r = (1 - cos(pi r/(R+1)))/2, r = 0..R+1, a normalized
    CDF (the arcsine law) that is dense near both boundaries (Section 3.3).
  * the rotation (Eq. 8) comes from the central neighbour difference
    (tangent_mode 0, the paper's), or from the direction of the derivative
    B'(t) of the sample's own segment (tangent_mode 1, the reading of the
    Gaussian's orientation as the curve's tangent); a closed row's
    derivative is that of its interpolated control points (Eq. 4).
  * sigma at the last sample of a row uses the previous pair; sigma_y of the
    last row uses the previous row; a zero-length neighbour vector gives
    theta = 0 (Eq. 7-8 "nearest available neighbour").
  * open curves: sigma_y = width (Section 3.3, width is the y-scale).
  * Sigma = (R S)(R S)^T + eps I (Eq. 11-12 plus a small isotropic floor eps,
    which keeps Sigma invertible when two samples coincide); a Gaussian is
    stored by R and the inverse scales of Sigma (see gaussian_table).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

F64 = torch.float64


@dataclass(frozen=True)
class SampleCfg:
    g_open: int = 16        # K, samples per open curve (Eq. 3)
    rows_closed: int = 4    # R + 2 rows per closed curve (Eq. 6)
    k_closed: int = 8       # K samples per row of a closed curve
    rho: float = 1.0        # the density constant of Eq. 7
    eps: float = 0.3        # isotropic covariance floor, px^2
    tangent_mode: int = 0   # rotation from: 0 the neighbour difference (Eq. 8), 1 the derivative B'(t)

    @property
    def per_closed(self) -> int:
        return self.rows_closed * self.k_closed


# --------------------------------------------------------------------------
# Eq. 1-2: Bernstein form
# --------------------------------------------------------------------------
def bernstein(M: int, j: int, t: torch.Tensor) -> torch.Tensor:
    """B_j^M(t) = C(M, j) (1 - t)^(M - j) t^j   (Eq. 2)."""
    return math.comb(M, j) * (1.0 - t) ** (M - j) * t ** j


def bezier(P: torch.Tensor, t: torch.Tensor) -> torch.Tensor:
    """B(t) = sum_j B_j^M(t) P_j   (Eq. 1).   P [..., M+1, 2], t [...]."""
    M = P.shape[-2] - 1
    out = torch.zeros(P.shape[:-2] + (2,), dtype=P.dtype)
    for j in range(M + 1):
        out = out + bernstein(M, j, t)[..., None] * P[..., j, :]
    return out


def bezier_derivative(P: torch.Tensor, t: torch.Tensor) -> torch.Tensor:
    """dB/dt of Eq. 1, the hodograph: M sum_{j<M} B_j^{M-1}(t) (P_{j+1} - P_j).
    P [..., M+1, 2], t [...]."""
    M = P.shape[-2] - 1
    out = torch.zeros(P.shape[:-2] + (2,), dtype=P.dtype)
    for j in range(M):
        out = out + (M * bernstein(M - 1, j, t))[..., None] * (P[..., j + 1, :] - P[..., j, :])
    return out


def chain_sample_params(K: int, S: int):
    """Segment index and local parameter of the K uniform samples on a chain
    of S cubic segments (Eq. 3 with u_k = k/(K-1) over the whole chain)."""
    if K < 2:
        raise ValueError("need at least two samples per chain")
    k = np.arange(K)
    s = np.minimum((S * k) // (K - 1), S - 1)
    t = (S * k - s * (K - 1)) / (K - 1)
    return s, t


def chain_points(ctrl: torch.Tensor, K: int) -> torch.Tensor:
    """Samples of a chain of cubic segments.  ctrl [..., 3S+1, 2] -> [..., K, 2]."""
    S = (ctrl.shape[-2] - 1) // 3
    s, t = chain_sample_params(K, S)
    pts = []
    for k in range(K):
        seg = ctrl[..., 3 * s[k]: 3 * s[k] + 4, :]
        tk = torch.full(seg.shape[:-2], float(t[k]), dtype=ctrl.dtype)
        pts.append(bezier(seg, tk))
    return torch.stack(pts, dim=-2)


def chain_tangents(ctrl: torch.Tensor, K: int) -> torch.Tensor:
    """The derivative of each sample's own segment at its local parameter
    (the samples of chain_points; a sample at a join belongs to the later
    segment).  ctrl [..., 3S+1, 2] -> [..., K, 2]."""
    S = (ctrl.shape[-2] - 1) // 3
    s, t = chain_sample_params(K, S)
    out = []
    for k in range(K):
        seg = ctrl[..., 3 * s[k]: 3 * s[k] + 4, :]
        tk = torch.full(seg.shape[:-2], float(t[k]), dtype=ctrl.dtype)
        out.append(bezier_derivative(seg, tk))
    return torch.stack(out, dim=-2)


# --------------------------------------------------------------------------
# Eq. 7-8 and 11-12
# --------------------------------------------------------------------------
def _norm(v: torch.Tensor) -> torch.Tensor:
    """Euclidean length with derivative 0 at the zero vector."""
    sq = (v * v).sum(-1)
    zero = sq == 0
    safe = torch.where(zero, torch.ones_like(sq), sq)
    return torch.where(zero, torch.zeros_like(sq), torch.sqrt(safe))


def _angle(v: torch.Tensor) -> torch.Tensor:
    """atan2(v_y, v_x) (Eq. 8); the zero vector has angle 0 and derivative 0."""
    zero = (v * v).sum(-1) == 0
    vx = torch.where(zero, torch.ones_like(v[..., 0]), v[..., 0])
    vy = torch.where(zero, torch.zeros_like(v[..., 1]), v[..., 1])
    return torch.where(zero, torch.zeros_like(vx), torch.atan2(vy, vx))


def along_row(X: torch.Tensor, rho: float, tangents: torch.Tensor = None):
    """sigma_x (Eq. 7, first line) and theta (Eq. 8) for samples X [..., K, 2]
    ordered along a curve.  With `tangents` given (tangent_mode 1, the
    reading of the rotation as the direction of B'(t)), theta is their angle
    instead of the neighbour difference's."""
    nxt = X[..., 1:, :] - X[..., :-1, :]                   # X_{k+1} - X_k
    sx_vec = torch.cat([nxt, nxt[..., -1:, :]], dim=-2)    # last uses (K-2, K-1)
    sigma_x = _norm(sx_vec) / rho
    if tangents is not None:
        return sigma_x, _angle(tangents)
    if X.shape[-2] >= 3:
        central = X[..., 2:, :] - X[..., :-2, :]           # X_{k+1} - X_{k-1}
        tang = torch.cat([nxt[..., :1, :], central, nxt[..., -1:, :]], dim=-2)
    else:
        tang = torch.cat([nxt, nxt], dim=-2)
    theta = _angle(tang)
    return sigma_x, theta


def covariance(theta, sigma_x, sigma_y, eps: float):
    """Sigma = (R S)(R S)^T + eps I with R the rotation by theta and
    S = diag(sigma_x, sigma_y)   (Eq. 11-12).   Returns [..., 2, 2]."""
    c, s = torch.cos(theta), torch.sin(theta)
    R = torch.stack([torch.stack([c, -s], -1), torch.stack([s, c], -1)], -2)
    zero = torch.zeros_like(sigma_x)
    S = torch.stack([torch.stack([sigma_x, zero], -1),
                     torch.stack([zero, sigma_y], -1)], -2)
    RS = R @ S
    eye = torch.eye(2, dtype=theta.dtype)
    return RS @ RS.transpose(-1, -2) + eps * eye


# --------------------------------------------------------------------------
# Section 3.3: open and closed curves
# --------------------------------------------------------------------------
def sample_open(ctrl, width, color, opac, cfg: SampleCfg):
    """Gaussians on open curves, [No, K] per field (Section 3.3)."""
    K = cfg.g_open
    X = chain_points(ctrl, K)                                  # [No, K, 2]
    sigma_x, theta = along_row(X, cfg.rho, chain_tangents(ctrl, K) if cfg.tangent_mode == 1 else None)
    sigma_y = width[:, None].expand(-1, K)
    seg, _ = chain_sample_params(K, 3)
    o = opac[:, torch.as_tensor(seg)]                          # per-segment opacity
    col = color[:, None, :].expand(-1, K, -1)
    return dict(mu=X, sigma_x=sigma_x, sigma_y=sigma_y, theta=theta, o=o, col=col)


def closed_boundaries(ctrl):
    """The two boundary groups of the paired structure (Section 3.3): both
    start at P0 and end at P6.  ctrl [Nc,12,2] -> A, B [Nc,7,2]."""
    A = ctrl[:, 0:7]
    B = torch.cat([ctrl[:, 0:1], ctrl[:, [11, 10, 9, 8, 7, 6]]], dim=1)
    return A, B


def closed_tau(rows: int) -> torch.Tensor:
    """Interpolation weights t_k of the interior rows (Section 3.3), the
    arcsine CDF at uniform steps; rows = R + 2 including both boundaries."""
    r = torch.arange(rows, dtype=F64)
    return (1.0 - torch.cos(math.pi * r / (rows - 1))) / 2.0


def sample_closed(ctrl, color, opac, cfg: SampleCfg, color2=None, opac2=None):
    """Gaussians filling closed curves, [Nc, R+2, K] per field (Eq. 4-8).

    Linear-gradient fills (Appendix D; reading): with color2 / opac2 given,
    sample k of every row takes x0 + u (x1 - x0), u = k / (K - 1), from the
    value x0 at P0 to x1 at P6, the two ends of both boundaries."""
    rows, K = cfg.rows_closed, cfg.k_closed
    A, B = closed_boundaries(ctrl)
    tau = closed_tau(rows)[None, :, None, None]
    Q = (1.0 - tau) * A[:, None] + tau * B[:, None]            # Eq. 4: [Nc, rows, 7, 2]
    X = chain_points(Q, K)                                     # Eq. 5-6: [Nc, rows, K, 2]
    sigma_x, theta = along_row(X, cfg.rho, chain_tangents(Q, K) if cfg.tangent_mode == 1 else None)
    nxt = X[:, 1:] - X[:, :-1]                                 # X_{r+1,k} - X_{r,k}
    sy_vec = torch.cat([nxt, nxt[:, -1:]], dim=1)              # last row uses (R, R+1)
    sigma_y = _norm(sy_vec) / cfg.rho                          # Eq. 7, second line
    u = torch.arange(K, dtype=F64) / (K - 1)
    if opac2 is None:
        o = opac[:, None, None].expand(-1, rows, K)
    else:
        o = (opac[:, None] + u[None, :] * (opac2 - opac)[:, None])[:, None, :].expand(-1, rows, K)
    if color2 is None:
        col = color[:, None, None, :].expand(-1, rows, K, -1)
    else:
        col = (color[:, None, :] + u[None, :, None] * (color2 - color)[:, None, :])[:, None].expand(-1, rows, K, -1)
    return dict(mu=X, sigma_x=sigma_x, sigma_y=sigma_y, theta=theta, o=o, col=col)


# --------------------------------------------------------------------------
# Section 3.3 "depth ... based on the area of curves" (float32, decides ranks)
# --------------------------------------------------------------------------
def area_keys_f32(open_ctrl, open_width, closed_ctrl) -> np.ndarray:
    """Depth key per curve in float32, each operation rounded in order.

    Reading: a closed curve's area is half the absolute shoelace sum of its
    12-point control polygon; an open curve's area is the length of its
    10-point control polygon times its width.  Open curves come first in the
    index space.
    """
    f = np.float32
    oc = np.asarray(open_ctrl, dtype=f).reshape(-1, 10, 2)
    ow = np.asarray(open_width, dtype=f).reshape(-1)
    cc = np.asarray(closed_ctrl, dtype=f).reshape(-1, 12, 2)
    keys_open = np.zeros(oc.shape[0], dtype=f)
    for j in range(9):
        dx = oc[:, j + 1, 0] - oc[:, j, 0]
        dy = oc[:, j + 1, 1] - oc[:, j, 1]
        keys_open = keys_open + np.sqrt(dx * dx + dy * dy)
    keys_open = keys_open * ow
    acc = np.zeros(cc.shape[0], dtype=f)
    for j in range(12):
        jn = (j + 1) % 12
        cross = cc[:, j, 0] * cc[:, jn, 1] - cc[:, jn, 0] * cc[:, j, 1]
        acc = acc + cross
    keys_closed = np.abs(acc) * f(0.5)
    return np.concatenate([keys_open, keys_closed]).astype(f)


def draw_order(open_ctrl, open_width, closed_ctrl, cfg: SampleCfg):
    """rank[i] (0 = front-most) and first[i], the index of curve i's first
    Gaussian in the draw-ordered table: curves sorted by ascending area so a
    small curve is never hidden behind a large one (Section 3.3); equal keys
    keep the lower curve index in front."""
    keys = area_keys_f32(open_ctrl, open_width, closed_ctrl)
    n_open = np.asarray(open_width).reshape(-1).shape[0]
    order = np.argsort(keys, kind="stable")
    rank = np.empty(keys.shape[0], dtype=np.int64)
    rank[order] = np.arange(keys.shape[0])
    count = np.where(np.arange(keys.shape[0]) < n_open, cfg.g_open, cfg.per_closed)
    first_by_rank = np.concatenate([[0], np.cumsum(count[order])[:-1]]).astype(np.int64)
    first = first_by_rank[rank]
    return rank, first


# --------------------------------------------------------------------------
# The Gaussian table (draw order)
# --------------------------------------------------------------------------
ALPHA_MIN = 1.0 / 255.0     # Gaussians with alpha below this are skipped
EXT_PAD = 0.01              # px added to the support half-extents


def gaussian_table(curves: dict, cfg: SampleCfg, first=None):
    """All Gaussians in draw order as a dict of fp64 tensors [Ng] (colour
    [Ng,3]).

    Each Gaussian is kept in the eigen-frame of Eq. 11-12: with the eps
    floor, Sigma = (R S)(R S)^T + eps I = R diag(sx^2 + eps, sy^2 + eps) R^T,
    so Sigma^-1 = R diag(isx^2, isy^2) R^T with
        R = [[ux, -uy], [uy, ux]],  (ux, uy) = (cos theta, sin theta),
        isx = (sx^2 + eps)^-1/2,    isy = (sy^2 + eps)^-1/2.
    Fields: mx, my, ux, uy, isx, isy, o, col, ext_x, ext_y, and for
    inspection sigma_x, sigma_y, theta, Sigma.

    ext_x/ext_y are the half extents of the axis-aligned box around the
    ellipse where alpha >= 1/255, i.e. 0.5 d^T Sigma^-1 d <= ln(255 o):
    sqrt(2 ln(255 o) Sigma_xx) (resp. yy) plus EXT_PAD px; -1 when o < 1/255
    (the Gaussian can never reach the threshold)."""
    oc, ow = curves["open_ctrl"], curves["open_width"]
    cc = curves["closed_ctrl"]
    if first is None:
        _, first = draw_order(oc.detach().numpy(), ow.detach().numpy(),
                              cc.detach().numpy(), cfg)
    parts = []
    n_open = oc.shape[0]
    if n_open:
        so = sample_open(oc, ow, curves["open_color"], curves["open_opac"], cfg)
        parts.append((so, cfg.g_open, 0))
    if cc.shape[0]:
        sc = sample_closed(cc, curves["closed_color"], curves["closed_opac"], cfg,
                           curves.get("closed_color2"), curves.get("closed_opac2"))
        sc = {k: v.reshape((v.shape[0], -1) + tuple(v.shape[3:])) for k, v in sc.items()}
        parts.append((sc, cfg.per_closed, n_open))
    n_g = n_open * cfg.g_open + cc.shape[0] * cfg.per_closed
    # destination index of every sampled Gaussian
    fields = {}
    idx_all = []
    for samp, per, base in parts:
        n = samp["o"].shape[0]
        idx = torch.as_tensor(first[base: base + n])[:, None] + torch.arange(per)[None, :]
        idx_all.append(idx.reshape(-1))
        for k, v in samp.items():
            fields.setdefault(k, []).append(v.reshape((n * per,) + tuple(v.shape[2:])))
    if not idx_all:
        z = torch.zeros(0, dtype=F64)
        return dict(mx=z, my=z, ux=z, uy=z, isx=z, isy=z, o=z, col=torch.zeros(0, 3, dtype=F64),
                    ext_x=z, ext_y=z, sigma_x=z, sigma_y=z, theta=z, Sigma=torch.zeros(0, 2, 2, dtype=F64))
    idx = torch.cat(idx_all)
    inv = torch.empty(n_g, dtype=torch.int64)
    inv[idx] = torch.arange(n_g)
    g = {k: torch.cat(v)[inv] for k, v in fields.items()}

    Sigma = covariance(g["theta"], g["sigma_x"], g["sigma_y"], cfg.eps)
    out = dict(mx=g["mu"][:, 0], my=g["mu"][:, 1],
               ux=torch.cos(g["theta"]), uy=torch.sin(g["theta"]),
               isx=(g["sigma_x"] ** 2 + cfg.eps) ** -0.5, isy=(g["sigma_y"] ** 2 + cfg.eps) ** -0.5,
               o=g["o"], col=g["col"], sigma_x=g["sigma_x"], sigma_y=g["sigma_y"],
               theta=g["theta"], Sigma=Sigma)
    with torch.no_grad():
        o = g["o"]
        ok = o >= ALPHA_MIN
        L = torch.log(torch.clamp(255.0 * o, min=1.0))
        ext_x = torch.sqrt(2.0 * L * Sigma[:, 0, 0]) + EXT_PAD
        ext_y = torch.sqrt(2.0 * L * Sigma[:, 1, 1]) + EXT_PAD
        out["ext_x"] = torch.where(ok, ext_x, torch.full_like(ext_x, -1.0))
        out["ext_y"] = torch.where(ok, ext_y, torch.full_like(ext_y, -1.0))
    return out


TABLE_FIELDS = 12
RECORD = ("mx", "my", "ux", "uy", "isx", "isy", "o", "r", "g", "b", "ext_x", "ext_y")


def table_to_f32(tab: dict) -> np.ndarray:
    """Pack a table into the float32 record of the CUDA library,
    [Ng, 12] = mx, my, ux, uy, isx, isy, o, r, g, b, ext_x, ext_y."""
    n = tab["mx"].shape[0]
    rec = np.zeros((n, TABLE_FIELDS), dtype=np.float32)
    cols = [tab["mx"], tab["my"], tab["ux"], tab["uy"], tab["isx"], tab["isy"], tab["o"],
            tab["col"][:, 0], tab["col"][:, 1], tab["col"][:, 2], tab["ext_x"], tab["ext_y"]]
    for i, c in enumerate(cols):
        rec[:, i] = c.detach().numpy().astype(np.float32)
    return rec


def table_from_f32(rec: np.ndarray) -> dict:
    """The inverse of table_to_f32, as fp64 tensors (exact)."""
    r = torch.as_tensor(np.asarray(rec, dtype=np.float32).astype(np.float64))
    return dict(mx=r[:, 0], my=r[:, 1], ux=r[:, 2], uy=r[:, 3], isx=r[:, 4], isy=r[:, 5],
                o=r[:, 6], col=r[:, 7:10], ext_x=r[:, 10], ext_y=r[:, 11])
