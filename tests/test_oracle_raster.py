"""Pins of the oracle's blending (Section 3.4, Eq. 9-10): a Gaussian density
from scipy, a sequential pure-Python restatement, invariants, and the
rotation symmetry of the whole sample + render chain."""

import math

import numpy as np
import pytest
import torch
from scipy.stats import multivariate_normal

import oracle
from oracle.curves import SampleCfg, table_from_f32
from oracle.raster import ALPHA_MAX, ALPHA_MIN, T_MIN

F64 = torch.float64


def _table(mx, my, Sig, o, col):
    """A table from covariances: R and the inverse scales from eigh."""
    Sig = np.asarray(Sig, dtype=np.float64)
    w, v = np.linalg.eigh(Sig)
    t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64))
    return dict(mx=t(mx), my=t(my), ux=t(v[:, 0, 0]), uy=t(v[:, 1, 0]), isx=t(w[:, 0] ** -0.5),
                isy=t(w[:, 1] ** -0.5), o=t(o), col=t(col), Sig=Sig)


def test_single_rotated_gaussian_matches_density_ratio():
    """alpha = o * pdf(p)/pdf(mu) of N(mu, Sigma) (scipy), one Gaussian."""
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    Sig = R @ np.diag([9.0, 1.5]) @ R.T
    mu = np.array([7.3, 5.1])
    o, col, bg = 0.8, np.array([0.2, 0.5, 0.9]), np.array([0.1, 0.0, 0.3])
    tab = _table([mu[0]], [mu[1]], Sig[None], [o], col[None])
    out = oracle.render_image(tab, 16, 12, bg=tuple(bg))
    rv = multivariate_normal(mu, Sig)
    peak = rv.pdf(mu)
    ys, xs = np.mgrid[0:12, 0:16]
    a = o * rv.pdf(np.stack([xs + 0.5, ys + 0.5], -1)) / peak
    a = np.where(a >= 1 / 255, np.minimum(a, 0.99), 0.0)
    exp = col[:, None, None] * a[None] + (1 - a)[None] * bg[:, None, None]
    assert np.allclose(out["img"].numpy(), exp, atol=1e-12)
    assert np.allclose(out["T"].numpy(), 1 - a, atol=1e-12)


def sequential_blend(tab, x, y, bg):
    """The blend written as the sequential per-pixel loop of a tile
    rasterizer, one Gaussian at a time, with the same three thresholds."""
    C = np.zeros(3)
    T = 1.0
    last = -1
    px, py = x + 0.5, y + 0.5
    for i in range(tab["mx"].shape[0]):
        d = np.array([px - float(tab["mx"][i]), py - float(tab["my"][i])])
        q = d @ np.linalg.solve(tab["Sig"][i], d)
        a = min(0.99, float(tab["o"][i]) * math.exp(-0.5 * q))
        if a < 1 / 255:
            continue
        Tn = T * (1 - a)
        if Tn < 1e-4:
            break
        C += tab["col"][i].numpy() * a * T
        T = Tn
        last = i
    return C + T * np.asarray(bg), T, last


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_scan_form_equals_sequential_loop(seed):
    rng = np.random.default_rng(seed)
    n = 60
    W, H = 12, 10
    th = rng.uniform(0, np.pi, n)
    s1, s2 = rng.uniform(0.5, 6, n), rng.uniform(0.5, 6, n)
    Sig = np.zeros((n, 2, 2))
    for i in range(n):
        R = np.array([[math.cos(th[i]), -math.sin(th[i])], [math.sin(th[i]), math.cos(th[i])]])
        Sig[i] = R @ np.diag([s1[i] ** 2, s2[i] ** 2]) @ R.T
    o = rng.uniform(0.05, 1.0, n)
    o[::7] = 1.0                       # some alphas hit the 0.99 clamp
    tab = _table(rng.uniform(-3, W + 3, n), rng.uniform(-3, H + 3, n), Sig, o, rng.uniform(0, 1, (n, 3)))
    bg = (0.3, 0.6, 0.1)
    out = oracle.render_image(tab, W, H, bg=bg)
    stops = 0
    for y in range(H):
        for x in range(W):
            C, T, last = sequential_blend(tab, x, y, bg)
            assert np.allclose(out["img"][:, y, x].numpy(), C, atol=1e-12)
            assert abs(float(out["T"][y, x]) - T) < 1e-12
            assert int(out["last"][y, x]) == last
            stops += T * (1 - 0.99) < 1e-4
    assert stops > 0                   # the stop rule was exercised


def test_transmittance_invariants():
    rng = np.random.default_rng(7)
    n = 200
    Sig = np.tile(np.diag([4.0, 4.0]), (n, 1, 1))
    tab = _table(rng.uniform(0, 8, n), rng.uniform(0, 8, n), Sig, rng.uniform(0.1, 1, n),
                 rng.uniform(0, 1, (n, 3)))
    xs = torch.arange(8, dtype=F64).repeat(8)
    ys = torch.arange(8, dtype=F64).repeat_interleave(8)
    r = oracle.render_pixels(tab, xs, ys)
    T = r["T"]
    assert torch.all(T >= T_MIN * (1 - ALPHA_MAX) - 1e-15) and torch.all(T <= 1)
    # per pixel, transmittance along the draw order never increases
    dx = 0.5 + xs[:, None] - tab["mx"][None]
    dy = 0.5 + ys[:, None] - tab["my"][None]
    a = tab["o"][None] * torch.exp(-0.5 * (dx * dx + dy * dy) / 4.0)
    a = torch.where(a >= ALPHA_MIN, torch.clamp(a, max=ALPHA_MAX), torch.zeros_like(a))
    Tcum = torch.cumprod(1 - a, 1)
    assert torch.all(Tcum[:, 1:] <= Tcum[:, :-1] + 1e-15)
    # colour is a convex combination when bg = 0 and colours are in [0,1]
    assert torch.all(r["C"] >= 0) and torch.all(r["C"] <= 1 + 1e-12)


def test_zero_opacity_gives_background():
    rng = np.random.default_rng(8)
    n = 30
    tab = _table(rng.uniform(0, 8, n), rng.uniform(0, 8, n), np.tile(np.eye(2) * 5, (n, 1, 1)),
                 np.zeros(n), rng.uniform(0, 1, (n, 3)))
    out = oracle.render_image(tab, 8, 8, bg=(0.25, 0.5, 0.75))
    assert torch.allclose(out["img"], torch.tensor([0.25, 0.5, 0.75], dtype=F64)[:, None, None].expand(3, 8, 8))
    assert torch.all(out["last"] == -1)


def test_front_gaussian_occludes():
    """Two opaque coincident Gaussians: the first in draw order wins."""
    Sig = np.tile(np.eye(2) * 100.0, (2, 1, 1))
    tab = _table([4, 4], [4, 4], Sig, [1.0, 1.0], [[1, 0, 0], [0, 0, 1]])
    out = oracle.render_image(tab, 8, 8)
    c = out["img"][:, 4, 4].numpy()
    # centre pixel: alpha_0 = 0.99 * exp(-small); second sees T = 1 - alpha_0
    assert c[0] > 0.98 and c[2] < 0.02
    assert np.isclose(c[0] + c[2] + float(out["T"][4, 4]), 1.0, atol=1e-12)


def _rot90_curves(curves, W):
    """Rotate the scene by 90 degrees: (x, y) -> (y, W - x)."""
    out = dict(curves)
    for k in ("open_ctrl", "closed_ctrl"):
        P = curves[k]
        out[k] = torch.stack([P[..., 1], W - P[..., 0]], -1)
    return out


def test_rotation_symmetry_of_sample_and_render():
    """Rotating the control points by 90 degrees rotates the image: catches
    swapped axes, transposed conics and sign errors in the off-diagonal."""
    from paper_2503_16424_gb300 import synth
    W = 24
    c = synth.make_curves(11, W, W, 3, 2, style="local")
    curves = {k: torch.as_tensor(v, dtype=F64) for k, v in c.as_dict().items()}
    cfg = SampleCfg(g_open=8, rows_closed=4, k_closed=5)
    tab = oracle.gaussian_table(curves, cfg)
    tab_r = oracle.gaussian_table(_rot90_curves(curves, W), cfg)
    img = oracle.render_image(tab, W, W, bg=(0.1, 0.2, 0.3))["img"].numpy()
    img_r = oracle.render_image(tab_r, W, W, bg=(0.1, 0.2, 0.3))["img"].numpy()
    # pixel (x, y) -> (y, W-1-x): img_r[:, W-1-x, y] = img[:, y, x]
    exp = np.rot90(img, k=1, axes=(1, 2))
    assert np.abs(img).max() > 0.1
    assert np.allclose(img_r, exp, atol=1e-9)


def test_render_of_f32_table_roundtrip():
    rec = np.random.default_rng(9).uniform(0, 1, (5, 12)).astype(np.float32)
    t = table_from_f32(rec)
    assert t["mx"].dtype == F64 and np.array_equal(t["col"].numpy().astype(np.float32), rec[:, 7:10])


def test_two_gaussians_at_a_pixel_closed_form():
    """Two Gaussians over one pixel: C = c1 a1 + c2 a2 (1 - a1) + bg (1 - a1)
    (1 - a2), T = (1 - a1)(1 - a2), with a_i = o_i exp(-d^T Sigma_i^-1 d / 2)
    written out from the densities (Eq. 9-10), both above 1/255 and below
    the clamp."""
    S1 = np.array([[6.0, 1.5], [1.5, 3.0]])
    S2 = np.array([[2.0, -0.4], [-0.4, 5.0]])
    mu = np.array([[3.2, 2.9], [4.1, 3.6]])
    o = np.array([0.7, 0.55])
    col = np.array([[0.9, 0.1, 0.2], [0.2, 0.6, 0.95]])
    bg = np.array([0.05, 0.3, 0.7])
    tab = _table(mu[:, 0], mu[:, 1], np.stack([S1, S2]), o, col)
    px, py = 3.5, 3.5
    a = [o[i] * math.exp(-0.5 * (np.array([px, py]) - mu[i]) @ np.linalg.solve(S, np.array([px, py]) - mu[i]))
         for i, S in enumerate((S1, S2))]
    assert all(1 / 255 < x < 0.99 for x in a)
    exp_C = col[0] * a[0] + col[1] * a[1] * (1 - a[0]) + bg * (1 - a[0]) * (1 - a[1])
    r = oracle.render_pixels(tab, torch.tensor([3.0], dtype=F64), torch.tensor([3.0], dtype=F64), bg=tuple(bg))
    assert np.allclose(r["C"][0].numpy(), exp_C, atol=1e-13)
    assert abs(float(r["T"][0]) - (1 - a[0]) * (1 - a[1])) < 1e-13


def test_clamp_bounds_the_transmittance_below():
    """n opaque coincident Gaussians: each alpha is clamped to 0.99, so
    before the stop rule T falls by 0.01 per Gaussian, and the pixel stops
    at the Gaussian that would take T below 1e-4: T_final = 0.01^2."""
    n = 5
    tab = _table([4.0] * n, [4.0] * n, np.tile(np.eye(2) * 50.0, (n, 1, 1)), [1.0] * n, np.ones((n, 3)))
    r = oracle.render_pixels(tab, torch.tensor([3.5], dtype=F64), torch.tensor([3.5], dtype=F64))
    # centre pixel (4, 4) is at the mean: alpha = min(0.99, 1) = 0.99
    assert abs(float(r["T"][0]) - 0.01 ** 2) < 1e-15
    assert int(r["last"][0]) == 1
