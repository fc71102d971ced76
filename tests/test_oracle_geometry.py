"""Pins of the oracle's curve geometry (Section 3.2-3.3, Eq. 1-8, 11-12)
against textbook algorithms, closed forms and invariants."""

import math

import numpy as np
import pytest
import torch

import oracle
from oracle.curves import SampleCfg, chain_points

F64 = torch.float64


def de_casteljau(P, t):
    """Textbook de Casteljau evaluation (repeated linear interpolation)."""
    pts = [P[..., j, :] for j in range(P.shape[-2])]
    while len(pts) > 1:
        pts = [(1 - t)[..., None] * a + t[..., None] * b for a, b in zip(pts[:-1], pts[1:])]
    return pts[0]


def test_bernstein_equals_de_casteljau():
    g = torch.Generator().manual_seed(0)
    for M in (1, 2, 3, 5):
        P = torch.rand(50, M + 1, 2, generator=g, dtype=F64) * 300
        t = torch.rand(50, generator=g, dtype=F64)
        assert torch.allclose(oracle.bezier(P, t), de_casteljau(P, t), atol=1e-12, rtol=0)


def test_bezier_endpoints_exact():
    g = torch.Generator().manual_seed(1)
    P = torch.rand(20, 4, 2, generator=g, dtype=F64) * 1000
    assert torch.equal(oracle.bezier(P, torch.zeros(20, dtype=F64)), P[:, 0])
    assert torch.equal(oracle.bezier(P, torch.ones(20, dtype=F64)), P[:, 3])


def test_bernstein_partition_of_unity():
    t = torch.linspace(0, 1, 101, dtype=F64)
    s = sum(oracle.bernstein(3, j, t) for j in range(4))
    assert torch.allclose(s, torch.ones_like(t), atol=1e-15)


def test_chain_params_cover_segments_and_joins():
    s, t = oracle.chain_sample_params(16, 3)
    assert s[0] == 0 and t[0] == 0 and s[-1] == 2 and t[-1] == 1
    assert np.all(np.diff(s) >= 0) and np.all((t >= 0) & (t <= 1))
    # u_k = (s_k + t_k)/3 is uniform
    assert np.allclose((s + t) / 3, np.arange(16) / 15, atol=1e-15)
    with pytest.raises(ValueError):
        oracle.chain_sample_params(1, 3)


def _line_curve(p0, p1, n_pts):
    j = torch.arange(n_pts, dtype=F64)[:, None] / (n_pts - 1)
    return torch.as_tensor(p0, dtype=F64) + j * (torch.as_tensor(p1, dtype=F64) - torch.as_tensor(p0, dtype=F64))


@pytest.mark.parametrize("K", [2, 5, 16, 33])
def test_open_straight_line_closed_form(K):
    """Evenly spaced collinear control points: every cubic segment is a
    constant-speed line, so samples are evenly spaced, sigma_x = L/((K-1) rho),
    theta is the line's angle and sigma_y is the width."""
    p0, p1 = (10.0, 20.0), (130.0, 70.0)
    ctrl = _line_curve(p0, p1, 10)[None]
    rho = 1.7
    cfg = SampleCfg(g_open=K, rho=rho)
    out = oracle.sample_open(ctrl, torch.tensor([2.5], dtype=F64), torch.zeros(1, 3, dtype=F64),
                             torch.tensor([[0.2, 0.5, 0.9]], dtype=F64), cfg)
    L = math.hypot(p1[0] - p0[0], p1[1] - p0[1])
    u = np.arange(K) / (K - 1)
    exp_mu = np.array(p0)[None] + u[:, None] * (np.array(p1) - np.array(p0))[None]
    assert np.allclose(out["mu"][0].numpy(), exp_mu, atol=1e-10)
    assert np.allclose(out["sigma_x"][0].numpy(), L / ((K - 1) * rho), atol=1e-10)
    assert np.allclose(out["theta"][0].numpy(), math.atan2(50, 120), atol=1e-12)
    assert np.allclose(out["sigma_y"][0].numpy(), 2.5)
    # per-segment opacity follows the segment of each sample
    seg = np.minimum((3 * np.arange(K)) // (K - 1), 2)
    assert np.allclose(out["o"][0].numpy(), np.array([0.2, 0.5, 0.9])[seg])


def test_covariance_eigen_structure():
    """Eq. 11-12: Sigma - eps I has eigenvalues sigma_x^2, sigma_y^2 with the
    sigma_x axis along (cos theta, sin theta)."""
    g = torch.Generator().manual_seed(3)
    th = (torch.rand(40, generator=g, dtype=F64) - 0.5) * 2 * math.pi
    sx = torch.rand(40, generator=g, dtype=F64) * 5 + 2.0
    sy = torch.rand(40, generator=g, dtype=F64) * 1.5 + 0.1
    eps = 0.3
    S = oracle.covariance(th, sx, sy, eps).numpy()
    for i in range(40):
        w, v = np.linalg.eigh(S[i] - eps * np.eye(2))
        assert np.allclose(sorted(w), sorted([sy[i] ** 2, sx[i] ** 2]), rtol=1e-12)
        major = v[:, np.argmax(w)]
        assert abs(abs(major @ [math.cos(th[i]), math.sin(th[i])]) - 1) < 1e-10


def _closed_from_boundaries(A, B):
    """12 stored points from boundary A (P0..P6) and B (P0, P11..P6)."""
    ctrl = torch.zeros(12, 2, dtype=F64)
    ctrl[0:7] = A
    for j, idx in enumerate([11, 10, 9, 8, 7]):
        ctrl[idx] = B[j + 1]
    assert torch.equal(B[0], A[0]) and torch.equal(B[6], A[6])
    return ctrl


def test_closed_boundaries_order():
    ctrl = torch.arange(24, dtype=F64).reshape(1, 12, 2)
    A, B = oracle.closed_boundaries(ctrl)
    assert A[0, :, 0].tolist() == [0, 2, 4, 6, 8, 10, 12]
    assert B[0, :, 0].tolist() == [0, 22, 20, 18, 16, 14, 12]


def test_closed_coinciding_boundaries_give_equal_rows():
    g = torch.Generator().manual_seed(4)
    A = torch.rand(7, 2, generator=g, dtype=F64) * 100
    ctrl = _closed_from_boundaries(A, A.clone())[None]
    cfg = SampleCfg(rows_closed=6, k_closed=9)
    out = oracle.sample_closed(ctrl, torch.rand(1, 3, dtype=F64), torch.tensor([0.7], dtype=F64), cfg)
    X = out["mu"][0]
    assert torch.allclose(X, X[0:1].expand_as(X), atol=1e-12)
    assert torch.allclose(out["sigma_y"], torch.zeros_like(out["sigma_y"]))


def test_closed_rows_interpolate_between_boundaries():
    """Boundary A on y=0, boundary B with the same x and a bulge in y: the
    row r is B scaled by tau_r in y (interpolation of control points, Eq. 4,
    is interpolation of the curves, Eq. 5)."""
    x = torch.arange(7, dtype=F64) * 10
    A = torch.stack([x, torch.zeros(7, dtype=F64)], -1)
    B = torch.stack([x, torch.tensor([0, 30, 30, 30, 30, 30, 0], dtype=F64)], -1)
    ctrl = _closed_from_boundaries(A, B)[None]
    rows, K = 7, 11
    cfg = SampleCfg(rows_closed=rows, k_closed=K, rho=1.0)
    out = oracle.sample_closed(ctrl, torch.rand(1, 3, dtype=F64), torch.tensor([0.7], dtype=F64), cfg)
    X = out["mu"][0]                                           # [rows, K, 2]
    tau = oracle.closed_tau(rows)
    u = torch.arange(K, dtype=F64) / (K - 1)
    assert torch.allclose(X[:, :, 0], (60 * u)[None].expand(rows, K), atol=1e-10)
    yB = X[-1, :, 1]
    assert torch.allclose(X[:, :, 1], tau[:, None] * yB[None], atol=1e-10)
    # sigma_y is the distance to the next row (Eq. 7), last row uses the previous
    dy = (tau[1:] - tau[:-1])[:, None] * yB[None]
    exp = torch.cat([dy, dy[-1:]], 0).abs()
    assert torch.allclose(out["sigma_y"][0], exp, atol=1e-10)


def test_closed_tau_is_normalized_cdf_dense_at_boundaries():
    for rows in (3, 4, 8, 22):
        tau = oracle.closed_tau(rows).numpy()
        assert tau[0] == 0 and abs(tau[-1] - 1) < 1e-15
        assert np.all(np.diff(tau) > 0)
        assert np.allclose(tau + tau[::-1], 1.0, atol=1e-15)
        if rows >= 4:
            d = np.diff(tau)
            assert d[0] < d[len(d) // 2] and d[-1] < d[len(d) // 2]


def test_area_keys_closed_forms():
    # regular 12-gon of circumradius r has area 3 r^2
    r = 16.0
    ang = 2 * np.pi * np.arange(12) / 12
    poly = np.stack([100 + r * np.cos(ang), 50 + r * np.sin(ang)], -1)[None]
    line = np.stack([np.linspace(0, 90, 10), np.linspace(0, 120, 10)], -1)[None]
    keys = oracle.area_keys_f32(line, np.array([2.0]), poly)
    assert keys.dtype == np.float32
    assert abs(keys[0] - 150.0 * 2.0) < 1e-3       # length 150 x width 2
    assert abs(keys[1] - 3 * r * r) < 1e-2
    # orientation does not matter
    keys_rev = oracle.area_keys_f32(line[:, ::-1], np.array([2.0]), poly[:, ::-1])
    assert abs(keys_rev[1] - keys[1]) < 1e-2


def test_draw_order_nested_squares():
    """Squares of side 10..80 in shuffled order: the smallest is in front;
    equal keys keep the lower index in front; first[] walks the counts."""
    sides = np.array([40, 10, 80, 20, 10, 60], dtype=np.float64)
    ctrl = []
    for s in sides:
        c = np.array([[0, 0], [s, 0], [s, s], [0, s]])
        t = np.linspace(0, 1, 4)[:-1]
        pts = np.concatenate([c[i] + t[:, None] * (c[(i + 1) % 4] - c[i]) for i in range(4)])
        ctrl.append(pts)
    ctrl = np.array(ctrl)
    cfg = SampleCfg(g_open=5, rows_closed=3, k_closed=4)
    rank, first = oracle.draw_order(np.zeros((0, 10, 2)), np.zeros(0), ctrl, cfg)
    assert rank.tolist() == [3, 0, 5, 2, 1, 4]
    assert first.tolist() == [36, 0, 60, 24, 12, 48]


def test_gaussian_table_draw_order_and_extent():
    cfg = SampleCfg(g_open=6, rows_closed=3, k_closed=4)
    g = torch.Generator().manual_seed(5)
    curves = dict(open_ctrl=torch.rand(3, 10, 2, generator=g, dtype=F64) * 64,
                  open_width=torch.tensor([1.0, 2.0, 3.0], dtype=F64),
                  open_color=torch.rand(3, 3, generator=g, dtype=F64),
                  open_opac=torch.tensor([[0.5, 0.001, 0.9]] * 3, dtype=F64),
                  closed_ctrl=torch.rand(2, 12, 2, generator=g, dtype=F64) * 64,
                  closed_color=torch.rand(2, 3, generator=g, dtype=F64),
                  closed_opac=torch.tensor([0.6, 0.8], dtype=F64))
    rank, first = oracle.draw_order(curves["open_ctrl"].numpy(), curves["open_width"].numpy(),
                                    curves["closed_ctrl"].numpy(), cfg)
    tab = oracle.gaussian_table(curves, cfg, first)
    assert tab["mx"].shape[0] == 3 * 6 + 2 * 12
    # Gaussians of curve i occupy [first[i], first[i] + count)
    for i in range(3):
        so = oracle.sample_open(curves["open_ctrl"][i:i + 1], curves["open_width"][i:i + 1],
                                curves["open_color"][i:i + 1], curves["open_opac"][i:i + 1], cfg)
        sl = slice(first[i], first[i] + 6)
        assert torch.allclose(tab["mx"][sl], so["mu"][0, :, 0])
        assert torch.allclose(tab["o"][sl], so["o"][0])
    # the extent box contains the alpha >= 1/255 ellipse: check on its boundary
    Sig = tab["Sigma"].detach()
    for i in range(tab["mx"].shape[0]):
        o = float(tab["o"][i])
        if o < 1 / 255:
            assert tab["ext_x"][i] < 0
            continue
        Lth = math.log(255 * o)
        w, v = np.linalg.eigh(Sig[i].numpy())
        th = np.linspace(0, 2 * np.pi, 721)
        pts = v @ (np.sqrt(2 * Lth * w)[:, None] * np.stack([np.cos(th), np.sin(th)]))
        assert np.abs(pts[0]).max() <= float(tab["ext_x"][i]) + 1e-9
        assert np.abs(pts[1]).max() <= float(tab["ext_y"][i]) + 1e-9
        assert np.abs(pts[0]).max() >= float(tab["ext_x"][i]) - 0.011


def test_chain_points_joins_are_shared():
    g = torch.Generator().manual_seed(6)
    ctrl = torch.rand(4, 10, 2, generator=g, dtype=F64) * 100
    X = chain_points(ctrl, 7)        # u = 0, 1/6, 2/6=join, ..., 4/6=join
    assert torch.allclose(X[:, 2], ctrl[:, 3], atol=1e-12)
    assert torch.allclose(X[:, 4], ctrl[:, 6], atol=1e-12)
    assert torch.equal(X[:, 0], ctrl[:, 0])
    assert torch.allclose(X[:, 6], ctrl[:, 9], atol=1e-12)


# ---- tangent_mode 1: the rotation from the derivative B'(t) ----

def test_bezier_derivative_equals_autograd_and_central_differences():
    """The hodograph against two independent derivatives of Eq. 1: autograd
    of bezier() with respect to t, and fp64 central differences."""
    rng = np.random.default_rng(11)
    P = torch.as_tensor(rng.uniform(-50, 50, (30, 4, 2)))
    t = torch.as_tensor(rng.uniform(0.01, 0.99, 30)).requires_grad_(True)
    d = oracle.curves.bezier_derivative(P, t.detach())
    B = oracle.bezier(P, t)
    gx, = torch.autograd.grad(B[:, 0].sum(), t, retain_graph=True)
    gy, = torch.autograd.grad(B[:, 1].sum(), t)
    assert torch.allclose(d, torch.stack([gx, gy], 1), rtol=1e-12, atol=1e-10)
    h = 1e-6
    td = t.detach()
    fd = (oracle.bezier(P, td + h) - oracle.bezier(P, td - h)) / (2 * h)
    assert torch.allclose(d, fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("K", [2, 7, 16])
def test_tangent_mode_on_a_straight_line_equals_eq8(K):
    """Evenly spaced collinear points: B'(t) points along the line, so both
    modes give the line's angle, and sigma is unchanged."""
    ctrl = _line_curve((10.0, 20.0), (130.0, 70.0), 10)[None]
    args = (ctrl, torch.tensor([2.5], dtype=F64), torch.zeros(1, 3, dtype=F64), torch.tensor([[0.2, 0.5, 0.9]],
                                                                                            dtype=F64))
    a = oracle.sample_open(*args, SampleCfg(g_open=K, tangent_mode=0))
    b = oracle.sample_open(*args, SampleCfg(g_open=K, tangent_mode=1))
    assert np.allclose(b["theta"][0].numpy(), math.atan2(50, 120), atol=1e-12)
    assert torch.allclose(a["theta"], b["theta"], atol=1e-12)
    assert torch.equal(a["sigma_x"], b["sigma_x"]) and torch.equal(a["mu"], b["mu"])


def test_tangent_mode_follows_the_curve_direction():
    """On a random open curve, every sample's theta (mode 1) is the direction
    of its own segment's chord B(t + h) - B(t - h) (one-sided at a segment's
    start), a derivative-free estimate of the tangent."""
    rng = np.random.default_rng(12)
    ctrl = torch.as_tensor(rng.uniform(0, 100, (3, 10, 2)))
    K = 13
    out = oracle.sample_open(ctrl, torch.ones(3, dtype=F64), torch.zeros(3, 3, dtype=F64),
                             torch.ones(3, 3, dtype=F64), SampleCfg(g_open=K, tangent_mode=1))
    s, t = oracle.chain_sample_params(K, 3)
    h = 1e-5
    for k in range(K):
        seg = ctrl[:, 3 * s[k]: 3 * s[k] + 4]
        lo = max(t[k] - h, 0.0)
        hi = min(t[k] + h, 1.0)
        chord = oracle.bezier(seg, torch.full((3,), hi, dtype=F64)) - oracle.bezier(seg, torch.full((3,), lo,
                                                                                                   dtype=F64))
        ang = torch.atan2(chord[:, 1], chord[:, 0])
        diff = torch.remainder(out["theta"][:, k] - ang + math.pi, 2 * math.pi) - math.pi
        assert float(diff.abs().max()) <= 1e-4, k


def test_tangent_mode_closed_rows_interpolate_the_boundary_derivatives():
    """A closed row is (1 - tau) A + tau B (Eq. 4), so its derivative is
    (1 - tau) A'(t) + tau B'(t) (linearity of Eq. 1): mode 1's theta is the
    angle of that combination."""
    rng = np.random.default_rng(13)
    ctrl = torch.as_tensor(rng.uniform(0, 100, (2, 12, 2)))
    cfg = SampleCfg(rows_closed=5, k_closed=9, tangent_mode=1)
    out = oracle.sample_closed(ctrl, torch.zeros(2, 3, dtype=F64), torch.ones(2, dtype=F64), cfg)
    A, B = oracle.closed_boundaries(ctrl)
    dA = oracle.curves.chain_tangents(A, 9)
    dB = oracle.curves.chain_tangents(B, 9)
    tau = oracle.closed_tau(5)
    for r in range(5):
        v = (1 - tau[r]) * dA + tau[r] * dB
        exp = torch.atan2(v[..., 1], v[..., 0])
        assert torch.allclose(out["theta"][:, r], exp, atol=1e-10), r


def test_tangent_mode_zero_derivative_gives_theta_zero():
    """Coincident control points: B'(t) = 0, theta = 0 (the zero-vector rule
    of Eq. 8's reading), with a zero derivative."""
    ctrl = torch.full((1, 10, 2), 7.0, dtype=F64, requires_grad=True)
    out = oracle.sample_open(ctrl, torch.ones(1, dtype=F64), torch.zeros(1, 3, dtype=F64),
                             torch.ones(1, 3, dtype=F64), SampleCfg(g_open=6, tangent_mode=1))
    assert float(out["theta"].abs().max()) == 0.0
    g, = torch.autograd.grad(out["theta"].sum(), ctrl)
    assert float(g.abs().max()) == 0.0
