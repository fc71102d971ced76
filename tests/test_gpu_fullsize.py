"""Parity at the full benchmark size (2048x2048, 2048 open + 2048 closed
curves, 64 Gaussians per curve = 262,144 Gaussians, about 10^7 tile pairs),
in the launch configuration bench.py times: draw order and every tile key
bit-exact, all Gaussians of the sampling, sampled pixels of the blend, and
the backward of a loss on a 32x32 crop."""

import numpy as np
import pytest
import torch

import oracle
from oracle.curves import SampleCfg as OCfg, table_to_f32, table_from_f32
from oracle.pipeline import as_curves
from paper_2503_16424_gb300 import synth
from tests.gpu_cases import blend_grad_bound, grad_check, grad_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem():
    from paper_2503_16424_gb300 import bs
    from paper_2503_16424_gb300.raster import Rasterizer
    w = synth.WORKLOADS["hires_2048_4096"]
    arr = synth.make_curves(w["seed"], w["W"], w["H"], w["n_open"], w["n_closed"], style=w["style"]).as_dict()
    ocfg = OCfg(g_open=w["g_open"], rows_closed=w["rows_closed"], k_closed=w["k_closed"])
    rank, first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], ocfg)
    with torch.no_grad():
        tab = oracle.gaussian_table(as_curves(arr), ocfg, first)
    cfg = bs.SampleCfg(g_open=w["g_open"], rows_closed=w["rows_closed"], k_closed=w["k_closed"])
    curves = bs.CurveSet.from_arrays(arr, device="cuda")
    r = Rasterizer(bs.Canvas(w["W"], w["H"], w["tile"]), cfg, curves.n_open, curves.n_closed,
                   pair_capacity=1 << 25)
    return dict(bs=bs, w=w, arr=arr, rank=rank, first=first, tab=tab, rec=table_to_f32(tab), r=r,
                curves=curves)


def test_full_order_and_sampling(problem):
    p = problem
    r = p["r"]
    r.forward(p["curves"])
    assert np.array_equal(r.rank.cpu().numpy(), p["rank"])
    assert np.array_equal(r.first.cpu().numpy(), p["first"])
    got = r.gauss.cpu().numpy().astype(np.float64)
    tab = p["tab"]
    ref64 = np.stack([tab[k].numpy() for k in ("mx", "my", "ux", "uy", "isx", "isy")], 1)
    pos = np.abs(got[:, 0:2] - ref64[:, 0:2]).max() / 2048
    u = np.abs(got[:, 2:4] - ref64[:, 2:4]).max()
    sc = (np.abs(got[:, 4:6] - ref64[:, 4:6]) / ref64[:, 4:6]).max()
    print(f"full sampling: position err {pos:.1e} of canvas, direction err {u:.1e}, scale err {sc:.1e}")
    assert pos <= 1e-5 and u <= 1e-5 and sc <= 1e-5


def test_full_binning_bit_exact(problem):
    p = problem
    bs = p["bs"]
    rec = p["rec"]
    keys, ranges, _ = oracle.tile_keys(rec, 2048, 2048, 16)
    gauss = torch.as_tensor(rec, device="cuda")
    b = bs.Binning(bs.Canvas(2048, 2048), "cuda", pair_capacity=1 << 25).run(gauss)
    print(f"full binning: {keys.shape[0]} pairs")
    assert b.device_status() == 0
    assert b.n_pairs == keys.shape[0]
    assert np.array_equal(b.keys[:b.n_pairs].cpu().numpy().view(np.uint32), keys)
    assert np.array_equal(b.ranges.cpu().numpy().view(np.uint32), ranges)
    p["binning"] = b
    p["gauss_in"] = gauss


def test_full_blend_sampled_pixels(problem):
    p = problem
    bs = p["bs"]
    if "binning" not in p:
        pytest.skip("needs the binning test")
    canvas = bs.Canvas(2048, 2048)
    img, T, nc = bs.render_fwd(p["gauss_in"], canvas, p["binning"])
    rng = np.random.default_rng(0)
    n = 192
    xs = rng.integers(0, 2048, n)
    ys = rng.integers(0, 2048, n)
    tab = table_from_f32(p["rec"])
    ref = {"C": [], "T": [], "flag": []}
    for s in range(0, n, 16):
        rr = oracle.render_pixels(tab, xs[s:s + 16].astype(np.float64), ys[s:s + 16].astype(np.float64),
                                  margin=1e-5)
        for k in ref:
            ref[k].append(rr[k])
    C = torch.cat(ref["C"]).numpy()
    flag = torch.cat(ref["flag"]).numpy()
    got = img.cpu().numpy()[:, ys, xs].T.astype(np.float64)
    err = np.abs(got - C).max(1)
    print(f"full blend: {n} pixels, flagged {flag.sum()}, max err {err[~flag].max():.1e}, "
          f"incl. flagged {err.max():.1e}")
    assert int((flag & (err > 1e-5)).sum()) == 0      # no excused pixel among the samples
    assert err[~flag].max() <= 1e-5
    p["fwd"] = (img, T, nc)


def test_full_backward_crop(problem):
    p = problem
    bs = p["bs"]
    if "fwd" not in p:
        pytest.skip("needs the blend test")
    img, T, nc = p["fwd"]
    x0, y0, side = 1008, 1008, 32
    tab = table_from_f32(p["rec"])
    ys, xs = torch.meshgrid(torch.arange(y0, y0 + side, dtype=torch.float64),
                            torch.arange(x0, x0 + side, dtype=torch.float64), indexing="ij")
    xs, ys = xs.reshape(-1), ys.reshape(-1)
    # Gaussians whose support box touches the crop (all others have alpha < 1/255 there)
    ex, ey = tab["ext_x"], tab["ext_y"]
    near = ((ex >= 0) & (tab["mx"] + ex >= x0 + 0.5) & (tab["mx"] - ex <= x0 + side - 0.5)
            & (tab["my"] + ey >= y0 + 0.5) & (tab["my"] - ey <= y0 + side - 0.5))
    idx = torch.nonzero(near)[:, 0]
    sub = {k: v[idx] for k, v in tab.items()}
    pf = oracle.render_pixels(sub, xs, ys, margin=1e-4)
    rng = np.random.default_rng(1)
    dC = torch.as_tensor(rng.normal(0, 1e-6, (side * side, 3)))
    dC[pf["flag"]] = 0.0
    dimg = torch.zeros(3, 2048, 2048, dtype=torch.float32)
    dimg[:, y0:y0 + side, x0:x0 + side] = dC.float().reshape(side, side, 3).permute(2, 0, 1)
    dgauss, _ = bs.render_bwd(p["gauss_in"], bs.Canvas(2048, 2048), p["binning"], T, nc, dimg.cuda())
    ref = oracle.render_grads(sub, xs, ys, dC.float().double())
    got = dgauss.cpu().double()
    others = torch.ones(got.shape[0], dtype=torch.bool)
    others[idx] = False
    assert float(got[others].abs().max()) == 0.0
    g = got[idx]
    cols = {"mx": 0, "my": 1, "ux": 2, "uy": 3, "isx": 4, "isy": 5, "o": 6, "col": slice(7, 10)}
    bound = blend_grad_bound(p["rec"][idx.numpy()], 2048, 2048, dC.float().double(), xs=xs, ys=ys, tab=sub)
    errs = {k: grad_rel_err(g[:, c], ref[k]) for k, c in cols.items()}
    ratio = {k: grad_check(g[:, c], ref[k], bound[k]) for k, c in cols.items()}
    print(f"full backward crop: {idx.numel()} Gaussians near the crop, rel errs " +
          ", ".join(f"{k} {v:.1e}" for k, v in errs.items()) +
          "; of the bar: " + ", ".join(f"{k} {v:.2f}" for k, v in ratio.items()))
    for k, e in ratio.items():
        assert e <= 1.0, k


def test_full_crop_curve_gradients_match_finite_differences(problem):
    """The 2048 x 2048 workload's curve gradients of an L2 loss on the 32 x 32
    crop at (1008, 1008), against fp64 central differences of the oracle's
    crop loss: the perturbed curve is re-sampled by the oracle, every other
    Gaussian that reaches the crop is the GPU's record, and the crop is
    blended by brute force in draw order.  Pixels with a threshold decision
    within 1e-4 (a kink of the blend) are masked on both sides.  Bar: 1e-3
    relative (floor 1e-6 max|g|) plus the entry's float32 rounding bound plus
    the difference quotient's own error, estimated from a second step."""
    from oracle.bounds import blend_abs, sample_abs_vjp
    from tests.gpu_cases import DEPTH, U32, tiles_per_gaussian
    p = problem
    bs, r, w, arr = p["bs"], p["r"], p["w"], p["arr"]
    r.forward(p["curves"])
    rec = r.gauss.cpu().numpy()
    first = r.first.cpu().numpy().astype(np.int64)
    n_open, per_open, per_closed = w["n_open"], w["g_open"], w["rows_closed"] * w["k_closed"]
    ocfg = OCfg(g_open=w["g_open"], rows_closed=w["rows_closed"], k_closed=w["k_closed"])
    x0 = y0 = 1008
    side = 32
    yy, xx = torch.meshgrid(torch.arange(y0, y0 + side, dtype=torch.float64),
                            torch.arange(x0, x0 + side, dtype=torch.float64), indexing="ij")
    xs, ys = xx.reshape(-1), yy.reshape(-1)
    tgt = synth.procedural_target(w["seed"] + 1, 2048, 2048, w["n_shapes"])
    t_crop = torch.as_tensor(tgt[:, y0:y0 + side, x0:x0 + side]).permute(1, 2, 0).reshape(-1, 3).double()
    tab = table_from_f32(rec)
    ex, ey = tab["ext_x"], tab["ext_y"]
    near = ((ex >= 0) & (tab["mx"] + ex >= x0 + 0.5) & (tab["mx"] - ex <= x0 + side - 0.5)
            & (tab["my"] + ey >= y0 + 0.5) & (tab["my"] - ey <= y0 + side - 0.5)).numpy()
    # the curve owning each Gaussian (curves are draw-ordered runs from first)
    order = np.argsort(first)
    owner = np.empty(rec.shape[0], np.int64)
    for c in order:
        n = per_open if c < n_open else per_closed
        owner[first[c]:first[c] + n] = c
    counts = np.bincount(owner[near], minlength=first.shape[0])
    opens = [int(c) for c in np.argsort(-counts[:n_open])[:2] if counts[c] > 0]
    closeds = [int(c) + n_open for c in np.argsort(-counts[n_open:])[:2] if counts[c + n_open] > 0]
    chosen = opens + closeds
    assert len(chosen) == 4
    rows = {c: np.arange(first[c], first[c] + (per_open if c < n_open else per_closed)) for c in chosen}
    sub_idx = np.unique(np.concatenate([np.nonzero(near)[0]] + list(rows.values())))
    pos = {g: i for i, g in enumerate(sub_idx)}
    sub = {k: v[torch.as_tensor(sub_idx)] for k, v in tab.items()}
    mask = ~oracle.render_pixels(sub, xs, ys, margin=1e-4)["flag"]
    img = r.img[:, y0:y0 + side, x0:x0 + side].cpu().double().permute(1, 2, 0).reshape(-1, 3)
    n_crop = 3 * side * side
    dC = (2.0 * (img - t_crop) / n_crop) * mask[:, None].double()
    dimg = torch.zeros(3, 2048, 2048, dtype=torch.float32)
    dimg[:, y0:y0 + side, x0:x0 + side] = dC.float().reshape(side, side, 3).permute(2, 0, 1)
    grad = r.backward(p["curves"], dimg.cuda())

    def one_curve(c, a):
        """The oracle's records of curve c of the arrays a, alone."""
        one = {k: v[c:c + 1] if k.startswith("open") else v[:0] for k, v in a.items() if k.startswith("open")}
        one.update({k: (v[c - n_open:c - n_open + 1] if c >= n_open else v[:0]) for k, v in a.items()
                    if k.startswith("closed")})
        if c < n_open:
            one.update({k: v[:0] for k, v in a.items() if k.startswith("closed")})
        with torch.no_grad():
            return oracle.gaussian_table(as_curves(one), ocfg, np.array([0]))

    def crop_loss(c, a):
        t1 = one_curve(c, a)
        s = {k: v.clone() for k, v in sub.items()}
        ix = torch.as_tensor([pos[g] for g in rows[c]])
        for k in ("mx", "my", "ux", "uy", "isx", "isy", "o", "col"):
            s[k][ix] = t1[k]
        C = oracle.render_pixels(s, xs, ys)["C"]
        d = (C - t_crop) * mask[:, None].double()
        return float((d * d).sum()) / n_crop

    loss0 = float(((img - t_crop) ** 2 * mask[:, None].double()).sum()) / n_crop
    keys0 = oracle.area_keys_f32(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"])
    in_crop = np.unique(owner[near])

    def central(c, k, i, h):
        vals = []
        for sgn in (1.0, -1.0):
            a = {kk: np.array(v, dtype=np.float64) for kk, v in arr.items()}
            row = c if k.startswith("open") else c - n_open
            a[k].reshape(a[k].shape[0], -1)[row, i] += sgn * h
            keys = oracle.area_keys_f32(a["open_ctrl"].astype(np.float32), a["open_width"].astype(np.float32),
                                        a["closed_ctrl"].astype(np.float32))
            # the draw order among the curves reaching the crop is unchanged
            assert np.array_equal(np.argsort(keys[in_crop], kind="stable"), np.argsort(keys0[in_crop], kind="stable"))
            vals.append(crop_loss(c, a))
        return (vals[0] - vals[1]) / (2 * h)

    # the float32 rounding bound of the chosen curves' gradients
    A = blend_abs(sub, xs, ys, dC)
    dtab = oracle.render_grads(sub, xs, ys, dC)
    ntile = tiles_per_gaussian(rec[sub_idx], 2048, 2048)
    cf = (DEPTH + ntile) * U32
    checked = 0
    for c in chosen:
        kind = "open" if c < n_open else "closed"
        ix = torch.as_tensor([pos[g] for g in rows[c]])
        one = {k: v[c:c + 1] for k, v in arr.items() if k.startswith("open")} if kind == "open" else \
            {k: v[c - n_open:c - n_open + 1] for k, v in arr.items() if k.startswith("closed")}
        other = "closed" if kind == "open" else "open"
        one.update({k: v[:0] for k, v in arr.items() if k.startswith(other)})
        gb = {k: (cf[ix][:, None] * A[k][ix] if A[k].dim() == 2 else cf[ix] * A[k][ix]) for k in A}
        dtab_c = {k: v[ix] for k, v in dtab.items()}
        scale = {k: gb[k] + DEPTH * U32 * dtab_c[k].abs() for k in gb}
        bound = sample_abs_vjp(as_curves(one), ocfg, scale, np.array([0]))
        # the two control coordinates with the largest gradient, and the attributes
        ck = kind + "_ctrl"
        gc = getattr(grad, ck).cpu().double()[c if kind == "open" else c - n_open].reshape(-1)
        top = [int(i) for i in torch.argsort(gc.abs(), descending=True)[:2]]
        params = [(ck, top[0]), (ck, top[1])] + ([("open_width", 0), ("open_color", 1)] if kind == "open"
                                                 else [("closed_color", 2), ("closed_opac", 0)])
        for k, i in params:
            row = c if kind == "open" else c - n_open
            g_all = getattr(grad, k).cpu().double()
            g = float(g_all[row].reshape(-1)[i])
            gmax = float(g_all.abs().max())
            base = float(np.asarray(arr[k])[row].reshape(-1)[i])
            # px for positions: small enough that no unmasked threshold decision moves across
            h = 1e-5 if k.endswith("ctrl") else 1e-5 * max(1.0, abs(base))
            fd, fd2 = central(c, k, i, h), central(c, k, i, 2 * h)
            b = float(bound[k][0].reshape(-1)[i])
            # the quotient's own error: truncation (from the second step) and the
            # fp64 rounding of the two crop losses (64 eps |L| each, over 2h)
            allow = 1e-3 * max(abs(fd), 1e-6 * gmax) + b + abs(fd - fd2) / 3 + 64 * 2.2e-16 * loss0 / h
            print(f"crop FD: curve {c} {k}[{i}]: gpu {g:.6e} fd {fd:.6e} (2h {fd2:.6e}), allowance {allow:.2e}")
            assert abs(g - fd) <= allow, (c, k, i, g, fd, fd2)
            checked += 1
    assert checked == 16
