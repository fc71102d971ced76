"""Batches of images of different sizes and curve counts (bs_batch_*), and
the Adam step (bs_adam_step), against the CPU oracle applied image by image.

Each image of a batch is an independent instance of the method, so the
oracle of a batch is the oracle of each image.  Bars as in the single-canvas
parity tests: draw order and tile lists bit-exact, samples within 1e-5,
forward pixels within 1e-5 absolute off the oracle's flagged pixels,
gradients within 1e-3 relative.  The batched kernels run the same per-tile
and per-curve code as the single-canvas ones, so images, transmittances,
contributor counts, tables and dL/dimg also equal the single-canvas results
bit for bit."""

import numpy as np
import pytest
import torch

import oracle
from oracle.curves import SampleCfg as OCfg, table_from_f32
from oracle.pipeline import as_curves, sample_vjp
from paper_2503_16424_gb300 import synth
from tests.gpu_cases import blend_grad_bound, curve_grad_bound, grad_check, grad_rel_err

pytestmark = pytest.mark.gpu

KEYS = ("open_ctrl", "open_width", "open_color", "open_opac", "closed_ctrl", "closed_color", "closed_opac")
OPEN_KEYS = KEYS[:4]
CLOSED_KEYS = KEYS[4:]


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


# (W, H, n_open, n_closed, g_open, rows, kc, bg, seed): ragged canvases, an
# open-only, a closed-only, a 1x1 and a curve-free image, one with enough
# pairs for several sort partitions, and one whose curves have 512 samples
# or more (so the batch's sampling runs both the narrow and the wide launch)
SPECS = [
    (100, 73, 12, 6, 12, 5, 7, (0.2, 0.5, 0.1), 11),
    (64, 48, 6, 0, 10, 4, 6, (0.0, 0.0, 0.0), 12),
    (33, 90, 0, 4, 8, 4, 6, (0.3, 0.3, 0.3), 13),
    (1, 1, 2, 1, 6, 3, 4, (0.1, 0.2, 0.3), 14),
    (48, 40, 0, 0, 8, 4, 4, (0.5, 0.4, 0.3), 15),
    (256, 200, 60, 30, 16, 4, 8, (0.0, 0.1, 0.2), 16),
    (90, 70, 2, 2, 600, 82, 8, (0.2, 0.2, 0.2), 17),
]


def make_batch(bs, specs, style="local"):
    images, arrs, targets = [], [], []
    for (W, H, no, nc, g, rows, kc, bg, seed) in specs:
        images.append(bs.BatchImage(W, H, no, nc, bs.SampleCfg(g_open=g, rows_closed=rows, k_closed=kc), bg))
        arrs.append(synth.make_curves(seed, W, H, no, nc, style=style).as_dict())
        targets.append(synth.procedural_target(seed + 100, W, H, 6))
    cat = {k: np.concatenate([a[k] for a in arrs], 0) for k in KEYS}
    curves = bs.CurveSet.from_arrays(cat, device="cuda")
    target = torch.as_tensor(np.concatenate([t.reshape(-1) for t in targets]), device="cuda")
    return images, arrs, targets, curves, target


def image_curve_slices(batch, b):
    """Index arrays of image b's curves in the batch numbering (open, then closed)."""
    im = batch.images[b]
    o = np.arange(batch.open0[b], batch.open0[b] + im.n_open)
    c = batch.n_open + np.arange(batch.closed0[b], batch.closed0[b] + im.n_closed)
    return np.concatenate([o, c]).astype(np.int64)


def ocfg_of(im):
    return OCfg(g_open=im.sample.g_open, rows_closed=im.sample.rows_closed, k_closed=im.sample.k_closed,
                tangent_mode=im.sample.tangent_mode)


@pytest.fixture(scope="module")
def ragged(bs):
    from paper_2503_16424_gb300.batch import BatchRasterizer
    images, arrs, targets, curves, target = make_batch(bs, SPECS)
    r = BatchRasterizer(images, pair_capacity=1 << 16)
    r.fit_capacity(curves)
    r.forward(curves, target)
    torch.cuda.synchronize()
    assert r.batch.status()[0] == bs.BS_OK
    return dict(images=images, arrs=arrs, targets=targets, curves=curves, target=target, r=r)


def test_batch_curve_order_bit_exact(bs, ragged):
    r = ragged["r"]
    rank, first = r.rank.cpu().numpy(), r.first.cpu().numpy()
    for b, (im, arr) in enumerate(zip(ragged["images"], ragged["arrs"])):
        idx = image_curve_slices(r.batch, b)
        o_rank, o_first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], ocfg_of(im))
        assert np.array_equal(rank[idx], o_rank), b
        assert np.array_equal(first[idx].astype(np.int64), np.asarray(o_first, dtype=np.int64) + r.batch.gauss0[b]), b


def test_batch_table_matches_oracle_and_single_canvas(bs, ragged):
    r = ragged["r"]
    gauss = r.gauss.cpu().numpy()
    for b, (im, arr) in enumerate(zip(ragged["images"], ragged["arrs"])):
        g0, n = r.batch.gauss0[b], r.batch.n_gauss_of[b]
        if n == 0:
            continue
        mine = gauss[g0:g0 + n].astype(np.float64)
        oc = ocfg_of(im)
        _, o_first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], oc)
        tab = oracle.gaussian_table(as_curves(arr), oc, o_first)
        ref = np.stack([tab[k].detach().numpy() for k in ("mx", "my", "ux", "uy", "isx", "isy")], 1)
        assert np.abs(mine[:, 0:2] - ref[:, 0:2]).max() / max(im.width, im.height) <= 1e-5
        assert np.abs(mine[:, 2:4] - ref[:, 2:4]).max() <= 1e-5
        assert (np.abs(mine[:, 4:6] - ref[:, 4:6]) / ref[:, 4:6]).max() <= 1e-5
        # the single-canvas call on this image alone gives the same records
        cv = bs.CurveSet.from_arrays(arr, device="cuda")
        _, first1 = bs.curve_order(cv, im.sample)
        single = bs.sample_curves(cv, im.sample, first1).cpu().numpy()
        assert np.array_equal(single, gauss[g0:g0 + n]), b


def test_batch_tile_lists_bit_exact(bs, ragged):
    r = ragged["r"]
    gauss = r.gauss.cpu().numpy()
    vals = r.vals.cpu().numpy().view(np.uint32)
    ranges = r.ranges.cpu().numpy().view(np.uint32)
    total = 0
    for b, im in enumerate(ragged["images"]):
        g0, n = r.batch.gauss0[b], r.batch.n_gauss_of[b]
        t0 = r.batch.tile0[b]
        tiles_x, tiles_y = -(-im.width // 16), -(-im.height // 16)
        if n == 0:
            assert np.all(ranges[t0:t0 + tiles_x * tiles_y] == 0)
            continue
        keys, oranges, counts = oracle.tile_keys(gauss[g0:g0 + n], im.width, im.height, 16)
        gbits, _ = oracle.key_bits(n, tiles_x * tiles_y)
        local = keys & np.uint32((1 << gbits) - 1)
        for t in range(tiles_x * tiles_y):
            s, e = ranges[t0 + t]
            os_, oe = oranges[t]
            mine = vals[s:e].astype(np.int64) - g0
            ref = local[os_:oe].astype(np.int64)
            assert np.array_equal(mine, ref), (b, t)
        total += int(counts.sum())
    assert r.batch.status()[1] == total


def test_batch_forward_matches_oracle_and_single_canvas(bs, ragged):
    from paper_2503_16424_gb300.raster import Rasterizer
    r = ragged["r"]
    gauss = r.gauss.cpu().numpy()
    loss = r.loss.cpu().numpy()
    for b, (im, arr, tgt) in enumerate(zip(ragged["images"], ragged["arrs"], ragged["targets"])):
        g0, n = r.batch.gauss0[b], r.batch.n_gauss_of[b]
        img = r.batch.image(r.img, b).cpu().double()
        if n == 0:   # no Gaussian: T = 1 and C = bg at every pixel (Eq. 9)
            bg = torch.tensor(im.bg, dtype=torch.float64)[:, None, None].expand(3, im.height, im.width)
            assert torch.equal(img, bg.to(torch.float32).double())
        else:
            tab = table_from_f32(gauss[g0:g0 + n])
            ref = oracle.render_image(tab, im.width, im.height, bg=im.bg, margin=1e-5)
            ok = ~ref["flag"]
            err = (img - ref["img"]).abs().amax(0)
            assert float(((~ok) & (err > 1e-5)).double().mean()) < 1e-4, b   # excused pixels
            assert float(err[ok].max()) <= 1e-5, b
        l_ref, _ = oracle.l2_loss(img, tgt)
        assert abs(loss[b] - float(l_ref)) <= 1e-6 * max(1.0, float(l_ref)), b
        # the single-canvas path on this image alone: bit-identical results
        cv = bs.CurveSet.from_arrays(arr, device="cuda")
        one = Rasterizer(bs.Canvas(im.width, im.height, 16, im.bg), im.sample, im.n_open, im.n_closed,
                         pair_capacity=4096)
        one.forward(cv)
        tg = torch.as_tensor(tgt, device="cuda")
        bs.render_fwd_l2(one.gauss, one.canvas, one.binning, tg, out=(one.img, one.T, one.nc), dimg=one.dimg,
                         loss=one.loss)
        assert torch.equal(one.img, r.batch.image(r.img, b)), b
        assert torch.equal(one.T, r.batch.pixel_map(r.T, b)), b
        assert torch.equal(one.nc, r.batch.pixel_map(r.nc, b)), b
        assert torch.equal(one.dimg, r.batch.image(r.dimg, b)), b


def test_batch_backward_matches_oracle(bs, ragged):
    """Curve gradients of every image (flagged pixels masked on both sides)
    against the oracle's vector-Jacobian products."""
    r = ragged["r"]
    curves = ragged["curves"]
    gauss = r.gauss.cpu().numpy()
    dimg = r.dimg.clone()
    masks = []
    for b, im in enumerate(ragged["images"]):
        g0, n = r.batch.gauss0[b], r.batch.n_gauss_of[b]
        if n == 0:
            continue
        ref = oracle.render_image(table_from_f32(gauss[g0:g0 + n]), im.width, im.height, bg=im.bg)
        ok = (~ref["flag"]).to("cuda")
        r.batch.image(dimg, b).mul_(ok[None].float())
        masks.append(ok)
    grad = curves.zeros_like()
    r.backward(curves, dimg, grad)
    for b, (im, arr) in enumerate(zip(ragged["images"], ragged["arrs"])):
        if im.n_open + im.n_closed == 0:
            continue
        oc = ocfg_of(im)
        g0, n = r.batch.gauss0[b], r.batch.n_gauss_of[b]
        _, o_first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], oc)
        tab = table_from_f32(gauss[g0:g0 + n])
        ys, xs = torch.meshgrid(torch.arange(im.height, dtype=torch.float64),
                                torch.arange(im.width, dtype=torch.float64), indexing="ij")
        dC = r.batch.image(dimg, b).cpu().double().permute(1, 2, 0).reshape(-1, 3)
        dtab = oracle.render_grads(tab, xs.reshape(-1), ys.reshape(-1), dC, bg=im.bg)
        dref = sample_vjp(as_curves(arr), oc, dtab, o_first)
        cb = curve_grad_bound(arr, oc, o_first, blend_grad_bound(gauss[g0:g0 + n], im.width, im.height, dC, im.bg),
                              dtab)
        for k in KEYS:
            if k in OPEN_KEYS:
                got = getattr(grad, k)[r.batch.open0[b]:r.batch.open0[b] + im.n_open]
            else:
                got = getattr(grad, k)[r.batch.closed0[b]:r.batch.closed0[b] + im.n_closed]
            if got.numel() == 0:
                continue
            e = grad_check(got.cpu(), dref[k], cb[k])
            assert e <= 1.0, (b, k, e)


def test_batch_with_mixed_tangent_modes_matches_oracle_and_single_canvas(bs):
    """Images of one batch may take their rotations from different rules:
    Eq. 8's neighbour difference (tangent_mode 0) beside the derivative
    B'(t) (tangent_mode 1).  Per image: the table against the oracle and bit
    for bit against the single-canvas call with the same mode, and the curve
    gradients against the oracle (bars as above)."""
    from paper_2503_16424_gb300.batch import BatchRasterizer
    specs = SPECS[:3] + SPECS[5:6]
    modes = (1, 0, 1, 1)
    images, arrs, targets, curves, target = make_batch(bs, specs)
    for im, m in zip(images, modes):
        im.sample = bs.SampleCfg(g_open=im.sample.g_open, rows_closed=im.sample.rows_closed,
                                 k_closed=im.sample.k_closed, tangent_mode=m)
    r = BatchRasterizer(images, pair_capacity=1 << 16)
    r.fit_capacity(curves)
    r.forward(curves, target)
    torch.cuda.synchronize()
    assert r.batch.status()[0] == bs.BS_OK
    gauss = r.gauss.cpu().numpy()
    dimg = r.dimg.clone()
    for b, im in enumerate(images):
        g0, n = r.batch.gauss0[b], r.batch.n_gauss_of[b]
        ref = oracle.render_image(table_from_f32(gauss[g0:g0 + n]), im.width, im.height, bg=im.bg)
        r.batch.image(dimg, b).mul_((~ref["flag"]).to("cuda")[None].float())
    grad = curves.zeros_like()
    r.backward(curves, dimg, grad)
    for b, (im, arr) in enumerate(zip(images, arrs)):
        g0, n = r.batch.gauss0[b], r.batch.n_gauss_of[b]
        oc = ocfg_of(im)
        _, o_first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], oc)
        tab = oracle.gaussian_table(as_curves(arr), oc, o_first)
        mine = gauss[g0:g0 + n].astype(np.float64)
        ref = np.stack([tab[k].detach().numpy() for k in ("mx", "my", "ux", "uy", "isx", "isy")], 1)
        assert np.abs(mine[:, 0:2] - ref[:, 0:2]).max() / max(im.width, im.height) <= 1e-5, b
        assert np.abs(mine[:, 2:4] - ref[:, 2:4]).max() <= 1e-5, b
        assert (np.abs(mine[:, 4:6] - ref[:, 4:6]) / ref[:, 4:6]).max() <= 1e-5, b
        cv = bs.CurveSet.from_arrays(arr, device="cuda")
        _, first1 = bs.curve_order(cv, im.sample)
        assert np.array_equal(bs.sample_curves(cv, im.sample, first1).cpu().numpy(), gauss[g0:g0 + n]), b
        ftab = table_from_f32(gauss[g0:g0 + n])
        ys, xs = torch.meshgrid(torch.arange(im.height, dtype=torch.float64),
                                torch.arange(im.width, dtype=torch.float64), indexing="ij")
        dC = r.batch.image(dimg, b).cpu().double().permute(1, 2, 0).reshape(-1, 3)
        dtab = oracle.render_grads(ftab, xs.reshape(-1), ys.reshape(-1), dC, bg=im.bg)
        dref = sample_vjp(as_curves(arr), oc, dtab, o_first)
        cb = curve_grad_bound(arr, oc, o_first, blend_grad_bound(gauss[g0:g0 + n], im.width, im.height, dC, im.bg),
                              dtab)
        for k in KEYS:
            if k in OPEN_KEYS:
                got = getattr(grad, k)[r.batch.open0[b]:r.batch.open0[b] + im.n_open]
            else:
                got = getattr(grad, k)[r.batch.closed0[b]:r.batch.closed0[b] + im.n_closed]
            if got.numel() == 0:
                continue
            e = grad_check(got.cpu(), dref[k], cb[k])
            assert e <= 1.0, (b, k, e)


def test_batch_capacity_overflow_renders_nothing_and_reports(bs):
    from paper_2503_16424_gb300.batch import BatchRasterizer
    images, arrs, targets, curves, target = make_batch(bs, SPECS[:3])
    r = BatchRasterizer(images, pair_capacity=64)
    r.forward(curves, target)
    st, n_pairs = r.batch.status()
    assert st == bs.BS_ERR_CAPACITY and n_pairs > 64
    assert torch.count_nonzero(r.ranges) == 0
    for b, im in enumerate(images):   # nothing blended: the background everywhere
        bg = torch.tensor(im.bg, device="cuda", dtype=torch.float32)[:, None, None]
        assert torch.equal(r.batch.image(r.img, b), bg.expand(3, im.height, im.width))
    r.grow(n_pairs)
    r.forward(curves, target)
    st2, n2 = r.batch.status()
    assert st2 == bs.BS_OK and n2 == n_pairs


def test_batch_three_sort_passes_on_a_large_canvas(bs):
    """More than 2^16 tiles: three sort passes over the tile bits."""
    from paper_2503_16424_gb300.batch import BatchRasterizer
    specs = [(4100, 4100, 40, 20, 16, 4, 8, (0.0, 0.0, 0.0), 21), (70, 50, 5, 3, 12, 4, 6, (0.1, 0.1, 0.1), 22)]
    images, arrs, targets, curves, target = make_batch(bs, specs)
    r = BatchRasterizer(images, pair_capacity=1 << 16)
    r.fit_capacity(curves)
    r.forward(curves, target)
    st, total = r.batch.status()
    assert st == bs.BS_OK
    gauss = r.gauss.cpu().numpy()
    vals = r.vals.cpu().numpy().view(np.uint32)
    ranges = r.ranges.cpu().numpy().view(np.uint32)
    seen = 0
    for b, im in enumerate(images):
        g0, n = r.batch.gauss0[b], r.batch.n_gauss_of[b]
        tiles_x = -(-im.width // 16)
        keys, oranges, counts = oracle.tile_keys(gauss[g0:g0 + n], im.width, im.height, 16)
        gbits, _ = oracle.key_bits(n, tiles_x * (-(-im.height // 16)))
        local = keys & np.uint32((1 << gbits) - 1)
        nz = np.nonzero(oranges[:, 1] > oranges[:, 0])[0]
        for t in nz:
            s, e = ranges[r.batch.tile0[b] + t]
            assert np.array_equal(vals[s:e].astype(np.int64) - g0, local[oranges[t, 0]:oranges[t, 1]].astype(np.int64))
        seen += int(counts.sum())
        # sampled pixels of the blend against the oracle's brute force
        rng = np.random.default_rng(b)
        xs = rng.integers(0, im.width, 64)
        ys = rng.integers(0, im.height, 64)
        px = oracle.render_pixels(table_from_f32(gauss[g0:g0 + n]), xs, ys, bg=im.bg)
        img = r.batch.image(r.img, b).cpu().double()
        got = img[:, torch.as_tensor(ys), torch.as_tensor(xs)].T
        ok = ~px["flag"]
        assert float((got - px["C"]).abs().amax(1)[ok].max()) <= 1e-5
    assert seen == total


def test_adam_step_matches_oracle(bs):
    rng = np.random.default_rng(5)
    n1, n2 = 1000, 77
    p1 = rng.normal(0, 1, n1).astype(np.float32)
    p2 = rng.uniform(0, 1, n2).astype(np.float32)
    scale = rng.uniform(0.5, 3.0, n1 // 10).astype(np.float32)
    t = {k: torch.as_tensor(v, device="cuda") for k, v in dict(p1=p1, p2=p2, scale=scale).items()}
    g1 = torch.zeros(n1, device="cuda")
    g2 = torch.zeros(n2, device="cuda")
    m1, v1, m2, v2 = (torch.zeros_like(x) for x in (g1, g1, g2, g2))
    groups = [bs.AdamGroup(t["p1"], g1, m1, v1, 0.05, row_scale=t["scale"], row_len=10),
              bs.AdamGroup(t["p2"], g2, m2, v2, 0.2, lo=0.0, hi=1.0)]
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    ref = [(p1.astype(np.float64), np.zeros(n1), np.zeros(n1)), (p2.astype(np.float64), np.zeros(n2), np.zeros(n2))]
    lr1 = np.float32(0.05) * np.repeat(scale, 10)   # the kernel's float32 product
    for it in range(1, 5):
        gg1 = rng.normal(0, 1e-2 * it, n1).astype(np.float32)
        gg2 = rng.normal(0, 1.0, n2).astype(np.float32)
        gg2[:5] = 0.0
        g1.copy_(torch.as_tensor(gg1))
        g2.copy_(torch.as_tensor(gg2))
        bs.adam_step(groups, step)
        # the call takes float32 hyperparameters: the oracle gets those values
        # (1 - float32(0.999) differs from 0.001 by 1.3e-5 relative)
        hp = dict(beta1=float(np.float32(0.9)), beta2=float(np.float32(0.999)), eps=float(np.float32(1e-8)))
        ref[0] = oracle.adam_step(ref[0][0], gg1, ref[0][1], ref[0][2], it, lr1, **hp)
        ref[1] = oracle.adam_step(ref[1][0], gg2, ref[1][1], ref[1][2], it, float(np.float32(0.2)), lo=0.0, hi=1.0,
                                  **hp)
    torch.cuda.synchronize()
    assert int(step.item()) == 4
    assert np.abs(t["p1"].cpu().numpy() - ref[0][0]).max() <= 1e-5
    assert np.abs(t["p2"].cpu().numpy() - ref[1][0]).max() <= 1e-5
    assert t["p2"].min().item() >= 0.0 and t["p2"].max().item() <= 1.0
    assert np.abs(m1.cpu().numpy() - ref[0][1]).max() <= 1e-7
    assert (np.abs(v2.cpu().numpy() - ref[1][2]) / np.maximum(ref[1][2], 1e-12)).max() <= 1e-5


def test_graph_replay_matches_eager_steps(bs):
    from paper_2503_16424_gb300.batch import BatchOptimizer, BatchRasterizer
    specs = SPECS[:3] + SPECS[5:]
    res = {}
    for graph in (False, True):
        images, arrs, targets, curves, target = make_batch(bs, specs)
        r = BatchRasterizer(images, pair_capacity=1 << 16)
        opt = BatchOptimizer(r, curves, target, graph=graph, check_every=3)
        losses = []
        for _ in range(6):
            opt.step()
            losses.append(r.loss.clone())
        torch.cuda.synchronize()
        res[graph] = (torch.stack(losses).cpu().numpy(), curves, int(opt.adam.t.item()))
        if graph:
            assert opt.graph is not None
    (l0, c0, t0), (l1, c1, t1) = res[False], res[True]
    assert t0 == t1 == 6
    assert np.allclose(l0, l1, rtol=1e-4, atol=1e-9)
    for k in KEYS:
        a, b = getattr(c0, k), getattr(c1, k)
        if a.numel():
            assert float((a - b).abs().max()) <= 1e-2, k


def test_batched_and_plain_reach_the_same_psnr(bs):
    """The same Adam steps through the batch and image by image through the
    single-canvas calls give the same PSNR on every image."""
    from paper_2503_16424_gb300.batch import BatchOptimizer, BatchRasterizer, PlainOptimizer
    specs = [SPECS[0], SPECS[1], SPECS[5]]
    images, arrs, targets, curves, target = make_batch(bs, specs)
    r = BatchRasterizer(images, pair_capacity=1 << 16)
    opt = BatchOptimizer(r, curves, target, graph=True, check_every=0)
    for _ in range(30):
        opt.step()
    r.forward(curves, target)
    p_batch = r.psnr(target)
    per_img = [bs.CurveSet.from_arrays(a, device="cuda") for a in arrs]
    tg = [torch.as_tensor(t, device="cuda") for t in targets]
    plain = PlainOptimizer(images, per_img, tg)
    for _ in range(30):
        plain.step()
    p_plain = []
    for (rr, cv, t, _, _) in plain.items:
        img = rr.forward(cv)
        mse = float(((img - t).double() ** 2).mean())
        p_plain.append(-10.0 * np.log10(mse))
    print("PSNR batch", np.round(p_batch, 3), "plain", np.round(p_plain, 3))
    assert np.allclose(p_batch, p_plain, atol=0.05)
    init = BatchRasterizer(images, pair_capacity=1 << 16)
    _, _, _, c_init, _ = make_batch(bs, specs)
    init.fit_capacity(c_init)
    init.forward(c_init, target)
    assert all(a > b for a, b in zip(p_batch, init.psnr(target)))
