"""The single-canvas step without host synchronisation: the binning that
reads nothing back (bs_bin_tiles_async) against the synchronising one and
the oracle, its capacity overflow, one whole step captured as a CUDA graph
against the eager step, the library's non-finite status word
(bs_sync_status), and the autograd Function called twice before one
backward."""

import numpy as np
import pytest
import torch

import oracle
from oracle.curves import table_to_f32
from paper_2503_16424_gb300 import synth
from tests.gpu_cases import CASES, arrays, oracle_table

pytestmark = pytest.mark.gpu

KEYS = ("open_ctrl", "open_width", "open_color", "open_opac", "closed_ctrl", "closed_color", "closed_opac")


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


@pytest.mark.parametrize("name", ["tiny256", "mixed", "ragged"])
def test_async_binning_matches_sync_and_oracle(bs, name):
    """Keys and ranges bit-exact against the oracle and the synchronising
    call; the device pair count matches; the status word stays 0."""
    case = CASES[name]
    tab, _, _ = oracle_table(case)
    rec = table_to_f32(tab)
    keys, ranges, _ = oracle.tile_keys(rec, case.W, case.H, 16)
    gauss = torch.as_tensor(rec, device="cuda")
    canvas = bs.Canvas(case.W, case.H, 16, case.bg)
    b = bs.Binning(canvas, "cuda", pair_capacity=keys.shape[0] + 5000).prepare(rec.shape[0])
    p_dev = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    for _ in range(2):      # twice on the same workspace
        b.run_async(gauss, p_dev)
        st, n = b.result()
        assert st == bs.BS_OK and n == keys.shape[0] == int(p_dev.item())
        assert np.array_equal(b.keys[:n].cpu().numpy().view(np.uint32), keys)
        assert np.array_equal(b.ranges.cpu().numpy().view(np.uint32), ranges)
    s = bs.Binning(canvas, "cuda", pair_capacity=1024).run(gauss)
    assert np.array_equal(s.keys[:s.n_pairs].cpu().numpy(), b.keys[:n].cpu().numpy())


def test_async_binning_overflow_empties_the_ranges_and_reports(bs):
    case = CASES["mixed"]
    tab, _, _ = oracle_table(case)
    rec = table_to_f32(tab)
    keys, ranges, _ = oracle.tile_keys(rec, case.W, case.H, 16)
    gauss = torch.as_tensor(rec, device="cuda")
    canvas = bs.Canvas(case.W, case.H, 16, case.bg)
    b = bs.Binning(canvas, "cuda", pair_capacity=64).prepare(rec.shape[0], 64)
    b.run_async(gauss)
    st, n = b.result()
    assert st == bs.BS_ERR_CAPACITY and n == keys.shape[0]
    assert torch.count_nonzero(b.ranges) == 0
    img, T, nc = bs.render_fwd(gauss, canvas, b)          # nothing blended: the background
    bg = torch.tensor(case.bg, device="cuda")[:, None, None].expand(3, case.H, case.W)
    assert torch.equal(img, bg) and torch.all(T == 1) and torch.all(nc == 0)
    b.prepare(rec.shape[0], n)                              # exactly enough room
    b.run_async(gauss)
    assert b.result() == (bs.BS_OK, n)
    assert np.array_equal(b.keys[:n].cpu().numpy().view(np.uint32), keys)


def _problem(bs, seed=5, W=96, H=80, no=10, nc=5):
    from paper_2503_16424_gb300.raster import Rasterizer
    arr = synth.make_curves(seed, W, H, no, nc, style="local").as_dict()
    cfg = bs.SampleCfg(g_open=10, rows_closed=4, k_closed=6)
    tgt = torch.as_tensor(synth.procedural_target(seed, W, H, 6), device="cuda")

    def make():
        curves = bs.CurveSet.from_arrays(arr, device="cuda")
        r = Rasterizer(bs.Canvas(W, H, 16, (0.1, 0.2, 0.3)), cfg, curves.n_open, curves.n_closed,
                       pair_capacity=256)
        return r, curves
    return make, tgt


def test_step_graph_replays_the_eager_step(bs):
    """A captured step (order, sampling, async binning, blend + L2, backward)
    gives the eager step's image, transmittance, contributor counts and
    table bit for bit; loss and gradients up to the order of their float
    atomics."""
    from paper_2503_16424_gb300.raster import StepGraph
    make, tgt = _problem(bs)
    r, curves = make()
    grad = curves.zeros_like()
    sg = StepGraph(r, curves, tgt, grad)
    sg()                 # eager, fits the capacity
    sg()                 # captured
    assert sg.graph is not None
    sg()                 # replayed
    assert sg.check() == (bs.BS_OK, r.binning.n_pairs)
    e, ce = make()
    loss, g_e = e.step(ce, tgt)
    torch.cuda.synchronize()
    for a, b in ((r.img, e.img), (r.T, e.T), (r.nc, e.nc), (r.gauss, e.gauss), (r.dimg, e.dimg)):
        assert torch.equal(a, b)
    assert abs(float(r.loss) - float(loss)) <= 1e-12 * float(loss)
    for k in KEYS:
        a, b = getattr(grad, k), getattr(g_e, k)
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * float(b.abs().max()) + 1e-30), k


def test_step_graph_grows_the_capacity_after_an_overflow(bs):
    """Curves that grow between steps overflow the captured capacity: that
    replay blends nothing and check() reports it; the next call captures
    again with room, and the step matches the eager one."""
    from paper_2503_16424_gb300.raster import StepGraph
    make, tgt = _problem(bs)
    r, curves = make()
    grad = curves.zeros_like()
    sg = StepGraph(r, curves, tgt, grad, headroom=1.0)
    sg()
    sg()
    assert sg.check()[0] == bs.BS_OK
    curves.open_width.mul_(20.0)         # wider strokes: 485 -> 2531 pairs, past 485 + 1024
    sg()
    st, n = sg.check()
    assert st == bs.BS_ERR_CAPACITY and n > 0 and sg.graph is None
    bg = torch.tensor((0.1, 0.2, 0.3), device="cuda")[:, None, None].expand_as(r.img)
    assert torch.equal(r.img, bg)
    sg()
    assert sg.check() == (bs.BS_OK, n) and sg.overflows == 1
    e, ce = make()
    ce.open_width.mul_(20.0)
    e.step(ce, tgt)
    assert torch.equal(r.img, e.img)


def test_nonfinite_records_and_gradients_set_the_status_word(bs):
    """A NaN control point gives non-finite records (bs_sample_curves); an
    infinite dL/dimg gives non-finite gradients (bs_render_bwd); either sets
    BS_ERR_NOT_FINITE, which a clear resets.  The NaN curve is never binned,
    so the image stays finite."""
    make, tgt = _problem(bs)
    assert bs.sync_status(clear=True) in (bs.BS_OK, bs.BS_ERR_NOT_FINITE)
    r, curves = make()
    r.step(curves, tgt)
    assert bs.sync_status(clear=True) == bs.BS_OK
    curves.open_ctrl[2, 4, 0] = float("nan")
    img = r.forward(curves)
    assert bs.sync_status(clear=False) == bs.BS_ERR_NOT_FINITE
    assert bool(torch.isfinite(img).all())
    assert bs.sync_status(clear=True) == bs.BS_ERR_NOT_FINITE     # still set until cleared
    assert bs.sync_status(clear=True) == bs.BS_OK
    r2, c2 = make()
    r2.forward(c2)
    dimg = torch.zeros_like(r2.img)
    dimg[0, 40, 30] = float("inf")
    r2.backward(c2, dimg)
    assert bs.sync_status(clear=True) == bs.BS_ERR_NOT_FINITE
    r2.step(c2, tgt)
    assert bs.sync_status(clear=True) == bs.BS_OK


def test_autograd_function_twice_before_one_backward(bs):
    """Two renders with different curves on one rasterizer in one loss: each
    call's gradient equals a separate rasterizer's step on its own curves."""
    from paper_2503_16424_gb300.raster import rasterize
    make, tgt = _problem(bs)
    r, cA = make()
    _, cB = make()
    cB.open_ctrl.add_(1.5)
    cB.closed_color.mul_(0.5)
    pA = bs.CurveSet(**{k: getattr(cA, k).clone().requires_grad_(True) for k in KEYS})
    pB = bs.CurveSet(**{k: getattr(cB, k).clone().requires_grad_(True) for k in KEYS})
    imgA = rasterize(r, pA)
    imgB = rasterize(r, pB)
    loss = ((imgA - tgt) ** 2).mean() + ((imgB - tgt) ** 2).mean()
    loss.backward()
    for p, c in ((pA, cA), (pB, cB)):
        e, _ = make()
        _, g = e.step(c, tgt)
        for k in KEYS:
            a, b = getattr(p, k).grad, getattr(g, k)
            assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * float(b.abs().max()) + 1e-30), k


def test_step_graph_captures_again_after_the_binning_buffers_move(bs):
    """A synchronising call between replays (here a forward whose pairs
    overflow the capacity, so the binning grows its buffers) leaves the
    captured graph pointing at freed buffers: the next call must capture
    again, and its step must equal the eager one."""
    from paper_2503_16424_gb300.raster import StepGraph
    make, tgt = _problem(bs)
    r, curves = make()
    grad = curves.zeros_like()
    sg = StepGraph(r, curves, tgt, grad, headroom=1.0)
    sg()
    sg()
    before = r.binning.allocations
    curves.open_width.mul_(20.0)         # 485 -> 2531 pairs: the forward's binning grows its buffers
    r.forward(curves)
    assert r.binning.allocations > before
    sg()
    assert sg.check()[0] == bs.BS_OK and sg.overflows == 0
    e, ce = make()
    ce.open_width.mul_(20.0)
    loss, _ = e.step(ce, tgt)
    torch.cuda.synchronize()
    assert torch.equal(r.img, e.img) and torch.equal(r.gauss, e.gauss)
    assert abs(float(r.loss) - float(loss)) <= 1e-12 * float(loss)


def test_step_graph_check_right_after_a_shrinking_fit(bs):
    """A rasterizer made with a large capacity: the first (eager) call fits
    the capacity down, which allocates a workspace no binning has written
    yet; check() at once must report the eager run's pairs, not read the
    fresh workspace, and the replays that follow must match."""
    from paper_2503_16424_gb300.raster import Rasterizer, StepGraph
    make, tgt = _problem(bs)
    _, curves = make()
    r = Rasterizer(bs.Canvas(96, 80, 16, (0.1, 0.2, 0.3)), bs.SampleCfg(g_open=10, rows_closed=4, k_closed=6),
                   curves.n_open, curves.n_closed, pair_capacity=1 << 20)
    grad = curves.zeros_like()
    sg = StepGraph(r, curves, tgt, grad)
    sg()
    before = r.binning.allocations
    st, n = sg.check()
    assert st == bs.BS_OK and 0 < n < r.binning.capacity < (1 << 20) and r.binning.allocations == before
    assert r.binning.device_status() == bs.BS_OK
    sg()
    assert sg.check() == (bs.BS_OK, n) and sg.overflows == 0
