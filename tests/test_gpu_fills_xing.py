"""The Xing loss kernel (bs_xing_loss) and linear-gradient fills of closed
curves (Appendix D) against the oracle: loss within 1e-6 relative,
gradients within 1e-3 relative; fill colours and opacities of the sampled
table within 2e-7 of the oracle's (float32 interpolation), uniform fills
bit-identical to curves without fill arrays."""

import numpy as np
import pytest
import torch

import oracle
from oracle.curves import SampleCfg as OCfg, table_from_f32
from oracle.pipeline import as_curves, sample_vjp
from oracle.xing import xing_loss as oracle_xing
from paper_2503_16424_gb300 import synth
from tests.gpu_cases import grad_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def test_xing_loss_and_gradient_match_oracle(bs):
    a = synth.make_curves(21, 200, 160, 3, 40, style="local").as_dict()
    rng = np.random.default_rng(2)
    a["closed_ctrl"] = (a["closed_ctrl"] + rng.normal(0, 8, a["closed_ctrl"].shape)).astype(np.float32)
    curves = bs.CurveSet.from_arrays(a)
    # the gradient is added to what the buffer holds: start from values of
    # its own magnitude (float32 keeps their sum exact enough)
    base = torch.as_tensor(rng.uniform(-1e-4, 1e-4, a["closed_ctrl"].shape).astype(np.float32), device="cuda")
    g = base.clone()
    loss = bs.xing_loss(curves, 0.5, g)
    t = torch.tensor(a["closed_ctrl"], dtype=torch.float64, requires_grad=True)
    L = oracle_xing(t, 0.5)
    (gref,) = torch.autograd.grad(L, t)
    assert float(L.detach()) > 0.0
    assert abs(float(loss) - float(L.detach())) <= 1e-6 * float(L.detach())
    assert grad_rel_err(g.double().cpu() - base.double().cpu(), gref) <= 1e-3


def _fill_case(seed):
    a = synth.make_curves(seed, 96, 80, 4, 6, style="local").as_dict()
    rng = np.random.default_rng(seed)
    a["closed_color2"] = rng.uniform(0, 1, (6, 3)).astype(np.float32)
    a["closed_opac2"] = rng.uniform(0.3, 1, 6).astype(np.float32)
    return a


def test_gradient_fill_sampling_and_backward_match_oracle(bs):
    a = _fill_case(31)
    cfg = bs.SampleCfg(g_open=10, rows_closed=4, k_closed=7)
    ocfg = OCfg(g_open=10, rows_closed=4, k_closed=7)
    curves = bs.CurveSet.from_arrays(a)
    _, first = bs.curve_order(curves, cfg)
    gauss = bs.sample_curves(curves, cfg, first).cpu().numpy()
    o_rank, o_first = oracle.draw_order(a["open_ctrl"], a["open_width"], a["closed_ctrl"], ocfg)
    assert np.array_equal(first.cpu().numpy(), o_first)
    tab = oracle.gaussian_table(as_curves(a), ocfg, o_first)
    assert np.abs(gauss[:, 6] - tab["o"].detach().numpy()).max() <= 2e-7
    assert np.abs(gauss[:, 7:10] - tab["col"].detach().numpy()).max() <= 2e-7
    # uniform fills: the same table as curves without fill arrays
    u = dict(a, closed_color2=a["closed_color"].copy(), closed_opac2=a["closed_opac"].copy())
    plain = {k: v for k, v in a.items() if k not in ("closed_color2", "closed_opac2")}
    g_u = bs.sample_curves(bs.CurveSet.from_arrays(u), cfg, first).cpu().numpy()
    g_p = bs.sample_curves(bs.CurveSet.from_arrays(plain), cfg, first).cpu().numpy()
    assert np.array_equal(g_u, g_p)
    # backward through the fills: per-Gaussian gradients -> curve gradients
    rng = np.random.default_rng(5)
    dg = np.zeros((gauss.shape[0], 12), np.float32)
    dg[:, :10] = rng.normal(0, 1, (gauss.shape[0], 10))
    grad = bs.sample_curves_bwd(curves, cfg, first, torch.as_tensor(dg, device="cuda"))
    keys = ("mx", "my", "ux", "uy", "isx", "isy", "o")
    dtab = {k: torch.as_tensor(dg[:, i], dtype=torch.float64) for i, k in enumerate(keys)}
    dtab["col"] = torch.as_tensor(dg[:, 7:10], dtype=torch.float64)
    ref = sample_vjp(as_curves(a), ocfg, dtab, o_first)
    for k in ("closed_color", "closed_opac", "closed_color2", "closed_opac2", "closed_ctrl", "open_ctrl"):
        e = grad_rel_err(getattr(grad, k).cpu(), ref[k])
        assert e <= 1e-3, (k, e)
