"""The C ABI library loads and exports every function include/bs.h declares;
host-side argument validation and pure host arithmetic work without a GPU
(no compute call is made here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|bs_status|int64_t)\s*(bs_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import build_lib
    build_lib.build()
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def test_header_declares_the_hot_path():
    names = declared_functions()
    for f in ("bs_sample_curves", "bs_bin_tiles", "bs_render_fwd", "bs_render_bwd", "bs_curve_order",
              "bs_l2_loss_grad", "bs_sample_curves_bwd", "bs_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol(bs):
    lib = ctypes.CDLL(bs.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_num_gaussians_host_arithmetic(bs):
    cfg = bs.SampleCfg(g_open=64, rows_closed=8, k_closed=8)
    assert bs.num_gaussians(2048, 2048, cfg) == 262144
    assert bs.num_gaussians(64, 0, bs.SampleCfg(g_open=16)) == 1024
    c = bs.SampleCfg(g_open=1).c()
    assert bs.lib.bs_num_gaussians(1, 0, ctypes.byref(c)) == -1


def test_workspace_size_host_arithmetic(bs):
    n1 = bs.bin_tiles_workspace(1000, bs.Canvas(256, 256), 10000)
    n2 = bs.bin_tiles_workspace(1000, bs.Canvas(256, 256), 20000)
    assert n2 > n1 > 10000 * 4


def test_invalid_arguments_are_rejected_on_the_host(bs):
    cfg = bs.SampleCfg(g_open=16).c()
    curves = bs.bs_curves(5, 0, None, None, None, None, None, None, None, None)
    st = bs.lib.bs_curve_order(ctypes.byref(curves), ctypes.byref(cfg), None, None, None)
    assert st == bs.BS_ERR_INVALID_ARG
    assert b"open curve arrays" in bs.lib.bs_last_error()
    cv = bs.Canvas(0, 10).c()
    nb = ctypes.c_size_t(0)
    assert bs.lib.bs_bin_tiles_workspace(10, ctypes.byref(cv), 100, ctypes.byref(nb)) == bs.BS_ERR_INVALID_ARG
    cv = bs.Canvas(64, 64, tile=12).c()
    assert bs.lib.bs_bin_tiles_workspace(10, ctypes.byref(cv), 100, ctypes.byref(nb)) == bs.BS_ERR_UNSUPPORTED
    # keys wider than 32 bits (22 tile + 20 Gaussian bits): two 64-bit key
    # buffers of the capacity in the workspace instead of one 32-bit buffer
    cv = bs.Canvas(32768, 32768).c()
    assert bs.lib.bs_bin_tiles_workspace(1 << 20, ctypes.byref(cv), 100000, ctypes.byref(nb)) == bs.BS_OK
    wide = nb.value
    cv = bs.Canvas(2048, 2048).c()
    assert bs.lib.bs_bin_tiles_workspace(1 << 18, ctypes.byref(cv), 100000, ctypes.byref(nb)) == bs.BS_OK
    assert wide - nb.value >= 100000 * (16 - 4)
    assert bs.lib.bs_status_string(bs.BS_ERR_TIMEOUT) == b"BS_ERR_TIMEOUT"
    bad = bs.SampleCfg(g_open=16, rho=0.0).c()
    assert bs.lib.bs_sample_curves(ctypes.byref(curves), ctypes.byref(bad), None, None) == bs.BS_ERR_INVALID_ARG


def test_binding_refuses_cpu_tensors(bs):
    import torch
    with pytest.raises(TypeError):
        bs.CurveSet(*(torch.zeros(0, 10, 2),) * 7).check()


def test_prune_densify_host_validation(bs):
    cv = bs.Canvas(64, 48).c()
    nb = ctypes.c_size_t(0)
    assert bs.lib.bs_prune_densify_workspace(10, 5, ctypes.byref(cv), ctypes.byref(nb)) == bs.BS_OK
    small = nb.value
    assert small >= 64 * 48 * (4 + 4 + 4)           # labels, counts, region keys
    bs.lib.bs_prune_densify_workspace(10, 5000, ctypes.byref(cv), ctypes.byref(nb))
    assert nb.value > small
    assert bs.lib.bs_prune_densify_workspace(40000, 30000, ctypes.byref(cv), ctypes.byref(nb)) == \
        bs.BS_ERR_INVALID_ARG
    cfg = bs.PDCfg().c()
    curves = bs.bs_curves_mut(3, 0, None, None, None, None, None, None, None)
    st = bs.lib.bs_prune_densify(ctypes.byref(curves), ctypes.byref(cfg), ctypes.byref(cv), None, None, None, 0,
                                 None, None, None)
    assert st == bs.BS_ERR_INVALID_ARG and b"open curve arrays" in bs.lib.bs_last_error()
    empty = bs.bs_curves_mut(0, 0, None, None, None, None, None, None, None)
    for bad in (bs.PDCfg(t_end=0), bs.PDCfg(step=-1), bs.PDCfg(new_width=0.0), bs.PDCfg(new_opacity=1.5),
                bs.PDCfg(err_thresh=float("nan"))):
        c = bad.c()
        assert bs.lib.bs_prune_densify(ctypes.byref(empty), ctypes.byref(c), ctypes.byref(cv), None, None, None,
                                       0, None, None, None) == bs.BS_ERR_INVALID_ARG
    # no image, then too small a workspace
    assert bs.lib.bs_prune_densify(ctypes.byref(empty), ctypes.byref(cfg), ctypes.byref(cv), None, None, None, 0,
                                   None, None, None) == bs.BS_ERR_INVALID_ARG
    fake = ctypes.c_void_p(1 << 20)
    assert bs.lib.bs_prune_densify(ctypes.byref(empty), ctypes.byref(cfg), ctypes.byref(cv), fake, fake, fake, 16,
                                   None, None, None) == bs.BS_ERR_INVALID_ARG
    assert b"workspace" in bs.lib.bs_last_error()


def _batch(bs, images, tile=16, capacity=100000):
    arr = (bs.bs_batch_image * len(images))(*(im.c() for im in images))
    return arr, bs.bs_batch(ctypes.cast(arr, ctypes.c_void_p), len(images), tile, capacity, None, 0)


def test_batch_plan_host_arithmetic(bs):
    images = [bs.BatchImage(300, 200, 5, 3, bs.SampleCfg(g_open=16, rows_closed=4, k_closed=8)),
              bs.BatchImage(64, 64, 0, 2, bs.SampleCfg(g_open=8, rows_closed=6, k_closed=4)),
              bs.BatchImage(1, 1, 1, 0, bs.SampleCfg(g_open=4))]
    arr, b = _batch(bs, images)
    sz = bs.bs_batch_sizes()
    assert bs.lib.bs_batch_plan(ctypes.byref(b), ctypes.byref(sz)) == bs.BS_OK
    assert (sz.n_open, sz.n_closed) == (6, 5)
    assert sz.n_gauss == 5 * 16 + 3 * 32 + 2 * 24 + 4
    assert sz.n_pixels == 300 * 200 + 64 * 64 + 1
    assert sz.n_tiles == 19 * 13 + 4 * 4 + 1
    assert sz.ws_bytes > 2 * 8 * 100000      # two 64-bit key buffers of the capacity
    arr2, b2 = _batch(bs, images, capacity=200000)
    sz2 = bs.bs_batch_sizes()
    assert bs.lib.bs_batch_plan(ctypes.byref(b2), ctypes.byref(sz2)) == bs.BS_OK
    assert sz2.ws_bytes > sz.ws_bytes


def test_batch_plan_rejects_bad_batches(bs):
    good = bs.BatchImage(32, 32, 1, 1, bs.SampleCfg())
    sz = bs.bs_batch_sizes()
    _, b = _batch(bs, [good], capacity=0)
    assert bs.lib.bs_batch_plan(ctypes.byref(b), ctypes.byref(sz)) == bs.BS_ERR_INVALID_ARG
    _, b = _batch(bs, [good, bs.BatchImage(32, 32, 1, 0, bs.SampleCfg(g_open=1))])
    assert bs.lib.bs_batch_plan(ctypes.byref(b), ctypes.byref(sz)) == bs.BS_ERR_INVALID_ARG
    assert b"image 1" in bs.lib.bs_last_error()
    _, b = _batch(bs, [bs.BatchImage(0, 32, 1, 0, bs.SampleCfg())])
    assert bs.lib.bs_batch_plan(ctypes.byref(b), ctypes.byref(sz)) == bs.BS_ERR_INVALID_ARG
    _, b = _batch(bs, [good], tile=12)
    assert bs.lib.bs_batch_plan(ctypes.byref(b), ctypes.byref(sz)) == bs.BS_ERR_UNSUPPORTED
    # a workspace smaller than the plan is refused before anything runs
    arr, b = _batch(bs, [good])
    b.ws, b.ws_bytes = ctypes.c_void_p(256), 16
    assert bs.lib.bs_batch_setup(ctypes.byref(b), None) == bs.BS_ERR_INVALID_ARG


def test_adam_rejects_bad_groups(bs):
    cfg = bs.bs_adam_cfg(0.9, 0.999, 1e-8)
    g = bs.bs_adam_group(None, None, None, None, 10, 0.1, 0.0, 1.0, None, 1)
    arr = (bs.bs_adam_group * 1)(g)
    assert bs.lib.bs_adam_step(arr, 1, ctypes.byref(cfg), ctypes.c_void_p(256), None) == bs.BS_ERR_INVALID_ARG
    assert bs.lib.bs_adam_step(arr, 0, ctypes.byref(cfg), ctypes.c_void_p(256), None) == bs.BS_ERR_INVALID_ARG
    bad = bs.bs_adam_cfg(1.0, 0.999, 1e-8)
    ok = (bs.bs_adam_group * 1)(bs.bs_adam_group(None, None, None, None, 0, 0.1, 0.0, 1.0, None, 1))
    assert bs.lib.bs_adam_step(ok, 1, ctypes.byref(bad), ctypes.c_void_p(256), None) == bs.BS_ERR_INVALID_ARG


def test_net_host_arithmetic_and_validation(bs):
    """The head holds 64 outputs of 256 features; a training step refuses a
    missing target array before it touches the device."""
    assert bs.lib.bs_net_param_count(5) == 64 * 256 + 64
    assert bs.lib.bs_net_param_count(0) == 32 * 16 * 8 + 32
    assert bs.lib.bs_net_param_count(6) == -1
    fake = ctypes.c_void_p(256)
    net = bs.bs_net((ctypes.c_void_p * bs.NET_LAYERS)(*([fake.value] * bs.NET_LAYERS)),
                    (ctypes.c_void_p * bs.NET_LAYERS)(*([fake.value] * bs.NET_LAYERS)))
    grad = bs.bs_net_grad((ctypes.c_void_p * bs.NET_LAYERS)(*([fake.value] * bs.NET_LAYERS)))
    tgt = bs.bs_net_curves(**{k: fake.value for k in bs.NET_CURVE_KEYS})
    tgt.open_width = None
    st = bs.lib.bs_net_train_step(ctypes.byref(net), fake, 1, 64, ctypes.byref(tgt), fake, 1 << 30,
                                  ctypes.byref(grad), fake, None)
    assert st == bs.BS_ERR_INVALID_ARG and b"target" in bs.lib.bs_last_error()
    st = bs.lib.bs_net_train_step(ctypes.byref(net), fake, 1, 48, ctypes.byref(tgt), fake, 1 << 30,
                                  ctypes.byref(grad), fake, None)
    assert st == bs.BS_ERR_INVALID_ARG    # side not a multiple of 32
