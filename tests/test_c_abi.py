"""The C ABI from plain C programs (tests/c/*.c), without Python or PyTorch
in the loop: the host-only calls (CPU) and one whole optimisation step on
the GPU, each compared with the same calls made through the Python binding.
The programs are compiled here against include/bs.h and libbs.so."""

import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from paper_2503_16424_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2503_16424_gb300")
INCLUDE = os.path.join(ROOT, "include")
KEYS = ("open_ctrl", "open_width", "open_color", "open_opac", "closed_ctrl", "closed_color", "closed_opac")


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def _compile(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr


def test_host_calls_from_c_match_the_binding(bs, tmp_path):
    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "bs_host")
    _compile([cc, "-std=c99", "-Wall", "-Werror", "-I", INCLUDE, os.path.join(ROOT, "tests", "c", "bs_host.c"),
              "-L", PKG, "-lbs", f"-Wl,-rpath,{PKG}", "-o", exe])
    svg = str(tmp_path / "out.svg")
    r = subprocess.run([exe, svg], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    out = {ln.split()[0]: ln.split()[1:] for ln in r.stdout.splitlines()}
    cfg = bs.SampleCfg(g_open=16, rows_closed=4, k_closed=8)
    assert int(out["num_gaussians"][0]) == bs.num_gaussians(5, 3, cfg) == 5 * 16 + 3 * 32
    assert int(out["num_gaussians_bad"][0]) == -1
    assert int(out["bin_workspace"][0]) == bs.bin_tiles_workspace(262144, bs.Canvas(2048, 2048, 16), 11428828)
    assert int(out["bin_workspace_bad_tile"][0]) != bs.BS_OK and out["bin_workspace_bad_tile"][1] == "1"
    sizes = bs.batch_sizes([bs.BatchImage(100, 73, 12, 6, bs.SampleCfg(12, 5, 7), (0.2, 0.5, 0.1)),
                            bs.BatchImage(256, 200, 60, 30, bs.SampleCfg(16, 4, 8, tangent_mode=1), (0.0, 0.1, 0.2))],
                           tile=16, pair_capacity=1 << 20)
    assert [int(v) for v in out["batch"]] == [sizes[k] for k in ("n_open", "n_closed", "n_gauss", "n_pixels",
                                                                  "n_tiles", "ws_bytes")]
    assert [int(v) for v in out["net_params"]] == [bs.net_param_count(0), bs.net_param_count(5)]
    # the same two curves through the binding give the same document
    oc = np.array([[3.0 + 2.5 * j, 10.0 + j % 3] for j in range(10)], np.float32)[None]
    ccl = np.array([[30.0 + 0.5 * (j * j % 7), 20.0 + 1.25 * j] for j in range(12)], np.float32)[None]
    arrays = dict(open_ctrl=oc, open_width=np.array([1.5], np.float32),
                  open_color=np.array([[0.1, 0.2, 0.3]], np.float32), open_opac=np.array([[0.9, 0.5, 0.7]], np.float32),
                  closed_ctrl=ccl, closed_color=np.array([[0.6, 0.25, 1.0]], np.float32),
                  closed_opac=np.array([0.8], np.float32))
    doc = bs.svg_export(arrays, 64, 48, rank=np.array([1, 0], np.uint32), own_opacity=True)
    with open(svg) as f:
        assert f.read() == doc
    assert int(out["svg_bytes"][0]) == len(doc.encode()) + 1


@pytest.mark.gpu
@pytest.mark.parametrize("seed,W,H,no,nc,tmode", [(21, 96, 80, 10, 5, 0), (22, 130, 70, 6, 8, 1)])
def test_a_step_from_c_matches_the_binding(bs, tmp_path, seed, W, H, no, nc, tmode):
    """Draw order, sampling, binning, blend + L2, backward through bs.h
    from C with cudaMalloc'd buffers: image and pair count equal to the
    binding's bit for bit, the loss to the order of its double sums, the
    curve gradients to the order of their float atomics."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "bs_step")
    _compile([nvcc, "-x", "c", "-I", INCLUDE, os.path.join(ROOT, "tests", "c", "bs_step.c"), "-L", PKG, "-lbs",
              "-Xlinker", f"-rpath={PKG}", "-o", exe])
    from paper_2503_16424_gb300.raster import Rasterizer
    arr = synth.make_curves(seed, W, H, no, nc, style="local").as_dict()
    tgt = synth.procedural_target(seed + 1, W, H, 6)
    cfg = bs.SampleCfg(g_open=12, rows_closed=4, k_closed=6, tangent_mode=tmode)
    bg = (0.1, 0.2, 0.3)
    inp = str(tmp_path / "in.bin")
    with open(inp, "wb") as f:
        f.write(np.array([W, H, 16, no, nc, cfg.g_open, cfg.rows_closed, cfg.k_closed, tmode], np.int32).tobytes())
        f.write(np.array([cfg.rho, cfg.cov_eps, *bg], np.float32).tobytes())
        for k in KEYS:
            f.write(np.ascontiguousarray(arr[k], np.float32).tobytes())
        f.write(np.ascontiguousarray(tgt, np.float32).tobytes())
    outp = str(tmp_path / "out.bin")
    r = subprocess.run([exe, inp, outp], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    raw = open(outp, "rb").read()
    loss_c = float(np.frombuffer(raw[:8], np.float64)[0])
    pairs_c = int(np.frombuffer(raw[8:16], np.int64)[0])
    rest = np.frombuffer(raw[16:], np.float32)
    img_c, rest = rest[:3 * H * W].reshape(3, H, W), rest[3 * H * W:]
    grads_c = {}
    for k in KEYS:
        n = np.asarray(arr[k]).size
        grads_c[k], rest = rest[:n].reshape(np.asarray(arr[k]).shape), rest[n:]
    assert rest.size == 0
    curves = bs.CurveSet.from_arrays(arr, device="cuda")
    rz = Rasterizer(bs.Canvas(W, H, 16, bg), cfg, no, nc, pair_capacity=1 << 16)
    loss, grad = rz.step(curves, torch.as_tensor(tgt, device="cuda"))
    torch.cuda.synchronize()
    assert np.array_equal(img_c, rz.img.cpu().numpy())
    assert pairs_c == rz.binning.n_pairs
    assert abs(loss_c - float(loss)) <= 1e-12 * float(loss)
    for k in KEYS:
        ref = getattr(grad, k).cpu().numpy()
        if ref.size == 0:
            continue
        scale = float(np.abs(ref).max())
        assert np.allclose(grads_c[k], ref, rtol=1e-5, atol=1e-6 * scale + 1e-30), k
