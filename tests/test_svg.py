"""SVG export (Appendix C, Algorithm 2) through the library's host-only
call: every path reproduces its curve's control points exactly (float32
read back from 9 significant digits), the commands follow Algorithm 2, the
colours are rgb(round(255 c)), and the document is ordered back to front."""

import re
import xml.etree.ElementTree as ET

import numpy as np
import pytest

from paper_2503_16424_gb300 import synth

NS = "{http://www.w3.org/2000/svg}"


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import build_lib
    build_lib.build()
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def _numbers(d):
    return [float(x) for x in re.findall(r"[-+0-9.eE]+", d)]


def test_closed_and_open_paths_follow_algorithm_2(bs):
    a = synth.make_curves(5, 300, 200, 4, 6, style="local").as_dict()
    rank = np.random.default_rng(0).permutation(10).astype(np.uint32)
    doc = bs.svg_export(a, 300, 200, rank=rank)
    root = ET.fromstring(doc)
    assert root.get("width") == "300" and root.get("height") == "200"
    paths = root.findall(NS + "path")
    assert len(paths) == 10
    # back to front: descending rank
    order = np.argsort(-rank.astype(np.int64), kind="stable")
    for p, idx in zip(paths, order):
        d = p.get("d")
        if idx < 4:
            P = a["open_ctrl"][idx]
            cmds = re.findall(r"[MCZ]", d)
            assert cmds == ["M", "C", "C", "C"]
            assert np.array_equal(np.float32(_numbers(d)), P.reshape(-1))
            assert p.get("fill") == "none"
            col = np.rint(255 * np.clip(a["open_color"][idx], 0, 1)).astype(int)
            assert p.get("stroke") == "rgb(%d,%d,%d)" % tuple(col)
            assert np.float32(p.get("stroke-width")) == np.float32(2) * a["open_width"][idx]
        else:
            j = idx - 4
            P = a["closed_ctrl"][j]
            assert re.findall(r"[MCZ]", d) == ["M", "C", "C", "C", "C", "Z"]
            ring = np.concatenate([P, P[:1]], 0).reshape(-1)          # P0 .. P11, P0
            assert np.array_equal(np.float32(_numbers(d)), ring)
            col = np.rint(255 * np.clip(a["closed_color"][j], 0, 1)).astype(int)
            assert p.get("fill") == "rgb(%d,%d,%d)" % tuple(col)
            assert p.get("fill-opacity") == "1"


def test_gradient_fills_and_own_opacity(bs):
    a = synth.make_curves(6, 120, 90, 0, 3, style="local").as_dict()
    rng = np.random.default_rng(1)
    a["closed_color2"] = rng.uniform(0, 1, (3, 3)).astype(np.float32)
    a["closed_opac2"] = rng.uniform(0.3, 1, 3).astype(np.float32)
    doc = bs.svg_export(a, 120, 90, own_opacity=True)
    root = ET.fromstring(doc)
    grads = root.find(NS + "defs").findall(NS + "linearGradient")
    assert len(grads) == 3
    for j, g in enumerate(grads):
        P = a["closed_ctrl"][j]
        assert [np.float32(g.get(k)) for k in ("x1", "y1", "x2", "y2")] == [P[0, 0], P[0, 1], P[6, 0], P[6, 1]]
        s0, s1 = g.findall(NS + "stop")
        c0 = np.rint(255 * a["closed_color"][j]).astype(int)
        c1 = np.rint(255 * a["closed_color2"][j]).astype(int)
        assert s0.get("stop-color") == "rgb(%d,%d,%d)" % tuple(c0)
        assert s1.get("stop-color") == "rgb(%d,%d,%d)" % tuple(c1)
        assert np.float32(s0.get("stop-opacity")) == a["closed_opac"][j]
        assert np.float32(s1.get("stop-opacity")) == a["closed_opac2"][j]
    for j, p in enumerate(root.findall(NS + "path")):
        assert p.get("fill") == "url(#f%d)" % j


def test_size_query_and_small_buffer(bs):
    import ctypes
    a = synth.make_curves(7, 64, 64, 2, 2, style="local").as_dict()
    doc = bs.svg_export(a, 64, 64)
    c = bs.bs_curves(2, 2, *(ctypes.c_void_p(np.ascontiguousarray(a[k]).ctypes.data) for k in bs.CURVE_FIELDS))
    need = ctypes.c_size_t(0)
    buf = ctypes.create_string_buffer(8)
    assert bs.lib.bs_svg_export(ctypes.byref(c), None, 64, 64, 0, buf, 8, ctypes.byref(need)) == bs.BS_ERR_INVALID_ARG
    assert need.value == len(doc) + 1
