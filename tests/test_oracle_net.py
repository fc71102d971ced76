"""Pins of the network oracle (the learned initialiser's proposal network):
the convolution against a brute-force loop over the library's weight
layout, the head's curve mapping in closed form, and the gradients against
central finite differences."""

import numpy as np
import torch

from oracle import net


def _weights(rng, scale=0.2):
    out = []
    for l in range(6):
        cin, cout, k = (net.CH[l], net.CH[l + 1], 4) if l < 5 else (256, net.HEAD, 1)
        out.append(rng.normal(0, scale / np.sqrt(k * k * cin), cout * k * k * cin + cout).astype(np.float32))
    return out


def test_conv_matches_brute_force_on_the_library_layout():
    rng = np.random.default_rng(0)
    cin, cout, H = 8, 4, 6
    w = rng.normal(size=(cout, 4, 4, cin))          # [Cout][ky][kx][Cin]
    b = rng.normal(size=cout)
    x = rng.normal(size=(1, cin, H, H))
    kern = torch.as_tensor(w).permute(0, 3, 1, 2)
    got = net.conv_layer(torch.as_tensor(x), kern, torch.as_tensor(b), 2, 1).numpy()
    ref = np.zeros((1, cout, H // 2, H // 2))
    for co in range(cout):
        for oy in range(H // 2):
            for ox in range(H // 2):
                acc = b[co]
                for ky in range(4):
                    for kx in range(4):
                        iy, ix = 2 * oy + ky - 1, 2 * ox + kx - 1
                        if 0 <= iy < H and 0 <= ix < H:
                            acc += np.dot(w[co, ky, kx, :], x[0, :, iy, ix])
                ref[0, co, oy, ox] = acc
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_unpack_reads_kernel_then_bias():
    rng = np.random.default_rng(1)
    w = _weights(rng)
    p = net.unpack(w)
    nw = 32 * 16 * 8
    assert torch.equal(p[0][0].permute(0, 2, 3, 1).reshape(-1), torch.as_tensor(w[0][:nw], dtype=torch.float64))
    assert torch.equal(p[0][1], torch.as_tensor(w[0][nw:], dtype=torch.float64))


def test_head_mapping_closed_form():
    head = torch.zeros(1, 4, net.HEAD, dtype=torch.float64)
    head[0, 3, 0] = np.arctanh(0.5)          # P_0.x of cell 3 (row 1, column 1 of a 64 x 64 patch)
    head[0, 3, 27] = np.log(3.0)             # opacity 3 / 4
    head[0, 2, 28 + 19] = np.arctanh(-0.25)  # Q_9.y of cell 2 (row 1, column 0)
    head[0, 1, 48] = np.log(3.0)             # width 3/4 of the largest
    head[0, 1, 53] = -np.log(3.0)            # middle segment opacity 1 / 4
    p = net.head_curves(head, 64)
    assert torch.allclose(p["ctrl"][0, 0], torch.tensor([[16.0, 16.0]] * 12, dtype=torch.float64))
    assert abs(float(p["ctrl"][0, 3, 0, 0]) - (48.0 + 0.5 * net.REACH)) < 1e-12
    assert abs(float(p["ctrl"][0, 3, 0, 1]) - 48.0) < 1e-12
    assert torch.allclose(p["color"], torch.full_like(p["color"], 0.5))
    assert abs(float(p["opac"][0, 3]) - 0.75) < 1e-12
    # the open stroke: zero outputs give the cell centre, half the largest width, grey, 0.5
    assert torch.allclose(p["open_ctrl"][0, 0], torch.tensor([[16.0, 16.0]] * 10, dtype=torch.float64))
    assert abs(float(p["open_ctrl"][0, 2, 9, 1]) - (48.0 - 0.25 * net.REACH)) < 1e-12
    assert abs(float(p["open_ctrl"][0, 2, 9, 0]) - 16.0) < 1e-12
    assert abs(float(p["open_width"][0, 0]) - 0.5 * net.WIDTH_MAX) < 1e-12
    assert abs(float(p["open_width"][0, 1]) - 0.75 * net.WIDTH_MAX) < 1e-12
    assert torch.allclose(p["open_color"], torch.full_like(p["open_color"], 0.5))
    assert abs(float(p["open_opac"][0, 1, 1]) - 0.25) < 1e-12 and abs(float(p["open_opac"][0, 1, 0]) - 0.5) < 1e-12


def test_loss_closed_form():
    """Zero outputs against targets one reach (or one largest width, one
    unit) away in every term give the count of terms per cell."""
    head = torch.zeros(1, 1, net.HEAD, dtype=torch.float64)
    p = net.head_curves(head, 32)
    t = dict(ctrl=p["ctrl"] + net.REACH, color=p["color"] + 1.0, opac=p["opac"] + 1.0,
             open_ctrl=p["open_ctrl"] - net.REACH, open_width=p["open_width"] + net.WIDTH_MAX,
             open_color=p["open_color"] - 1.0, open_opac=p["open_opac"] + 1.0)
    assert abs(float(net.loss(head, 32, t)) - (24 + 3 + 1 + 20 + 1 + 3 + 3)) < 1e-12


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    w = _weights(rng, scale=1.0)
    x = rng.uniform(0, 1, (2, 3, 32, 32))
    t = dict(ctrl=rng.uniform(0, 32, (2, 1, 12, 2)), color=rng.uniform(0, 1, (2, 1, 3)), opac=rng.uniform(0, 1, (2, 1)),
             open_ctrl=rng.uniform(0, 32, (2, 1, 10, 2)), open_width=rng.uniform(0.5, 6, (2, 1)),
             open_color=rng.uniform(0, 1, (2, 1, 3)), open_opac=rng.uniform(0, 1, (2, 1, 3)))
    L, g = net.loss_and_grads(w, x, t)
    w64 = [a.astype(np.float64) for a in w]

    def f(ws):
        head, _ = net.forward(net.unpack(ws), x)
        return float(net.loss(head, 32, t))
    assert abs(f(w64) - L) < 1e-12
    checked = 0
    for l in (0, 2, 4, 5):
        gl = g[l]
        order = np.argsort(-np.abs(gl))[:3]      # the largest entries: well above the FD noise
        for i in order:
            h = 1e-6
            wp = [a.copy() for a in w64]
            wm = [a.copy() for a in w64]
            wp[l][i] += h
            wm[l][i] -= h
            fd = (f(wp) - f(wm)) / (2 * h)
            assert abs(fd - gl[i]) <= 1e-5 * max(1.0, abs(gl[i])), (l, i, fd, gl[i])
            checked += 1
    assert checked == 12
