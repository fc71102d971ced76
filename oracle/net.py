"""The learned initialiser's proposal network in float64 (not in the paper;
the network the library's bs_net_* calls run).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Weights come in the library's layout: layer l's float32 array holds the
kernel [Cout][ky][kx][Cin] and then the bias [Cout].  Layers 0..4 are 4 x 4
convolutions of stride 2 and padding 1 with ReLU (channels 8, 32, 64, 128,
256, 256; the RGB input padded with zero channels to 8), layer 5 a 1 x 1
head to 64 outputs.  The convolution itself is torch's conv2d on the CPU (a
library primitive), pinned against a brute-force loop in the tests.  The
head's outputs o of cell c (centre (cx, cy)) map to one closed curve and one
open stroke (Section 3.2's two kinds):
  closed  P_j = (cx, cy) + reach tanh(o_2j, o_2j+1) (j < 12),
          colour sigmoid(o_24..26), opacity sigmoid(o_27);
  open    Q_j = (cx, cy) + reach tanh(o_28+2j, o_29+2j) (j < 10),
          width WIDTH_MAX sigmoid(o_48), colour sigmoid(o_49..51),
          segment opacities sigmoid(o_52..54);
outputs 55..63 are unused.  The loss against target curves is the mean
over cells of
  sum_j |P_j - P*_j|^2 / reach^2 + |c - c*|^2 + (a - a*)^2
  + sum_j |Q_j - Q*_j|^2 / reach^2 + (w - w*)^2 / WIDTH_MAX^2 + |c' - c'*|^2
  + sum_s (a'_s - a'*_s)^2.
Gradients by autograd.  With round_bf16 the input, the weights and every
activation are rounded to bfloat16 where the library stores them in
bfloat16, so that only the summation precision differs.
"""

from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CH = (8, 32, 64, 128, 256, 256)
HEAD = 64
REACH = 24.0
WIDTH_MAX = 8.0
CELL = 32
CURVE_KEYS = ("ctrl", "color", "opac", "open_ctrl", "open_width", "open_color", "open_opac")


def _bf16(x):
    return x.to(torch.bfloat16).to(torch.float64)


def unpack(weights, round_bf16=False):
    """List of (kernel [Cout][Cin][k][k], bias [Cout]) float64 tensors."""
    out = []
    for l, w in enumerate(weights):
        w = torch.as_tensor(np.asarray(w), dtype=torch.float64)
        if l < 5:
            cin, cout, k = CH[l], CH[l + 1], 4
        else:
            cin, cout, k = 256, HEAD, 1
        nw = cout * k * k * cin
        kern = w[:nw].reshape(cout, k, k, cin).permute(0, 3, 1, 2).contiguous()
        if round_bf16:
            kern = _bf16(kern)
        out.append((kern, w[nw:nw + cout].clone()))
    return out


def conv_layer(x, kern, bias, stride, pad):
    return F.conv2d(x, kern, bias, stride=stride, padding=pad)


def forward(params, patches, round_bf16=False):
    """Head outputs [n, cells, HEAD] (cells row-major) and the activations."""
    x = torch.as_tensor(np.asarray(patches), dtype=torch.float64) if not torch.is_tensor(patches) else patches.double()
    n, _, H, W = x.shape
    x = torch.cat([x, torch.zeros(n, CH[0] - 3, H, W, dtype=torch.float64)], 1)
    if round_bf16:
        x = _bf16(x)
    acts = [x]
    for l in range(5):
        kern, bias = params[l]
        x = torch.relu(conv_layer(x, kern, bias, 2, 1))
        if round_bf16:
            x = _bf16(x)
        acts.append(x)
    kern, bias = params[5]
    head = conv_layer(x, kern, bias, 1, 0)                   # [n, HEAD, g, g]
    return head.permute(0, 2, 3, 1).reshape(n, -1, HEAD), acts


def head_curves(head, side):
    """The proposals of head outputs [n, cells, 64]: dict of ctrl [n, cells,
    12, 2], color [n, cells, 3], opac [n, cells] (the closed curve) and
    open_ctrl [n, cells, 10, 2], open_width [n, cells], open_color [n,
    cells, 3], open_opac [n, cells, 3] (the open stroke), patch pixels."""
    g = side // CELL
    gy, gx = torch.meshgrid(torch.arange(g, dtype=torch.float64), torch.arange(g, dtype=torch.float64),
                            indexing="ij")
    centre = torch.stack([(gx.reshape(-1) + 0.5) * CELL, (gy.reshape(-1) + 0.5) * CELL], -1)   # [cells, 2]
    n = head.shape[0]
    return dict(ctrl=centre[None, :, None, :] + REACH * torch.tanh(head[..., :24].reshape(n, -1, 12, 2)),
                color=torch.sigmoid(head[..., 24:27]), opac=torch.sigmoid(head[..., 27]),
                open_ctrl=centre[None, :, None, :] + REACH * torch.tanh(head[..., 28:48].reshape(n, -1, 10, 2)),
                open_width=WIDTH_MAX * torch.sigmoid(head[..., 48]),
                open_color=torch.sigmoid(head[..., 49:52]), open_opac=torch.sigmoid(head[..., 52:55]))


def loss(head, side, targets: dict):
    """The mean over cells of the squared distances to the target curves
    (control points in units of the reach, widths of WIDTH_MAX)."""
    p = head_curves(head, side)
    t = {k: torch.as_tensor(np.asarray(targets[k]), dtype=torch.float64) for k in CURVE_KEYS}
    per = (((p["ctrl"] - t["ctrl"]) ** 2).sum((-1, -2)) / REACH ** 2 + ((p["color"] - t["color"]) ** 2).sum(-1)
           + (p["opac"] - t["opac"]) ** 2
           + ((p["open_ctrl"] - t["open_ctrl"]) ** 2).sum((-1, -2)) / REACH ** 2
           + (p["open_width"] - t["open_width"]) ** 2 / WIDTH_MAX ** 2
           + ((p["open_color"] - t["open_color"]) ** 2).sum(-1) + ((p["open_opac"] - t["open_opac"]) ** 2).sum(-1))
    return per.mean()


def loss_and_grads(weights, patches, targets: dict, round_bf16=False):
    """L and dL/d(master array of every layer), in the library's layout."""
    params = unpack(weights, round_bf16)
    leaves = []
    for kern, bias in params:
        kern.requires_grad_(True)
        bias.requires_grad_(True)
        leaves += [kern, bias]
    side = int(np.asarray(patches).shape[-1]) if not torch.is_tensor(patches) else int(patches.shape[-1])
    head, _ = forward(params, patches, round_bf16)
    L = loss(head, side, targets)
    grads = torch.autograd.grad(L, leaves)
    out = []
    for l in range(6):
        gk, gb = grads[2 * l], grads[2 * l + 1]
        out.append(np.concatenate([gk.permute(0, 2, 3, 1).reshape(-1).numpy(), gb.numpy()]))
    return float(L.detach()), out
