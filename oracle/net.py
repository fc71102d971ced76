"""The learned initialiser's proposal network in float64 (not in the paper;
the network the library's bs_net_* calls run).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Weights come in the library's layout: layer l's float32 array holds the
kernel [Cout][ky][kx][Cin] and then the bias [Cout].  Layers 0..4 are 4 x 4
convolutions of stride 2 and padding 1 with ReLU (channels 8, 32, 64, 128,
256, 256; the RGB input padded with zero channels to 8), layer 5 a 1 x 1
head to 32 outputs.  The convolution itself is torch's conv2d on the CPU (a
library primitive), pinned against a brute-force loop in the tests.  The
head's 28 used outputs o of cell c (centre (cx, cy)) map to a closed curve:
P_j = (cx, cy) + reach tanh(o_2j, o_2j+1), colour sigmoid(o_24..26),
opacity sigmoid(o_27).  The loss against target curves is
L = mean over cells of [sum_j |P_j - P*_j|^2 / reach^2 + |c - c*|^2 + (a - a*)^2].
Gradients by autograd.  With round_bf16 the input, the weights and every
activation are rounded to bfloat16 where the library stores them in
bfloat16, so that only the summation precision differs.
"""

from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CH = (8, 32, 64, 128, 256, 256)
HEAD = 32
REACH = 24.0
CELL = 32


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
    """Head outputs [n, cells, 32] (cells row-major) and the activations."""
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
    head = conv_layer(x, kern, bias, 1, 0)                   # [n, 32, g, g]
    return head.permute(0, 2, 3, 1).reshape(n, -1, HEAD), acts


def head_curves(head, side):
    """ctrl [n, cells, 12, 2], color [n, cells, 3], opac [n, cells]."""
    g = side // CELL
    gy, gx = torch.meshgrid(torch.arange(g, dtype=torch.float64), torch.arange(g, dtype=torch.float64),
                            indexing="ij")
    centre = torch.stack([(gx.reshape(-1) + 0.5) * CELL, (gy.reshape(-1) + 0.5) * CELL], -1)   # [cells, 2]
    ctrl = centre[None, :, None, :] + REACH * torch.tanh(head[..., :24].reshape(head.shape[0], -1, 12, 2))
    return ctrl, torch.sigmoid(head[..., 24:27]), torch.sigmoid(head[..., 27])


def loss(head, side, t_ctrl, t_color, t_opac):
    ctrl, color, opac = head_curves(head, side)
    t_ctrl = torch.as_tensor(np.asarray(t_ctrl), dtype=torch.float64)
    t_color = torch.as_tensor(np.asarray(t_color), dtype=torch.float64)
    t_opac = torch.as_tensor(np.asarray(t_opac), dtype=torch.float64)
    per = ((ctrl - t_ctrl) ** 2).sum((-1, -2)) / REACH ** 2 + ((color - t_color) ** 2).sum(-1) + (opac - t_opac) ** 2
    return per.mean()


def loss_and_grads(weights, patches, t_ctrl, t_color, t_opac, round_bf16=False):
    """L and dL/d(master array of every layer), in the library's layout."""
    params = unpack(weights, round_bf16)
    leaves = []
    for kern, bias in params:
        kern.requires_grad_(True)
        bias.requires_grad_(True)
        leaves += [kern, bias]
    side = int(np.asarray(patches).shape[-1]) if not torch.is_tensor(patches) else int(patches.shape[-1])
    head, _ = forward(params, patches, round_bf16)
    L = loss(head, side, t_ctrl, t_color, t_opac)
    grads = torch.autograd.grad(L, leaves)
    out = []
    for l in range(6):
        gk, gb = grads[2 * l], grads[2 * l + 1]
        out.append(np.concatenate([gk.permute(0, 2, 3, 1).reshape(-1).numpy(), gb.numpy()]))
    return float(L.detach()), out
