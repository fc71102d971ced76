"""Learned initialisation of curves: a convolutional proposal network
(bs_net_* calls) trained on curve sets the method itself optimised.

Pairs.  A pair is a procedural 256 x 256 patch and the 64 closed curves and
64 open strokes the method reaches on it from the baseline initialisation,
one of each per 32 x 32 cell: the circle of Section 4.1 (radius 10 px) and a
horizontal stroke through the cell centre (20 px long, width 2 px), both in
the cell's mean target colour at opacity 0.8, after `steps` Adam steps of
the batched path (64 patches per batch, one CUDA-graph replay per step).
Curve i of either kind stays the curve of cell i, which gives the network a
fixed slot per cell.

Network.  bs.h describes it: five stride-2 4 x 4 convolutions and a 1 x 1
head, bf16 tensor-core GEMMs with float32 accumulation; the head's bias
starts at the baseline initialisation, so an untrained network proposes
exactly the baseline curves (with colour 0.5).  Training minimises the
mean squared distance to the optimised curves (control points in units of
the 24 px reach, widths of the 8 px largest width) with Adam
(bs_adam_step) on float32 master weights.

Use.  A large target is cut into 256 x 256 patches; each patch's proposals,
shifted to the patch's place, initialise the method on the whole image.
Without the network the same image starts from the baseline curves.
"""

from __future__ import annotations

import math

import numpy as np
import torch

from . import bs, synth
from .batch import AdamCfg, BatchOptimizer, BatchRasterizer, CurveAdam

SIDE = 256
CELL = 32
GRID = SIDE // CELL
CELLS = GRID * GRID
RADIUS = 10.0
OPACITY = 0.8
STROKE_HALF = 10.0    # the baseline stroke runs from x - 10 to x + 10 px
STROKE_WIDTH = 2.0
# pair generation: a faster control-point step than the paper's 15k-step
# schedule, so that a few hundred steps move the curves (same for both arms
# of the evaluation)
PAIR_ADAM = AdamCfg(lr_ctrl=2e-3, lr_color=0.01, lr_opac=0.025)
KERNEL_CH = (8, 32, 64, 128, 256, 256)


def circle_points(cx, cy, r):
    """12 control points on the circle of radius r around (cx, cy) at angles
    2 pi j / 12: a closed curve of four cubic segments (P12 = P0)."""
    a = 2.0 * np.pi * np.arange(12) / 12.0
    return np.stack([cx[..., None] + r * np.cos(a), cy[..., None] + r * np.sin(a)], -1)


def stroke_points(cx, cy, half):
    """10 control points evenly along the horizontal segment from
    (cx - half, cy) to (cx + half, cy): an open curve of three segments."""
    x = half * (2.0 * np.arange(10) / 9.0 - 1.0)
    return np.stack([cx[..., None] + x, np.broadcast_to(cy[..., None], cy.shape + (10,))], -1)


def baseline_init(n_patches: int, side: int = SIDE, target: np.ndarray = None) -> dict:
    """The baseline curves of n patches of side `side` (curves patch by
    patch, cells row-major; keys bs.NET_CURVE_KEYS, float32 [n cells, ...],
    patch pixels): per cell a circle and a stroke, colours the cells' mean
    target colours (0.5 without a target)."""
    g = side // CELL
    gy, gx = np.meshgrid(np.arange(g), np.arange(g), indexing="ij")
    cx = np.broadcast_to((gx.reshape(-1) + 0.5) * CELL, (n_patches, g * g))
    cy = np.broadcast_to((gy.reshape(-1) + 0.5) * CELL, (n_patches, g * g))
    m = n_patches * g * g
    if target is None:
        color = np.full((m, 3), 0.5, np.float32)
    else:
        t = np.asarray(target, dtype=np.float64).reshape(n_patches, 3, g, CELL, g, CELL)
        color = np.clip(t.mean(axis=(3, 5)), 0.0, 1.0).transpose(0, 2, 3, 1).reshape(-1, 3).astype(np.float32)
    return dict(ctrl=circle_points(cx, cy, RADIUS).reshape(m, 12, 2).astype(np.float32), color=color,
                opac=np.full(m, OPACITY, np.float32),
                open_ctrl=stroke_points(cx, cy, STROKE_HALF).reshape(m, 10, 2).astype(np.float32),
                open_width=np.full(m, STROKE_WIDTH, np.float32), open_color=color.copy(),
                open_opac=np.full((m, 3), OPACITY, np.float32))


def _curve_set(d: dict, device):
    """CurveSet of a dict of bs.NET_CURVE_KEYS arrays (flat over curves)."""
    a = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in d.items()}
    return bs.CurveSet.from_arrays(dict(open_ctrl=a["open_ctrl"], open_width=a["open_width"],
                                        open_color=a["open_color"], open_opac=a["open_opac"],
                                        closed_ctrl=a["ctrl"], closed_color=a["color"], closed_opac=a["opac"]),
                                   device=device)


_POOL = None


def _target(args):
    seed, n_shapes = args
    return synth.procedural_target(seed, SIDE, SIDE, n_shapes)


def _targets(seeds, n_shapes, workers):
    """Procedural patches, drawn by a process pool when workers > 1 (spawned
    processes: they share nothing with this process's CUDA context)."""
    global _POOL
    if workers <= 1 or len(seeds) < 8:
        return np.stack([_target((s, n_shapes)) for s in seeds])
    if _POOL is None:
        import multiprocessing as mp
        _POOL = mp.get_context("spawn").Pool(workers)
    return np.stack(_POOL.map(_target, [(s, n_shapes) for s in seeds], chunksize=max(1, len(seeds) // workers)))


PAIR_KEYS = ("patches",) + bs.NET_CURVE_KEYS
_FROM_SET = dict(ctrl="closed_ctrl", color="closed_color", opac="closed_opac", open_ctrl="open_ctrl",
                 open_width="open_width", open_color="open_color", open_opac="open_opac")


def make_pairs(n: int, seed: int, steps: int = 200, n_shapes: int = 6, device="cuda", batch: int = 64,
               sample=(4, 8, 8), workers: int = 0):
    """n (patch, optimised curves) pairs.  Returns device tensors patches
    [n, 3, 256, 256] and the curves [n, 64, ...] under bs.NET_CURVE_KEYS;
    control points clamped to the network's reach around their cell, widths
    into the network's range.  sample: (rows, k) of the closed curves and
    the samples per open segment.  workers: host processes drawing the
    patches (0: the host's cores)."""
    import os
    workers = workers or min(16, os.cpu_count() or 1)
    rows, kc, g_open = sample
    out = {k: [] for k in PAIR_KEYS}
    for b0 in range(0, n, batch):
        m = min(batch, n - b0)
        tg = _targets([seed * 100003 + b0 + i for i in range(m)], n_shapes, workers)
        curves = _curve_set(baseline_init(m, SIDE, tg), device)
        images = [bs.BatchImage(SIDE, SIDE, CELLS, CELLS, bs.SampleCfg(g_open=g_open, rows_closed=rows, k_closed=kc))
                  for _ in range(m)]
        target = torch.as_tensor(tg.reshape(-1), device=device)
        r = BatchRasterizer(images, pair_capacity=1 << 22, device=device)
        opt = BatchOptimizer(r, curves, target, cfg=PAIR_ADAM, graph=True, check_every=0)
        for _ in range(steps):
            opt.step()
        out["patches"].append(torch.as_tensor(tg, device=device))
        for k in bs.NET_CURVE_KEYS:
            v = getattr(curves, _FROM_SET[k])
            out[k].append(v.view((m, CELLS) + tuple(v.shape[1:])).clone())
    res = {k: torch.cat(v, 0) for k, v in out.items()}
    g = torch.arange(GRID, device=device, dtype=torch.float32)
    cy, cx = torch.meshgrid((g + 0.5) * CELL, (g + 0.5) * CELL, indexing="ij")
    centre = torch.stack([cx.reshape(-1), cy.reshape(-1)], -1)[None, :, None, :]
    lim = 0.98 * bs.NET_REACH
    for k in ("ctrl", "open_ctrl"):
        res[k] = (centre + (res[k] - centre).clamp(-lim, lim)).contiguous()
    res["open_width"] = res["open_width"].clamp(0.02 * bs.NET_WIDTH_MAX, 0.98 * bs.NET_WIDTH_MAX).contiguous()
    return res


def initial_weights(seed: int = 0):
    """The master arrays of the six layers (float32, the library's layout):
    He-uniform convolutions, a small random head whose bias is the baseline
    initialisation (so that a zero feature map proposes the baseline curves
    with colour 0.5)."""
    rng = np.random.default_rng(seed)
    out = []
    for l in range(bs.NET_LAYERS):
        n = bs.net_param_count(l)
        if l < 5:
            cin, cout, ks = KERNEL_CH[l], KERNEL_CH[l + 1], 4
            fan_in = ks * ks * (3 if l == 0 else cin)
        else:
            cin, cout, ks, fan_in = 256, 64, 1, 256
        nw = cout * ks * ks * cin
        bound = math.sqrt(6.0 / fan_in) * (0.1 if l == 5 else 1.0)
        w = np.zeros(n, np.float32)
        w[:nw] = rng.uniform(-bound, bound, nw)
        if l == 0:   # the padding channels 3..7 of the input carry nothing
            w[:nw].reshape(cout, ks, ks, cin)[..., 3:] = 0.0
        if l == 5:
            a = 2.0 * np.pi * np.arange(12) / 12.0
            off = RADIUS / bs.NET_REACH
            b = w[nw:]
            b[0:24:2] = np.arctanh(off * np.cos(a))
            b[1:24:2] = np.arctanh(off * np.sin(a))
            b[27] = math.log(OPACITY / (1.0 - OPACITY))
            b[28:48:2] = np.arctanh(STROKE_HALF / bs.NET_REACH * (2.0 * np.arange(10) / 9.0 - 1.0))
            b[48] = math.log(STROKE_WIDTH / (bs.NET_WIDTH_MAX - STROKE_WIDTH))
            b[52:55] = math.log(OPACITY / (1.0 - OPACITY))
        out.append(w)
    return out


class InitNet:
    """The proposal network: float32 master weights, their bf16 copies,
    gradients and Adam state, on the device."""

    def __init__(self, device="cuda", seed: int = 0, lr: float = 1e-3):
        self.device = device
        self.w = [torch.as_tensor(w, device=device) for w in initial_weights(seed)]
        self.w_bf16 = [torch.empty(bs.net_param_count(l) - (64 if l == 5 else KERNEL_CH[l + 1]), dtype=torch.int16,
                                   device=device) for l in range(bs.NET_LAYERS)]
        self.g = [torch.zeros_like(w) for w in self.w]
        self.m = [torch.zeros_like(x) for x in self.w]
        self.v = [torch.zeros_like(x) for x in self.w]
        self.t = torch.zeros(1, dtype=torch.int32, device=device)
        self.groups = [bs.AdamGroup(p, g, m, v, lr) for p, g, m, v in zip(self.w, self.g, self.m, self.v)]
        self.loss = torch.zeros((), dtype=torch.float64, device=device)
        self._ws = {}
        bs.net_sync_weights(self.w, self.w_bf16)

    def ws(self, n: int, side: int = SIDE):
        key = (n, side)
        if key not in self._ws:
            self._ws[key] = torch.empty(bs.net_workspace(n, side), dtype=torch.uint8, device=self.device)
        return self._ws[key]

    def propose(self, patches: torch.Tensor) -> dict:
        """The proposals of patches [n, 3, side, side]: bs.NET_CURVE_KEYS ->
        [n, cells, ...] (patch pixels)."""
        n, side = int(patches.shape[0]), int(patches.shape[-1])
        cells = (side // CELL) ** 2
        out = {k: torch.empty((n, cells) + shape, device=self.device) for k, shape in bs.NET_CURVE_SHAPES.items()}
        bs.net_forward(self.w, self.w_bf16, patches.contiguous(), self.ws(n, side), curves=out)
        return out

    def train_step(self, patches, targets: dict):
        """Forward, backward, Adam, bf16 copies; the loss (device double)."""
        n, side = int(patches.shape[0]), int(patches.shape[-1])
        bs.net_train_step(self.w, self.w_bf16, self.g, patches, targets, self.ws(n, side), self.loss)
        bs.adam_step(self.groups, self.t)
        bs.net_sync_weights(self.w, self.w_bf16)
        return self.loss


def train(net: InitNet, data: dict, steps: int, batch: int = 64, seed: int = 0):
    """steps minibatch steps over the pairs (sampled with replacement);
    returns the loss of every step (synchronises once at the end)."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = int(data["patches"].shape[0])
    losses = torch.empty(steps, dtype=torch.float64, device=net.device)
    for i in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=gen).to(net.device)
        b = {k: data[k].index_select(0, idx).contiguous() for k in PAIR_KEYS}
        losses[i] = net.train_step(b.pop("patches"), b)
    return losses.cpu().numpy()


def image_patches(target: torch.Tensor):
    """[3, H, W] (H, W multiples of 256) -> patches [n, 3, 256, 256] in
    row-major patch order."""
    _, H, W = target.shape
    p = target.view(3, H // SIDE, SIDE, W // SIDE, SIDE).permute(1, 3, 0, 2, 4)
    return p.reshape(-1, 3, SIDE, SIDE).contiguous()


def to_image(props: dict, H: int, W: int) -> dict:
    """Patch proposals [n, cells, ...] -> the curves of the whole image
    (patch origins added to the control points, flat over curves)."""
    dev = props["ctrl"].device
    py, px = torch.meshgrid(torch.arange(H // SIDE, device=dev), torch.arange(W // SIDE, device=dev), indexing="ij")
    origin = torch.stack([px.reshape(-1), py.reshape(-1)], -1).float() * SIDE
    out = {}
    for k, v in props.items():
        if k in ("ctrl", "open_ctrl"):
            v = v + origin[:, None, None, :]
        out[k] = v.reshape((-1,) + tuple(v.shape[2:]))
    return out


def initial_curves(target: torch.Tensor, net: InitNet = None):
    """The curves initialising the method on target [3, H, W]: the
    network's proposals, or (net None) the baseline curves."""
    _, H, W = target.shape
    if net is None:
        n = (H // SIDE) * (W // SIDE)
        base = baseline_init(n, SIDE, image_patches(target).cpu().numpy())
        props = {k: torch.as_tensor(v, device=target.device).view((n, CELLS) + v.shape[1:]) for k, v in base.items()}
    else:
        props = net.propose(image_patches(target))
    return _curve_set(to_image(props, H, W), target.device)


def optimise(target: torch.Tensor, curves: bs.CurveSet, steps: int, sample=(4, 8, 8), every: int = 10,
             cfg: AdamCfg = PAIR_ADAM):
    """The method on one image from `curves` (in place): PSNR every `every`
    steps (index 0 = the initial curves) and the ms per step."""
    from .raster import Rasterizer
    _, H, W = target.shape
    rows, kc, g_open = sample
    r = Rasterizer(bs.Canvas(W, H, 16), bs.SampleCfg(g_open=g_open, rows_closed=rows, k_closed=kc), curves.n_open,
                   curves.n_closed, device=target.device, pair_capacity=1 << 22)
    grad = curves.zeros_like()
    adam = CurveAdam(curves, grad, [bs.BatchImage(W, H, curves.n_open, curves.n_closed, r.cfg)], cfg, target.device)
    psnr = []
    t_ms = 0.0
    for i in range(steps + 1):
        if i % every == 0 or i == steps:
            img = r.forward(curves)
            psnr.append(float(-10.0 * torch.log10(((img - target).double() ** 2).mean())))
        if i == steps:
            break
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r.step(curves, target, grad)
        adam.step()
        b.record()
        b.synchronize()
        t_ms += a.elapsed_time(b)
    return psnr, t_ms / max(1, steps)


def train_flops(n: int, side: int = SIDE) -> float:
    """Multiply-adds x 2 of one training step on n patches: per convolution
    the forward and the weight gradient each 2 M K Cout, the input gradient
    the same except for the first layer."""
    tot = 0.0
    for l in range(6):
        if l < 5:
            ho = side >> (l + 1)
            m, k, co = n * ho * ho, 16 * KERNEL_CH[l], KERNEL_CH[l + 1]
        else:
            m, k, co = n * (side // CELL) ** 2, 256, 64
        f = 2.0 * m * k * co
        tot += f * (2 if l == 0 else 3)
    return tot


def time_forward(n: int = 64, side: int = SIDE, reps: int = 20, engines=(0, 3, 1), device="cuda") -> dict:
    """ms of one forward of n random patches on each GEMM engine (0:
    mma.sync, 3: tcgen05 with thread-gathered operands, 1: the default, the
    convolutions of 64 or more input channels TMA-fed), CUDA events."""
    net = InitNet(device=device, seed=1)
    rng = np.random.default_rng(0)
    x = torch.as_tensor(rng.uniform(0, 1, (n, 3, side, side)).astype(np.float32), device=device)
    head = torch.empty(n, (side // CELL) ** 2, 64, device=device)
    out = {}
    try:
        for engine in engines:
            bs.debug_gemm_engine(engine)
            for _ in range(3):
                bs.net_forward(net.w, net.w_bf16, x, net.ws(n, side), head)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                bs.net_forward(net.w, net.w_bf16, x, net.ws(n, side), head)
            e1.record()
            torch.cuda.synchronize()
            out[engine] = e0.elapsed_time(e1) / reps
    finally:
        bs.debug_gemm_engine(1)
    return out


def time_train(n: int = 64, side: int = SIDE, reps: int = 20, engines=(0, 3, 1), device="cuda") -> dict:
    """ms of one training step (forward, backward, Adam, bf16 copies) of n
    random patches against random target curves on each GEMM engine, CUDA
    events."""
    net = InitNet(device=device, seed=1)
    rng = np.random.default_rng(0)
    x = torch.as_tensor(rng.uniform(0, 1, (n, 3, side, side)).astype(np.float32), device=device)
    cells = (side // CELL) ** 2
    t = {k: torch.as_tensor(rng.uniform(0.1, 0.9, (n, cells) + sh).astype(np.float32), device=device)
         for k, sh in bs.NET_CURVE_SHAPES.items()}
    out = {}
    try:
        for engine in engines:
            bs.debug_gemm_engine(engine)
            for _ in range(3):
                net.train_step(x, t)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                net.train_step(x, t)
            e1.record()
            torch.cuda.synchronize()
            out[engine] = e0.elapsed_time(e1) / reps
    finally:
        bs.debug_gemm_engine(1)
    return out


def main(argv=None):
    """Pairs -> training -> evaluation on 2048 x 2048 targets (64 patches
    each); prints one JSON line.  With --time-forward (--time-train), only
    the forward's (a training step's) time on each GEMM engine."""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--pair-steps", type=int, default=150)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--targets", type=int, default=2)
    ap.add_argument("--side", type=int, default=2048)
    ap.add_argument("--eval-steps", type=int, default=300)
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--time-forward", action="store_true", help="time one forward of --batch patches per engine")
    ap.add_argument("--time-train", action="store_true", help="time one training step of --batch patches per engine")
    ap.add_argument("--engines", default="0,3,1", help="GEMM engines for --time-forward")
    ap.add_argument("--reps", type=int, default=20)
    a = ap.parse_args(argv)
    if a.time_forward:
        ms = time_forward(a.batch, SIDE, a.reps, tuple(int(e) for e in a.engines.split(",")))
        print(json.dumps({"forward_ms_by_engine": ms, "patches": a.batch, "side": SIDE}))
        return
    if a.time_train:
        ms = time_train(a.batch, SIDE, a.reps, tuple(int(e) for e in a.engines.split(",")))
        print(json.dumps({"train_step_ms_by_engine": ms, "patches": a.batch, "side": SIDE,
                          "tflops_by_engine": {k: round(train_flops(a.batch) / (v * 1e-3) / 1e12, 2)
                                               for k, v in ms.items()}}))
        return
    dev = "cuda"
    t0 = time.perf_counter()
    data = make_pairs(a.pairs, seed=1, steps=a.pair_steps, device=dev)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    net = InitNet(device=dev, seed=0, lr=a.lr)
    learned_t0 = time.perf_counter()
    losses = train(net, data, a.train_steps, batch=a.batch)
    t_train = time.perf_counter() - learned_t0
    # the network's tensor-core throughput on one training batch
    idx = torch.arange(min(a.batch, a.pairs), device=dev)
    b = {k: data[k].index_select(0, idx).contiguous() for k in PAIR_KEYS}
    p = b.pop("patches")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        net.train_step(p, b)
    e0.record()
    for _ in range(10):
        net.train_step(p, b)
    e1.record()
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / 10
    evals = []
    for i in range(a.targets):
        tg = torch.as_tensor(synth.procedural_target(7000 + i, a.side, a.side, 200), device=dev)
        res = {}
        for name, m in (("baseline", None), ("learned", net)):
            s0 = time.perf_counter()
            curves = initial_curves(tg, m)
            torch.cuda.synchronize()
            init_ms = (time.perf_counter() - s0) * 1e3
            psnr, ms = optimise(tg, curves, a.eval_steps, every=a.every)
            res[name] = dict(psnr=[round(x, 3) for x in psnr], ms_per_step=round(ms, 4), init_ms=round(init_ms, 2))
        goal = res["baseline"]["psnr"][-1]
        hit = next((j for j, x in enumerate(res["learned"]["psnr"]) if x >= goal), None)
        steps_learned = None if hit is None else min(a.eval_steps, hit * a.every)
        res["baseline_final_db"] = goal
        res["learned_steps_to_baseline_final"] = steps_learned
        res["baseline_steps"] = a.eval_steps
        if steps_learned is not None:
            t_c = a.eval_steps * res["baseline"]["ms_per_step"] + res["baseline"]["init_ms"]
            t_l = steps_learned * res["learned"]["ms_per_step"] + res["learned"]["init_ms"]
            res["wall_ms_baseline"] = round(t_c, 2)
            res["wall_ms_learned"] = round(t_l, 2)
        evals.append(res)
    out = {
        "what": "learned initialisation vs the baseline initialisation of the method (circles and strokes)",
        "pairs": {"n": a.pairs, "optimiser_steps": a.pair_steps, "seconds": round(t_pairs, 2)},
        "train": {"steps": a.train_steps, "batch": a.batch, "seconds": round(t_train, 2),
                  "loss_first": round(float(losses[:10].mean()), 5), "loss_last": round(float(losses[-10:].mean()), 5),
                  "step_ms": round(step_ms, 4), "tflops": round(train_flops(a.batch) / (step_ms * 1e-3) / 1e12, 3)},
        "eval": {"side": a.side, "patches": (a.side // SIDE) ** 2, "curves": (a.side // SIDE) ** 2 * CELLS,
                 "targets": evals},
    }
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
