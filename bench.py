"""Throughput of the Bezier Splatting rasterizer: fwd+bwd raster steps/s.

One step = the whole hot path over one synthetic problem:
  curve order -> sample Gaussians -> bin (count, emit, radix sort, ranges)
  -> blend forward with the L2 loss gradient (one kernel) -> blend backward
  -> sampling backward,
captured as one CUDA graph (the binning reads nothing back) and replayed.
Workload (default): 2048x2048 RGB target, 2048 open + 2048 closed cubic
curves, 64 Gaussians per curve (262,144 Gaussians), 16x16 tiles.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload.  Under torchrun the ranks optimise
independent images (rank r's curves and target from seed + r; the images
share nothing, so there is no collective in the data path) and the batch of
the "batched" object is split across the ranks by pixel count.

The line's "batched" object measures the other half of the metric: 64
ragged images (sides 256..2048, 128..4096 curves each) optimised together,
sampling and tile side autotuned, one CUDA-graph replay per Adam step of
every image, against the same optimisation image by image (one graph replay
per image), both run for the same steps from the same curves: ms per step,
the PSNR curves, and the steps and wall-clock the batch needs to reach the
plain arm's final PSNR.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "hires_2048_4096"
METRIC = "fwd+bwd raster steps/s at 2048² (4096 curves); batched vs plain, same PSNR"
UNIT = "steps/s"
FP32_LANES_PER_SM = 128
RENDER_SOURCE = os.path.join(ROOT, "paper_2503_16424_gb300", "csrc", "bs_render.cu")

# Per (pixel, list entry) evaluation E of each blend kernel (E: the entries
# up to each pixel's stop point; the backward: up to its last blended
# entry), the FP32 floating-point operations the code issues and its MUFU
# operations: ncu's per-opcode thread-instruction counters of one launch on
# this workload (FFMA counted 2, FADD and FMUL 1, FFMA2/FADD2/FMUL2 twice
# that; MUFU = XU-pipe thread instructions), divided by that launch's E.
# Each entry holds the counters of one capture, the E it was divided by, and
# the 16-hex-digit SHA-256 prefix of the kernel source it was taken on; when
# the source has changed since, the figures are reported as stale (null).
# The instruction counts come from a quarter of the workload (1024 x 1024,
# 512 + 512 curves, the same sampling; a capture of several passes), and
# carry over per evaluation; the DRAM bytes (read + write, one launch) from a
# one-pass capture of the full workload.
NCU_CAPTURE = {
    "source_sha256_16": "6d4f75d78482383e",
    "workload": "hires_1024_1024",
    "render_fwd_kernel": {"flop_per_eval": 9.0216, "mufu_per_eval": 0.5828,
                          "ffma": 569099211, "fadd": 146802257, "fmul": 198282596, "xu": 95815936,
                          "evals": 164415545, "dram_bytes": 179548928,
                          "pipes": {"issue_active_pct": 71.8, "fma_pipe_pct": 32.1, "alu_pipe_pct": 41.7,
                                    "shared_pipe_pct": 17.7, "warps_active_pct": 38.3}},
    "render_bwd_kernel": {"flop_per_eval": 22.7272, "mufu_per_eval": 1.0985,
                          "ffma": 1094763846, "fadd": 836737013, "fmul": 641605293, "xu": 177278880,
                          "evals": 161386726, "dram_bytes": 127760896,
                          "pipes": {"issue_active_pct": 70.5, "fma_pipe_pct": 35.6, "alu_pipe_pct": 38.0,
                                    "shared_pipe_pct": 33.5, "warps_active_pct": 30.9}},
}


def fp32_peak_tflops(sm_mhz: float, n_sm: int = 152) -> float:
    """FP32 peak: n_sm SMs x 128 lanes x 2 FLOP (an FMA) x the SM clock."""
    return n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def set_workload(name: str):
    global WORKLOAD
    from paper_2503_16424_gb300 import synth
    if name not in synth.WORKLOADS:
        raise SystemExit(f"unknown workload {name}; one of {sorted(synth.WORKLOADS)}")
    WORKLOAD = name


def render_source_hash() -> str:
    with open(RENDER_SOURCE, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def capture_current() -> bool:
    return NCU_CAPTURE["source_sha256_16"] is not None and NCU_CAPTURE["source_sha256_16"] == render_source_hash()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def host_cpu() -> dict:
    """The host's core count and CPU model (lscpu's "Model name", else
    /proc/cpuinfo, else platform)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine()}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of every rank's x (a collective only when world > 1)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device) -> float:
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


def job_throughput(world: int, steps: int, ms: float) -> float:
    """Steps of all ranks per second of the slowest rank's clock."""
    return world * steps / (ms / 1e3)


def workload_inputs(seed_offset: int = 0):
    """The workload's curves and target (seeded; synth only, so that the
    oracle arm never loads the library)."""
    from paper_2503_16424_gb300 import synth
    w = synth.WORKLOADS[WORKLOAD]
    seed = w["seed"] + 100 * seed_offset
    arrays = synth.make_curves(seed, w["W"], w["H"], w["n_open"], w["n_closed"], style=w["style"]).as_dict()
    target = synth.procedural_target(seed + 1, w["W"], w["H"], w.get("n_shapes", 40))
    return w, arrays, target


def workload_config(w, n_pairs, world):
    return {"workload": WORKLOAD, "W": w["W"], "H": w["H"], "n_open": w["n_open"], "n_closed": w["n_closed"],
            "gaussians_per_curve": w["g_open"],
            "n_gaussians": w["n_open"] * w["g_open"] + w["n_closed"] * w["rows_closed"] * w["k_closed"],
            "tile": w["tile"], "n_pairs": n_pairs, "curve_init": w["style"],
            "l2": "working set larger than L2 (no flush)",
            "parallelism": "1 GPU" if world == 1 else f"independent images x{world}"}


def run_ours(args, rank, world):
    import torch
    from paper_2503_16424_gb300 import bs
    from paper_2503_16424_gb300.raster import Rasterizer, StepGraph

    local = int(os.environ.get("LOCAL_RANK", 0))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w, arrays, target_np = workload_inputs(rank)
    cfg = bs.SampleCfg(g_open=w["g_open"], rows_closed=w["rows_closed"], k_closed=w["k_closed"])
    canvas = bs.Canvas(w["W"], w["H"], w["tile"])
    curves = bs.CurveSet.from_arrays(arrays, device=dev)
    target = torch.as_tensor(target_np, device=dev)
    r = Rasterizer(canvas, cfg, curves.n_open, curves.n_closed, device=dev, pair_capacity=1 << 25)
    grad = curves.zeros_like()
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count

    # the step as one graph: the first call runs eagerly and sizes the pair
    # capacity, the second captures, the others replay
    sg = StepGraph(r, curves, target, grad)
    for _ in range(max(3, args.warmup)):
        sg()
    st, n_pairs = sg.check()
    if st != bs.BS_OK:
        raise RuntimeError(f"binning status {st} after the warm-up")
    stats = bs.render_stats(r.gauss, canvas, r.binning)     # work counters of this problem (untimed)

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            sg()
        t1.record(stream)
        torch.cuda.synchronize()
    st, _ = sg.check()
    if st != bs.BS_OK:
        raise RuntimeError(f"binning status {st} in the timed region")
    ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = ms / args.steps
    value = job_throughput(world, args.steps, ms)

    # the blend kernels' own durations, for the roofline: the same steps run
    # eagerly with CUDA events around the two kernels on their stream
    def mk():
        return torch.cuda.Event(enable_timing=True)
    ev = [[mk() for _ in range(4)] for _ in range(args.steps)]
    for i in range(args.steps):
        e = ev[i]
        bs.curve_order(curves, cfg, out=(r.rank, r.first))
        bs.sample_curves(curves, cfg, r.first, out=r.gauss)
        r.binning.run(r.gauss)
        e[0].record(stream)
        bs.render_fwd_l2(r.gauss, canvas, r.binning, target, out=(r.img, r.T, r.nc), dimg=r.dimg, loss=r.loss)
        e[1].record(stream)
        e[2].record(stream)
        bs.render_bwd(r.gauss, canvas, r.binning, r.T, r.nc, r.dimg, r.dgauss)
        e[3].record(stream)
        bs.sample_curves_bwd(curves, cfg, r.first, r.dgauss, grad)
    torch.cuda.synchronize()
    fwd_avg = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    bwd_avg = float(np.mean([e[2].elapsed_time(e[3]) for e in ev]))

    # end to end through the public API with host buffers: every step copies
    # its inputs (curves + target) from pinned memory and reads its loss and
    # gradients back.  Two device buffer sets, each with its own captured
    # step, and a copy stream: step i+1's inputs go up while step i computes,
    # step i's results come down after it; every copy of every step is inside
    # the timed region.
    host_in = {k: torch.as_tensor(v).pin_memory() for k, v in arrays.items()}
    host_target = torch.as_tensor(target_np).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host_in.values()) + host_target.numel() * 4
    d2h = sum(getattr(grad, k).numel() * getattr(grad, k).element_size() for k in bs.CURVE_FIELDS) + 8
    bufs = []
    for _ in range(2):
        cv = bs.CurveSet(**{k: getattr(curves, k).clone() for k in bs.CURVE_FIELDS})
        tg = target.clone()
        gr = curves.zeros_like()
        g = StepGraph(r, cv, tg, gr)
        g()
        g()
        bufs.append({"cv": cv, "tg": tg, "gr": gr, "sg": g,
                     "out": {k: torch.empty_like(getattr(grad, k), device="cpu").pin_memory()
                             for k in bs.CURVE_FIELDS},
                     "loss": torch.empty((), dtype=torch.float64).pin_memory(),
                     "loss_dev": torch.empty((), dtype=torch.float64, device=dev),
                     "up": torch.cuda.Event(), "done": torch.cuda.Event(), "down": torch.cuda.Event()})
    copy = torch.cuda.Stream(device=dev)

    def upload(b):
        with torch.cuda.stream(copy):
            copy.wait_event(b["done"])      # the step that last used these buffers has finished
            for k in bs.CURVE_FIELDS:
                getattr(b["cv"], k).copy_(host_in[k], non_blocking=True)
            b["tg"].copy_(host_target, non_blocking=True)
            b["up"].record(copy)

    def run_e2e(n):
        for b in bufs:
            b["done"].record(stream)
            b["down"].record(stream)
        upload(bufs[0])
        for i in range(n):
            b = bufs[i % 2]
            if i + 1 < n:
                upload(bufs[(i + 1) % 2])
            stream.wait_event(b["up"])
            stream.wait_event(b["down"])     # its gradients of two steps ago have been read back
            b["sg"]()
            b["loss_dev"].copy_(r.loss)       # the next step rewrites r.loss
            b["done"].record(stream)
            with torch.cuda.stream(copy):
                copy.wait_event(b["done"])
                for k in bs.CURVE_FIELDS:
                    b["out"][k].copy_(getattr(b["gr"], k), non_blocking=True)
                b["loss"].copy_(b["loss_dev"], non_blocking=True)
                b["down"].record(copy)
        torch.cuda.synchronize()

    run_e2e(3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    run_e2e(args.steps)
    e_ms = max_over_ranks((time.perf_counter() - e0) * 1e3, world, dev)
    e2e_value = job_throughput(world, args.steps, e_ms)
    for b in bufs:
        if b["sg"].check()[0] != bs.BS_OK:
            raise RuntimeError("binning overflow in the end-to-end region")
    # same inputs as the device-timed steps: the same gradients up to the
    # order of the backward's atomic sums
    g_e2e, g_dev = bufs[(args.steps - 1) % 2]["out"]["open_ctrl"], grad.open_ctrl.cpu()
    assert float((g_e2e - g_dev).abs().max()) <= 1e-3 * float(g_dev.abs().max()), "end-to-end gradients differ"

    # the periodic pass (every few hundred steps, outside the step): prune and
    # densify a copy of the curves against the last rendered image
    r.forward(curves)
    pd_cfg = bs.PDCfg(step=200, t_end=1000)
    pd_ms = []
    for i in range(3):
        pd_work = bs.CurveSet(**{k: getattr(curves, k).clone() for k in bs.CURVE_FIELDS})
        a, b = mk(), mk()
        a.record(stream)
        _, pd_stats = r.prune_densify(pd_work, target, pd_cfg)
        b.record(stream)
        torch.cuda.synchronize()
        if i:
            pd_ms.append(a.elapsed_time(b))

    peaks, src = load_peaks()
    clocks = clk.summary()
    e_fwd, e_bwd = stats["visits"], stats["n_contrib_sum"]
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(w, n_pairs, world), step="one CUDA graph replay"),
        "roofline": roofline(fwd_avg, bwd_avg, e_fwd, e_bwd, n_sm, peaks, src),
        "kernels_ms": {"render_fwd": round(fwd_avg, 4), "render_bwd": round(bwd_avg, 4)},
        "work": {"fwd_evals": e_fwd, "bwd_evals": e_bwd, "fwd_evals_performed": stats["evals"],
                 "blended": stats["blended"]},
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": None,
        "clocks": clocks,
        "periodic": {"prune_densify_ms": round(float(np.mean(pd_ms)), 4), "not_in_step": True, **pd_stats},
    }
    # kernels launched per step: curve_order 2 (count, first), sample 1,
    # binning (binning_launches), render_fwd with the L2 term 1, render_bwd 2
    # (blend backward, grads_from_sums), sample_bwd 1; memsets are not kernels
    per_step = 2 + 1 + binning_launches(canvas, r.n_gauss) + 1 + 2 + 1
    out["gpu_launches"] = per_step * args.steps
    if not args.no_batched:
        out["batched"] = run_batched(dev, args, rank, world)
    if not args.no_paper_shape:
        out["paper_shape"] = run_paper_shape(dev)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_culled()
        out["cpu_baseline_brute_force"] = cpu_baseline(side=8)
    return out


def binning_launches(canvas, n_gauss: int) -> int:
    """Kernels one bs_bin_tiles call launches on one canvas: zero, count,
    scan_partials and the tile scan (one CTA when the tile counts fit its
    shared memory, else row scans, column scans and the scan), then either
    the two-level counting sort (32-bit keys, at most 512 x 512 tiles: 7
    kernels) or the key emission and the radix passes (chunk_owner, emit,
    then upsweep, scan_parts and downsweep per pass, the first pass's counts
    coming from emit)."""
    tx, ty = -(-canvas.width // canvas.tile), -(-canvas.height // canvas.tile)
    n_tiles = tx * ty
    tbits = max(1, (n_tiles - 1).bit_length())
    gbits = max(1, (max(n_gauss, 1) - 1).bit_length())
    passes = -(-tbits // 8)
    ldc, nb = (tx + 3) & ~3, (1 if tx >= 1024 else min(min(1024 // tx, 64), ty))
    fused = ty * ldc + nb * tx + ty <= 48 * 1024 and passes <= 2
    n_g1 = -(-max(n_gauss, 1) // 256)
    rows = gbits + tbits <= 32 and ty <= 512 and tx <= 512 and ty * n_g1 <= (1 << 24)
    sort = 7 if rows else 2 + 3 * passes - 1
    return 3 + (1 if fused else 3) + sort


def roofline(fwd_ms, bwd_ms, e_fwd, e_bwd, n_sm, peaks, src):
    """The dominant blend kernel's FP32 rate against the FP32 peak (SMs x 128
    lanes x 2 FLOP x the maximum SM clock), from the FLOP per evaluation the
    code issues (ncu instruction counters of the current kernel source)."""
    mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = fp32_peak_tflops(mhz, n_sm)
    dom, t, e = ("render_bwd_kernel", bwd_ms, e_bwd) if bwd_ms >= fwd_ms else ("render_fwd_kernel", fwd_ms, e_fwd)
    fresh = capture_current()
    cap = NCU_CAPTURE.get(dom) if fresh else None
    out = {"bound": "alu", "kernel": dom, "unit": "TFLOP/s", "peak": round(peak, 2),
           "peak_source": f"FP32: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 x {mhz} MHz ({src} max clock)",
           "achieved": None, "frac": None, "traffic": None,
           "flop_per_eval": None, "evals": e, "kernel_ms": round(t, 4),
           "counters": "current" if fresh else "stale: the kernel source changed since the ncu capture"}
    if cap:
        ach = cap["flop_per_eval"] * e / (t * 1e-3) / 1e12
        out.update(achieved=round(ach, 3), frac=round(ach / peak, 4), flop_per_eval=cap["flop_per_eval"],
                   mufu_per_eval=cap.get("mufu_per_eval"), traffic=cap.get("dram_bytes"),
                   algorithmic_bytes=cap.get("algorithmic_bytes"), pipes=cap.get("pipes"))
        other = "render_fwd_kernel" if dom == "render_bwd_kernel" else "render_bwd_kernel"
        oc = NCU_CAPTURE.get(other)
        if oc:
            ot, oe = (fwd_ms, e_fwd) if other == "render_fwd_kernel" else (bwd_ms, e_bwd)
            oach = oc["flop_per_eval"] * oe / (ot * 1e-3) / 1e12
            out["other_kernel"] = {"kernel": other, "achieved": round(oach, 3), "frac": round(oach / peak, 4),
                                   "flop_per_eval": oc["flop_per_eval"], "kernel_ms": round(ot, 4)}
    return out


# The paper's own timings (RTX 4090 per the teaser caption; context, not a
# target): Table 1 at 2040 x 1344 with 2048 curves, forward and backward ms;
# Table 4, 2048 closed curves with R interior rows, forward (with gradients)
# and backward ms, resolution not stated.
PAPER_MS = {"open_2048": (4.5, 4.7, "Table 1"), "closed_2048_R20": (14.1, 24.58, "Table 1"),
            "closed_2048_R40": (14.79, 25.06, "Table 4"), "closed_2048_R80": (27.01, 33.40, "Table 4")}


def run_paper_shape(dev, steps=10, warmup=3):
    """Forward (draw order, sampling, binning, blend with the L2 term) and
    backward (blend backward, sampling backward) ms on the paper's shapes:
    2040 x 1344 with 2048 open curves of 64 Gaussians, or 2048 closed curves
    with R = 20, 40, 80 interior rows of 32 samples (Section 4, Table 1,
    Table 4)."""
    import torch
    from paper_2503_16424_gb300 import bs, synth
    from paper_2503_16424_gb300.raster import Rasterizer
    W, H = 2040, 1344
    target = torch.as_tensor(synth.procedural_target(21, W, H, 50), device=dev)
    out = {}
    stream = torch.cuda.current_stream()
    for name, (no, nc, g, rows, kc) in {"open_2048": (2048, 0, 64, 4, 8), "closed_2048_R20": (0, 2048, 16, 22, 32),
                                        "closed_2048_R40": (0, 2048, 16, 42, 32),
                                        "closed_2048_R80": (0, 2048, 16, 82, 32)}.items():
        curves = bs.CurveSet.from_arrays(synth.make_curves(21, W, H, no, nc, style="local").as_dict(), device=dev)
        cfg = bs.SampleCfg(g_open=g, rows_closed=rows, k_closed=kc)
        r = Rasterizer(bs.Canvas(W, H, 16), cfg, no, nc, device=dev, pair_capacity=1 << 24)
        grad = curves.zeros_like()
        ev = []
        for i in range(warmup + steps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            bs.curve_order(curves, cfg, out=(r.rank, r.first))
            bs.sample_curves(curves, cfg, r.first, out=r.gauss)
            r.binning.run(r.gauss)
            bs.render_fwd_l2(r.gauss, r.canvas, r.binning, target, out=(r.img, r.T, r.nc), dimg=r.dimg, loss=r.loss)
            e[1].record(stream)
            r.backward(curves, r.dimg, grad)
            e[2].record(stream)
            if i >= warmup:
                ev.append(e)
        torch.cuda.synchronize()
        fwd = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
        bwd = float(np.median([e[1].elapsed_time(e[2]) for e in ev]))
        pf, pb, src = PAPER_MS[name]
        out[name] = {"gaussians": r.n_gauss, "pairs": r.binning.n_pairs, "fwd_ms": round(fwd, 4),
                     "bwd_ms": round(bwd, 4), "paper_fwd_ms": pf, "paper_bwd_ms": pb, "paper_source": src}
        del r
    return {"canvas": f"{W}x{H}", "note": "context: the paper's numbers are another GPU's (RTX 4090), "
                                          "Table 4's resolution is not stated", "cases": out}


def _mean_psnr(losses):
    import torch
    return float((-10.0 * torch.log10(losses.double())).mean())


def run_batched(dev, args, rank, world):
    """Batched vs plain on the ragged 64-image workload (this rank's share of
    it under torchrun): both arms run the same Adam steps from the same
    curves, the batch as one graph replay per step of every image, the plain
    arm as one graph replay per image, both with pair capacity 1.5 x the
    pairs found and the binning status read after every step outside the
    timed window (an overflow is counted, and the capacity regrown).
    Reported: ms per step of every image (timed over a window of replays
    with no reads), the mean PSNR every `every` steps, and the steps and
    wall-clock (steps x ms per step) the batch needs to reach the plain
    arm's final mean PSNR."""
    import torch
    from paper_2503_16424_gb300 import autotune, bs, synth
    from paper_2503_16424_gb300.batch import BatchOptimizer, BatchRasterizer, PlainOptimizer, partition_images
    W = synth.BATCH_WORKLOAD
    layout_all = synth.batch_layout(W["seed"], W["n_images"], W["side"], W["aspect"], W["curves"])
    mine = partition_images([e["W"] * e["H"] for e in layout_all], world)[rank]
    layout = [layout_all[i] for i in mine]
    arrs, cat, targets = synth.batch_inputs(layout, W["n_shapes"])
    base = [bs.BatchImage(e["W"], e["H"], e["n_open"], e["n_closed"], bs.SampleCfg()) for e in layout]
    target = torch.as_tensor(np.concatenate([t.reshape(-1) for t in targets]), device=dev)
    images, tile, report = autotune.autotune(base, bs.CurveSet.from_arrays(cat, device=dev), target, arrs=arrs,
                                             device=dev)
    total, every, window = max(args.batched_steps, 25), 25, 20
    stream = torch.cuda.current_stream()

    def run(step_fn, losses_fn, check_fn):
        """total steps; the ms per step over replays 3 .. 3 + window (no
        reads inside); the mean PSNR after every `every` steps."""
        curve, ms = [], None
        for i in range(total):
            if i == 3:
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
            step_fn()
            if i == 2 + window:
                b.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b) / window
            if not 3 <= i <= 2 + window:
                check_fn()                           # a capacity overflow regrows and recaptures
            if i == 0 or (i + 1) % every == 0:      # outside the window (every > 2 + window)
                curve.append((i + 1, round(_mean_psnr(losses_fn()), 4)))
        check_fn()
        return curve, ms

    # batched: the eager first step fits the capacity, then graph replays
    curves = bs.CurveSet.from_arrays(cat, device=dev)
    r = BatchRasterizer(images, tile=tile, pair_capacity=1 << 24, device=dev)
    opt = BatchOptimizer(r, curves, target, graph=True, check_every=0)
    b_curve, b_ms = run(opt.step, lambda: r.loss, opt.check)
    st, n_pairs = r.batch.status()
    b_overflows = opt.overflows
    # plain: the same steps image by image, one graph replay per image
    per = [bs.CurveSet.from_arrays(a, device=dev) for a in arrs]
    tg = [torch.as_tensor(t, device=dev) for t in targets]
    plain = PlainOptimizer(images, per, tg, device=dev, tile=tile, graph=True, headroom=1.5)
    p_curve, p_ms = run(plain.step, plain.losses, plain.check)
    p_overflows = sum(g.overflows for g in plain.graphs)
    p_final = p_curve[-1][1]
    reach = next((s for s, p in b_curve if p >= p_final), None)
    n_img = len(images)
    # the job: every rank's images over the slowest rank's step
    job_b_ms, job_p_ms = max_over_ranks(b_ms, world, dev), max_over_ranks(p_ms, world, dev)
    job_imgs = sum_over_ranks(n_img, world, dev)
    passes = -(-max(1, (r.batch.n_tiles - 1).bit_length()) // 8)
    sizes = [im.sample.g_open for im in images if im.n_open] + \
            [im.sample.rows_closed * im.sample.k_closed for im in images if im.n_closed]
    classes = len({n >= 512 for n in sizes})
    return {
        "workload": W["name"], "images": n_img, "images_all_ranks": int(job_imgs), "rank_images": mine,
        "pixels": r.batch.n_pixels, "curves": r.batch.n_open + r.batch.n_closed, "gaussians": r.batch.n_gauss,
        "pairs": n_pairs, "binning_status": st, "autotune": report,
        "ms_per_step": round(b_ms, 4), "image_steps_per_s": round(job_imgs * 1e3 / job_b_ms, 2),
        "plain_ms_per_step": round(p_ms, 4), "plain_image_steps_per_s": round(job_imgs * 1e3 / job_p_ms, 2),
        "speedup_vs_plain": round(p_ms / b_ms, 3),
        "step": "draw order, sampling, binning, blend + L2, backward, Adam; batched = one CUDA graph replay "
                "for every image, plain = one CUDA graph replay per image",
        "launches_per_step": 17 + 3 * passes + 2 * classes,
        "psnr": {"steps": total, "every": every, "batched_curve_db": b_curve, "plain_curve_db": p_curve,
                 "batched_final_db": b_curve[-1][1], "plain_final_db": p_final,
                 "batched_steps_to_plain_final": reach,
                 "batched_ms_to_plain_final": round(reach * b_ms, 2) if reach else None,
                 "plain_ms_for_all_steps": round(total * p_ms, 2),
                 "capacity_overflows": {"batched": b_overflows, "plain": p_overflows}},
    }


def cpu_baseline(side=16):
    """The fp64 CPU oracle on a bounded sample of the workload: sampling of
    all curves, the brute-force blend (every Gaussian at every pixel) and its
    gradient at a side x side pixel crop extrapolated to the full image by
    pixel count, and the sampling backward of all curves."""
    import torch
    import oracle
    from oracle.curves import SampleCfg as OCfg
    from oracle.pipeline import as_curves, sample_vjp
    w, arrays, target_np = _oracle_problem()
    cfg = OCfg(g_open=w["g_open"], rows_closed=w["rows_closed"], k_closed=w["k_closed"])
    threads = torch.get_num_threads()
    t0 = time.perf_counter()
    cur = as_curves(arrays)
    _, first = oracle.draw_order(arrays["open_ctrl"], arrays["open_width"], arrays["closed_ctrl"], cfg)
    with torch.no_grad():
        tab = oracle.gaussian_table(cur, cfg, first)
    t_sample = time.perf_counter() - t0
    y0 = x0 = w["W"] // 2 - side // 2
    ys, xs = torch.meshgrid(torch.arange(y0, y0 + side, dtype=torch.float64),
                            torch.arange(x0, x0 + side, dtype=torch.float64), indexing="ij")
    xs, ys = xs.reshape(-1), ys.reshape(-1)
    t1 = time.perf_counter()
    with torch.no_grad():
        px = oracle.render_pixels(tab, xs, ys)
    tgt = torch.as_tensor(target_np[:, y0:y0 + side, x0:x0 + side]).permute(1, 2, 0).reshape(-1, 3)
    n_full = 3 * w["W"] * w["H"]
    dC = 2.0 * (px["C"] - tgt.double()) / n_full
    dtab = oracle.render_grads(tab, xs, ys, dC)
    t_pix = time.perf_counter() - t1
    t2 = time.perf_counter()
    sample_vjp(cur, cfg, dtab, first)
    t_vjp = time.perf_counter() - t2
    frac = (side * side) / (w["W"] * w["H"])
    step_s = t_sample + t_vjp + t_pix / frac
    return {"value": round(1.0 / step_s, 9), "unit": UNIT, "cores": threads, "kind": "oracle",
            "extrapolated": True, "host": host_cpu(),
            "sample": f"sampling of all {w['n_open'] + w['n_closed']} curves, brute-force blend and its "
                      f"gradient at a {side}x{side} pixel crop ({side * side} of {w['W'] * w['H']} pixels, "
                      f"time extrapolated by pixel count), sampling backward of all curves",
            "seconds": round(time.perf_counter() - t0, 2)}


def cpu_baseline_culled(steps: int = 2):
    """The oracle's whole step on all host cores, not extrapolated: fp64
    sampling of every curve (torch), the box-culled fp64 blend and its
    hand-derived backward (oracle/cull.c, OpenMP), the L2 gradient, and the
    sampling backward (torch autograd), `steps` times."""
    import torch
    import oracle
    from oracle import cull
    from oracle.curves import SampleCfg as OCfg
    from oracle.pipeline import as_curves, sample_vjp
    w, arrays, target_np = _oracle_problem()
    cfg = OCfg(g_open=w["g_open"], rows_closed=w["rows_closed"], k_closed=w["k_closed"])
    cull.build()
    t0 = time.perf_counter()
    for _ in range(steps):
        cur = as_curves(arrays)
        _, first = oracle.draw_order(arrays["open_ctrl"], arrays["open_width"], arrays["closed_ctrl"], cfg)
        with torch.no_grad():
            tab = {k: v.detach() for k, v in oracle.gaussian_table(cur, cfg, first).items()}
        img, T, used = cull.forward(tab, w["W"], w["H"])
        d = img - target_np
        dimg = 2.0 * d / d.size
        g = cull.backward(tab, w["W"], w["H"], dimg, T, used)
        sample_vjp(cur, cfg, g, first)
    secs = time.perf_counter() - t0
    return {"value": round(steps / secs, 6), "unit": UNIT, "cores": cull.threads(), "kind": "oracle",
            "extrapolated": False, "host": host_cpu(),
            "sample": f"the whole step on the 2048x2048 workload, {steps} times: fp64 sampling of all curves, "
                      "the box-culled fp64 blend and its hand-derived backward on all host cores (OpenMP), the L2 "
                      "gradient, the sampling backward", "seconds": round(secs, 2)}


_PROBLEM = {}


def _oracle_problem():
    """The workload's curves and target for the oracle (made once)."""
    if not _PROBLEM:
        w, arrays, target_np = workload_inputs(0)
        _PROBLEM.update(w=w, arrays=arrays, target=target_np)
    return _PROBLEM["w"], _PROBLEM["arrays"], _PROBLEM["target"]


def oracle_pairs() -> int:
    """The workload's (tile, Gaussian) pairs by the oracle's binning rule."""
    import torch
    import oracle
    from oracle.curves import SampleCfg as OCfg, table_to_f32
    from oracle.pipeline import as_curves
    w, arrays, _ = _oracle_problem()
    cfg = OCfg(g_open=w["g_open"], rows_closed=w["rows_closed"], k_closed=w["k_closed"])
    _, first = oracle.draw_order(arrays["open_ctrl"], arrays["open_width"], arrays["closed_ctrl"], cfg)
    with torch.no_grad():
        rec = table_to_f32(oracle.gaussian_table(as_curves(arrays), cfg, first))
    tx0, tx1, ty0, ty1, ok = oracle.tile_rects_f32(rec, w["W"], w["H"], w["tile"])
    return int(np.where(ok, (tx1 - tx0 + 1) * (ty1 - ty0 + 1), 0).sum())


def run_reference(args, rank):
    """The oracle arm: the CPU oracle, as it stands, on the same workload and
    metric; each step is the bounded sample of cpu_baseline, its time
    extrapolated to the whole image.  It loads no part of the library."""
    if rank != 0:
        return None
    w, _, _ = _oracle_problem()
    for _ in range(max(1, args.warmup)):
        cpu_baseline(side=8)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(side=8)["value"])
    total = time.perf_counter() - t0
    value = float(np.mean(vals))
    cb = cpu_baseline(side=8)
    cb["value"] = round(value, 9)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 9), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 / value, 3),
            "ms_per_step_extrapolated": True, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": workload_config(w, oracle_pairs(), 1),
            "cpu_baseline": cb, "wall_s": round(total, 2),
            "e2e": {"value": round(value, 9), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-paper-shape", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=200)
    ap.add_argument("--workload", default=WORKLOAD,
                    help="synthetic single-canvas workload (another one than the default is for profiler captures)")
    args = ap.parse_args()
    set_workload(args.workload)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
