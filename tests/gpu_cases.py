"""Seeded cases shared by the GPU parity tests: the same synthetic inputs go
to the CUDA library (through the C ABI binding) and to the CPU oracle."""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

import oracle
from oracle.curves import SampleCfg as OCfg, table_to_f32, table_from_f32
from oracle.pipeline import as_curves
from paper_2503_16424_gb300 import synth


@dataclass
class Case:
    name: str
    W: int
    H: int
    n_open: int
    n_closed: int
    style: str
    g_open: int
    rows: int
    kc: int
    seed: int
    bg: tuple = (0.0, 0.0, 0.0)
    dup: int = 0            # duplicate this many curves (equal draw keys)


CASES = {
    # the 256x256, 64-open-curve workload, full size
    "tiny256": Case("tiny256", 256, 256, 64, 0, "uniform", 16, 4, 8, 1),
    # ragged canvas (not a multiple of the tile), open + closed, background
    "ragged": Case("ragged", 100, 73, 12, 6, "local", 12, 5, 7, 2, bg=(0.2, 0.5, 0.1), dup=2),
    # several sort partitions, both curve kinds
    "mixed": Case("mixed", 192, 160, 40, 24, "local", 16, 4, 8, 3, bg=(0.0, 0.3, 0.6), dup=3),
    # curves of 512 samples or more (sampled by the wide CTAs): open curves
    # of 600 samples, closed curves of R = 80 interior rows (82 x 8), whose
    # rows near the boundaries are thin
    "dense": Case("dense", 120, 90, 2, 2, "local", 600, 82, 8, 4, bg=(0.1, 0.1, 0.1)),
}


def arrays(case: Case):
    a = synth.make_curves(case.seed, case.W, case.H, case.n_open, case.n_closed, style=case.style).as_dict()
    if case.dup:
        for k in ("open_ctrl", "open_width", "open_color", "open_opac"):
            if case.n_open > case.dup:
                a[k][-case.dup:] = a[k][:case.dup]
        for k in ("closed_ctrl", "closed_color", "closed_opac"):
            if case.n_closed > case.dup:
                a[k][-case.dup:] = a[k][:case.dup]
    return a


def ocfg(case: Case):
    return OCfg(g_open=case.g_open, rows_closed=case.rows, k_closed=case.kc)


def oracle_table(case: Case, arr=None):
    arr = arr if arr is not None else arrays(case)
    cfg = ocfg(case)
    rank, first = oracle.draw_order(arr["open_ctrl"], arr["open_width"], arr["closed_ctrl"], cfg)
    tab = oracle.gaussian_table(as_curves(arr), cfg, first)
    return tab, rank, first


def target(case: Case):
    return synth.procedural_target(case.seed + 1000, case.W, case.H, 12)


def grad_rel_err(got, exp, floor_frac=1e-3):
    """max_i |got_i - exp_i| / max(|exp_i|, floor_frac * max|exp|)."""
    got = torch.as_tensor(got, dtype=torch.float64).reshape(-1)
    exp = torch.as_tensor(exp, dtype=torch.float64).reshape(-1)
    if exp.numel() == 0:
        return 0.0
    floor = max(float(exp.abs().max()) * floor_frac, 1e-30)
    return float(((got - exp).abs() / torch.clamp(exp.abs(), min=floor)).max())


__all__ = ["CASES", "Case", "arrays", "ocfg", "oracle_table", "target", "grad_rel_err", "table_to_f32",
           "table_from_f32"]
