"""Section 3.4's blend and its backward in double precision with exact box
culling, on all host cores (cull.c, OpenMP), through ctypes.

TEST INFRASTRUCTURE ONLY (see the package docstring): the multi-core CPU
baseline of the measurement, checked against the brute-force blend of
raster.py and its autograd gradient.  The C source is compiled on first use
(gcc -O2 -fopenmp) into oracle/_build/.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cull.c")
LIB = os.path.join(HERE, "_build", "libcull.so")
FIELDS = ("mx", "my", "ux", "uy", "isx", "isy", "o")
_lib = None


def build(force: bool = False) -> str:
    """Compile cull.c into a shared library (portable flags, no -march)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99", "-o", tmp, SRC, "-lm"], check=True,
                       capture_output=True, text=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.cull_forward.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P, P, P]
        _lib.cull_backward.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, P, P, P, P]
        _lib.cull_forward.restype = _lib.cull_backward.restype = ctypes.c_int
        _lib.cull_threads.restype = ctypes.c_int
    return _lib


def threads() -> int:
    return int(_load().cull_threads())


def _columns(tab: dict):
    cols = [np.ascontiguousarray(tab[k].detach().numpy(), dtype=np.float64) for k in FIELDS]
    col = tab["col"].detach().numpy()
    cols += [np.ascontiguousarray(col[:, c], dtype=np.float64) for c in range(3)]
    cols += [np.ascontiguousarray(tab[k].detach().numpy(), dtype=np.float64) for k in ("ext_x", "ext_y")]
    ptrs = (ctypes.c_void_p * 12)(*(c.ctypes.data for c in cols))
    return cols, ptrs


def forward(tab: dict, W: int, H: int, bg=(0.0, 0.0, 0.0)):
    """img [3,H,W], T_final [H,W] and the per-pixel count of list entries up
    to the last blended one (the backward's walk length), as numpy."""
    lib = _load()
    cols, ptrs = _columns(tab)
    n = cols[0].shape[0]
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    used = np.zeros((H, W), dtype=np.int64)
    bgv = np.asarray(bg, dtype=np.float64)
    if lib.cull_forward(ptrs, n, W, H, bgv.ctypes.data, img.ctypes.data, T.ctypes.data, used.ctypes.data):
        raise MemoryError("cull_forward")
    return img, T, used


def backward(tab: dict, W: int, H: int, dimg, T, used, bg=(0.0, 0.0, 0.0)) -> dict:
    """dL/d(table field) given dL/dimg [3,H,W]: mx my ux uy isx isy o [Ng],
    col [Ng,3] (torch float64)."""
    lib = _load()
    cols, ptrs = _columns(tab)
    n = cols[0].shape[0]
    g = [np.zeros(n) for _ in range(10)]
    gp = (ctypes.c_void_p * 10)(*(x.ctypes.data for x in g))
    dimg = np.ascontiguousarray(dimg, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    used = np.ascontiguousarray(used, dtype=np.int64)
    bgv = np.asarray(bg, dtype=np.float64)
    if lib.cull_backward(ptrs, n, W, H, bgv.ctypes.data, dimg.ctypes.data, T.ctypes.data, used.ctypes.data, gp):
        raise MemoryError("cull_backward")
    out = {k: torch.as_tensor(g[i]) for i, k in enumerate(FIELDS)}
    out["col"] = torch.as_tensor(np.stack(g[7:10], 1))
    return out
