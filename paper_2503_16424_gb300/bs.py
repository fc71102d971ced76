"""Thin ctypes binding of libbs.so with the C ABI's names.

Argument marshalling only: every function takes torch CUDA tensors, checks
their dtype/shape/contiguity, passes raw device pointers and the current
stream to the library, and raises on a non-OK status.  All computation runs
in the library's CUDA kernels; there is no fallback path.  Importing this
module raises ImportError when libbs.so has not been built.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_int32, c_int64, c_size_t, c_uint32, c_void_p
from dataclasses import dataclass

import torch

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbs.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                      "(python -m paper_2503_16424_gb300.build_lib)")
lib = ctypes.CDLL(LIB_PATH)

GAUSS_FLOATS = 12
DGAUSS_FLOATS = 12

BS_OK, BS_ERR_INVALID_ARG, BS_ERR_CUDA, BS_ERR_CAPACITY, BS_ERR_TIMEOUT, BS_ERR_NOT_FINITE, \
    BS_ERR_UNSUPPORTED = range(7)


class bs_curves(ctypes.Structure):
    _fields_ = [("n_open", c_int32), ("n_closed", c_int32),
                ("open_ctrl", c_void_p), ("open_width", c_void_p), ("open_color", c_void_p),
                ("open_opac", c_void_p), ("closed_ctrl", c_void_p), ("closed_color", c_void_p),
                ("closed_opac", c_void_p), ("draw_first", c_void_p), ("closed_color2", c_void_p),
                ("closed_opac2", c_void_p)]


class bs_curves_grad(ctypes.Structure):
    _fields_ = [("open_ctrl", c_void_p), ("open_width", c_void_p), ("open_color", c_void_p),
                ("open_opac", c_void_p), ("closed_ctrl", c_void_p), ("closed_color", c_void_p),
                ("closed_opac", c_void_p), ("closed_color2", c_void_p), ("closed_opac2", c_void_p)]


class bs_sample_cfg(ctypes.Structure):
    _fields_ = [("g_open", c_int32), ("rows_closed", c_int32), ("k_closed", c_int32),
                ("rho", c_float), ("cov_eps", c_float), ("tangent_mode", c_int32)]


class bs_canvas(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("tile", c_int32), ("bg", c_float * 3)]


class bs_curves_mut(ctypes.Structure):
    _fields_ = [("n_open", c_int32), ("n_closed", c_int32),
                ("open_ctrl", c_void_p), ("open_width", c_void_p), ("open_color", c_void_p),
                ("open_opac", c_void_p), ("closed_ctrl", c_void_p), ("closed_color", c_void_p),
                ("closed_opac", c_void_p)]


class bs_pd_cfg(ctypes.Structure):
    _fields_ = [("op_start", c_float), ("op_end", c_float), ("step", c_int32), ("t_end", c_int32),
                ("area_min", c_float), ("color_eps", c_float), ("iou_min", c_float),
                ("err_thresh", c_float), ("split_drop", c_float), ("new_opacity", c_float),
                ("new_width", c_float)]


class bs_pd_stats(ctypes.Structure):
    _fields_ = [(k, c_int32) for k in ("pruned", "low_opacity", "small_area", "overlap", "split",
                                      "split_placed", "regions", "inserted", "transparent")]


class bs_batch_image(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("n_open", c_int32), ("n_closed", c_int32),
                ("sample", bs_sample_cfg), ("bg", c_float * 3)]


class bs_batch(ctypes.Structure):
    _fields_ = [("images", c_void_p), ("n_images", c_int32), ("tile", c_int32), ("pair_capacity", c_int64),
                ("ws", c_void_p), ("ws_bytes", c_size_t)]


class bs_batch_sizes(ctypes.Structure):
    _fields_ = [("n_open", c_int64), ("n_closed", c_int64), ("n_gauss", c_int64), ("n_pixels", c_int64),
                ("n_tiles", c_int64), ("ws_bytes", c_size_t)]


class bs_adam_group(ctypes.Structure):
    _fields_ = [("param", c_void_p), ("grad", c_void_p), ("m", c_void_p), ("v", c_void_p), ("n", c_int64),
                ("lr", c_float), ("lo", c_float), ("hi", c_float), ("row_scale", c_void_p), ("row_len", c_int32)]


class bs_adam_cfg(ctypes.Structure):
    _fields_ = [("beta1", c_float), ("beta2", c_float), ("eps", c_float)]


ADAM_MAX_GROUPS = 16
NET_LAYERS = 6
NET_REACH = 24.0
NET_WIDTH_MAX = 8.0
NET_CURVE_KEYS = ("ctrl", "color", "opac", "open_ctrl", "open_width", "open_color", "open_opac")


class bs_net(ctypes.Structure):
    _fields_ = [("w", c_void_p * NET_LAYERS), ("w_bf16", c_void_p * NET_LAYERS)]


class bs_net_grad(ctypes.Structure):
    _fields_ = [("g", c_void_p * NET_LAYERS)]


class bs_net_curves(ctypes.Structure):
    _fields_ = [(k, c_void_p) for k in NET_CURVE_KEYS]


def _sig(name, *args):
    f = getattr(lib, name)
    f.argtypes = list(args)
    f.restype = c_int
    return f


_P = c_void_p
lib.bs_num_gaussians.argtypes = [c_int32, c_int32, POINTER(bs_sample_cfg)]
lib.bs_num_gaussians.restype = c_int64
lib.bs_last_error.restype = c_char_p
lib.bs_status_string.argtypes = [c_int]
lib.bs_status_string.restype = c_char_p
_sig("bs_curve_order", POINTER(bs_curves), POINTER(bs_sample_cfg), _P, _P, _P)
_sig("bs_sample_curves", POINTER(bs_curves), POINTER(bs_sample_cfg), _P, _P)
_sig("bs_sample_curves_bwd", POINTER(bs_curves), POINTER(bs_sample_cfg), _P, POINTER(bs_curves_grad), _P)
_sig("bs_bin_tiles_workspace", c_int64, POINTER(bs_canvas), c_int64, POINTER(c_size_t))
_sig("bs_bin_tiles", _P, c_int64, POINTER(bs_canvas), _P, c_size_t, c_int64, POINTER(c_int64), _P, _P, _P)
_sig("bs_render_fwd", _P, c_int64, POINTER(bs_canvas), _P, _P, _P, _P, _P, _P)
_sig("bs_bin_tiles_static", _P, c_int64, POINTER(bs_canvas), c_int64, POINTER(c_int64), _P, _P, _P)
_sig("bs_bin_tiles_async", _P, c_int64, POINTER(bs_canvas), _P, c_size_t, c_int64, _P, _P, _P, _P)
_sig("bs_bin_tiles_result", _P, c_size_t, POINTER(c_int32), POINTER(c_int64), _P)
_sig("bs_sync_status", c_int32, POINTER(c_int32), _P)
_sig("bs_render_fwd_l2", _P, c_int64, POINTER(bs_canvas), _P, _P, _P, _P, _P, _P, _P, _P, _P)
_sig("bs_l2_loss_grad", _P, _P, c_int64, _P, _P, _P)
_sig("bs_render_stats", _P, c_int64, POINTER(bs_canvas), _P, _P, _P, _P, _P, _P, _P)
_sig("bs_render_bwd", _P, c_int64, POINTER(bs_canvas), _P, _P, _P, _P, _P, _P,
     POINTER(bs_curves), POINTER(bs_sample_cfg), POINTER(bs_curves_grad), _P)
_sig("bs_prune_densify_workspace", c_int32, c_int32, POINTER(bs_canvas), POINTER(c_size_t))
_sig("bs_prune_densify", POINTER(bs_curves_mut), POINTER(bs_pd_cfg), POINTER(bs_canvas), _P, _P, _P, c_size_t, _P,
     POINTER(bs_pd_stats), _P)
_sig("bs_device_status", _P, c_size_t, POINTER(c_int32), _P)
_B = POINTER(bs_batch)
_sig("bs_batch_plan", _B, POINTER(bs_batch_sizes))
_sig("bs_batch_setup", _B, _P)
_sig("bs_batch_curve_order", _B, POINTER(bs_curves), _P, _P, _P)
_sig("bs_batch_sample_curves", _B, POINTER(bs_curves), _P, _P)
_sig("bs_batch_bin_tiles", _B, _P, _P, _P, _P)
_sig("bs_batch_render_fwd", _B, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P)
_sig("bs_batch_render_bwd", _B, _P, _P, _P, _P, _P, _P, _P, POINTER(bs_curves), POINTER(bs_curves_grad), _P)
_sig("bs_batch_status", _B, POINTER(c_int32), POINTER(c_int64), _P)
_sig("bs_adam_step", POINTER(bs_adam_group), c_int32, POINTER(bs_adam_cfg), _P, _P)
_sig("bs_xing_loss", POINTER(bs_curves), c_float, _P, _P, _P)
_sig("bs_debug_gemm_engine", c_int32, POINTER(c_int64))
_sig("bs_svg_export", POINTER(bs_curves), _P, c_int32, c_int32, c_int32, _P, c_size_t, POINTER(c_size_t))
lib.bs_net_param_count.argtypes = [c_int32]
lib.bs_net_param_count.restype = c_int64
_sig("bs_net_workspace", c_int32, c_int32, POINTER(c_size_t))
_sig("bs_net_sync_weights", POINTER(bs_net), _P)
_sig("bs_net_forward", POINTER(bs_net), _P, c_int32, c_int32, _P, c_size_t, _P, POINTER(bs_net_curves), _P)
_sig("bs_net_train_step", POINTER(bs_net), _P, c_int32, c_int32, POINTER(bs_net_curves), _P, c_size_t, POINTER(bs_net_grad),
     _P, _P)
_sig("bs_debug_retry_limit", c_int64)
_sig("bs_debug_umma_wait", c_int64)


class BSError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        name = lib.bs_status_string(status).decode()
        super().__init__(f"{fn}: {name}: {lib.bs_last_error().decode()}")


def _check(fn, status):
    if status != BS_OK:
        raise BSError(fn, status)


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else c_void_p(0)


def _want(t, dtype, shape=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


@dataclass
class SampleCfg:
    g_open: int = 16
    rows_closed: int = 4
    k_closed: int = 8
    rho: float = 1.0
    cov_eps: float = 0.3
    tangent_mode: int = 0   # 0: Eq. 8's neighbour difference; 1: the derivative B'(t)

    def c(self):
        return bs_sample_cfg(self.g_open, self.rows_closed, self.k_closed, self.rho, self.cov_eps,
                             self.tangent_mode)


@dataclass
class Canvas:
    width: int
    height: int
    tile: int = 16
    bg: tuple = (0.0, 0.0, 0.0)

    def c(self):
        return bs_canvas(self.width, self.height, self.tile, (c_float * 3)(*self.bg))

    @property
    def n_tiles(self):
        t = self.tile
        return ((self.width + t - 1) // t) * ((self.height + t - 1) // t)


CURVE_FIELDS = ("open_ctrl", "open_width", "open_color", "open_opac",
                "closed_ctrl", "closed_color", "closed_opac")
FILL_FIELDS = ("closed_color2", "closed_opac2")


@dataclass
class CurveSet:
    """Device curve parameters (float32, contiguous) in pixel space with
    activated attributes; layouts as in bs.h."""
    open_ctrl: torch.Tensor     # [No,10,2]
    open_width: torch.Tensor    # [No]
    open_color: torch.Tensor    # [No,3]
    open_opac: torch.Tensor     # [No,3]
    closed_ctrl: torch.Tensor   # [Nc,12,2]
    closed_color: torch.Tensor  # [Nc,3]
    closed_opac: torch.Tensor   # [Nc]
    closed_color2: torch.Tensor = None  # [Nc,3] linear-gradient fill: colour at P6 (None: uniform)
    closed_opac2: torch.Tensor = None   # [Nc] opacity at P6 (None: uniform)

    @property
    def n_open(self):
        return int(self.open_ctrl.shape[0])

    @property
    def n_closed(self):
        return int(self.closed_ctrl.shape[0])

    def check(self):
        no, nc = self.n_open, self.n_closed
        shapes = dict(open_ctrl=(no, 10, 2), open_width=(no,), open_color=(no, 3), open_opac=(no, 3),
                      closed_ctrl=(nc, 12, 2), closed_color=(nc, 3), closed_opac=(nc,))
        shapes.update(closed_color2=(nc, 3), closed_opac2=(nc,))
        for k, s in shapes.items():
            if getattr(self, k) is not None:
                _want(getattr(self, k), torch.float32, s, k)
        return self

    def fields(self):
        """The names of the tensors this set holds (the fill fields when given)."""
        return CURVE_FIELDS + tuple(k for k in FILL_FIELDS if getattr(self, k) is not None)

    def c(self, draw_first=None):
        return bs_curves(self.n_open, self.n_closed, *(_ptr(getattr(self, k)) for k in CURVE_FIELDS),
                         _ptr(draw_first), *(_ptr(getattr(self, k)) for k in FILL_FIELDS))

    @staticmethod
    def from_arrays(arrays: dict, device="cuda"):
        return CurveSet(**{k: torch.as_tensor(arrays[k], dtype=torch.float32, device=device).contiguous()
                           for k in CURVE_FIELDS + FILL_FIELDS if k in arrays and arrays[k] is not None})

    def zeros_like(self):
        return CurveSet(**{k: torch.zeros_like(getattr(self, k)) for k in self.fields()})

    def grad_c(self):
        return bs_curves_grad(*(_ptr(getattr(self, k)) for k in CURVE_FIELDS + FILL_FIELDS))

    def mut_c(self):
        return bs_curves_mut(self.n_open, self.n_closed, *(_ptr(getattr(self, k)) for k in CURVE_FIELDS))


def num_gaussians(n_open, n_closed, cfg: SampleCfg) -> int:
    c = cfg.c()
    n = lib.bs_num_gaussians(n_open, n_closed, ctypes.byref(c))
    if n < 0:
        raise ValueError("invalid sample configuration")
    return int(n)


def curve_order(curves: CurveSet, cfg: SampleCfg, out=None):
    """rank [N] (0 = front) and first [N] Gaussian index, uint32 as int32
    (into out = (rank, first) when given)."""
    curves.check()
    n = curves.n_open + curves.n_closed
    dev = curves.open_ctrl.device
    if out is None:
        rank = torch.empty(n, dtype=torch.int32, device=dev)
        first = torch.empty(n, dtype=torch.int32, device=dev)
    else:
        rank, first = out
        _want(rank, torch.int32, (n,), "rank")
        _want(first, torch.int32, (n,), "first")
    c, k = curves.c(), cfg.c()
    _check("bs_curve_order", lib.bs_curve_order(ctypes.byref(c), ctypes.byref(k), _ptr(rank), _ptr(first),
                                                 _stream()))
    return rank, first


def sample_curves(curves: CurveSet, cfg: SampleCfg, first: torch.Tensor, out=None):
    ng = num_gaussians(curves.n_open, curves.n_closed, cfg)
    gauss = out if out is not None else torch.empty(ng, GAUSS_FLOATS, dtype=torch.float32,
                                                    device=curves.open_ctrl.device)
    _want(gauss, torch.float32, (ng, GAUSS_FLOATS), "gauss")
    c, k = curves.c(first), cfg.c()
    _check("bs_sample_curves", lib.bs_sample_curves(ctypes.byref(c), ctypes.byref(k), _ptr(gauss), _stream()))
    return gauss


def sample_curves_bwd(curves: CurveSet, cfg: SampleCfg, first: torch.Tensor, dgauss: torch.Tensor, grad=None):
    grad = grad if grad is not None else curves.zeros_like()
    c, k, g = curves.c(first), cfg.c(), grad.grad_c()
    _want(dgauss, torch.float32, None, "dgauss")
    _check("bs_sample_curves_bwd", lib.bs_sample_curves_bwd(ctypes.byref(c), ctypes.byref(k), _ptr(dgauss),
                                                             ctypes.byref(g), _stream()))
    return grad


def bin_tiles_workspace(n_gauss: int, canvas: Canvas, pair_capacity: int) -> int:
    cv = canvas.c()
    nb = c_size_t(0)
    _check("bs_bin_tiles_workspace", lib.bs_bin_tiles_workspace(n_gauss, ctypes.byref(cv), pair_capacity,
                                                                 ctypes.byref(nb)))
    return int(nb.value)


class Binning:
    """Device buffers of one binning: workspace, sorted keys, tile ranges.
    Grows its capacity when a call reports BS_ERR_CAPACITY."""

    def __init__(self, canvas: Canvas, device="cuda", pair_capacity: int = 1 << 20):
        self.canvas = canvas
        self.device = device
        self.capacity = 0
        self.n_gauss = -1
        self.ws = None
        self.keys = None
        self.ranges = torch.empty(canvas.n_tiles, 2, dtype=torch.int32, device=device)
        self._want_capacity = pair_capacity
        self.n_pairs = 0
        # allocations so far: a captured graph holds the addresses of the
        # buffers of one allocation, so it is stale once this count moves
        self.allocations = 0
        # whether the current workspace holds a binning (a new one holds none
        # until the next run), and the pairs of the last synchronising run
        self._binned = False
        self._last_pairs = 0

    def _alloc(self, n_gauss, capacity):
        nbytes = bin_tiles_workspace(n_gauss, self.canvas, capacity)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.keys = torch.empty(max(1, capacity), dtype=torch.int32, device=self.device)
        self.capacity = capacity
        self.n_gauss = n_gauss
        self.allocations += 1
        self._binned = False

    def run(self, gauss: torch.Tensor):
        n_gauss = int(gauss.shape[0])
        _want(gauss, torch.float32, (n_gauss, GAUSS_FLOATS), "gauss")
        if self.ws is None or n_gauss != self.n_gauss or self.capacity < self._want_capacity:
            self._alloc(n_gauss, max(self._want_capacity, self.capacity))
        cv = self.canvas.c()
        for _ in range(2):
            n_pairs = c_int64(0)
            st = lib.bs_bin_tiles(_ptr(gauss), n_gauss, ctypes.byref(cv), _ptr(self.ws), self.ws.numel(),
                                  self.capacity, ctypes.byref(n_pairs), _ptr(self.keys), _ptr(self.ranges),
                                  _stream())
            if st == BS_ERR_CAPACITY:
                self._want_capacity = int(n_pairs.value * 1.25) + 1024
                self._alloc(n_gauss, self._want_capacity)
                continue
            _check("bs_bin_tiles", st)
            self.n_pairs = int(n_pairs.value)
            self._last_pairs = self.n_pairs
            self._binned = True
            return self
        raise BSError("bs_bin_tiles", BS_ERR_CAPACITY)

    def prepare(self, n_gauss: int, capacity: int = None):
        """Allocate the workspace and key buffer for n_gauss Gaussians and
        `capacity` pairs (default: the current wish), once, ahead of run_async."""
        capacity = max(self._want_capacity, self.capacity) if capacity is None else capacity
        if self.ws is None or n_gauss != self.n_gauss or self.capacity < capacity:
            self._alloc(n_gauss, capacity)
        return self

    def fit(self, n_gauss: int, capacity: int):
        """prepare() for `capacity` pairs, also shrinking a capacity more than
        1.5 times that: the graph-safe binning sizes its grids by the
        capacity, so idle room costs launches of empty partitions."""
        if self.ws is None or n_gauss != self.n_gauss or self.capacity < capacity or self.capacity > 1.5 * capacity:
            self._alloc(n_gauss, capacity)
        self._want_capacity = capacity
        return self

    def run_async(self, gauss: torch.Tensor, n_pairs_dev: torch.Tensor = None):
        """bs_bin_tiles_async: the binning with no read-back, graph-capturable.
        The buffers must have been sized (prepare) beforehand; an overflow
        shows in result().  n_pairs_dev: optional device int64 [1] for P."""
        n_gauss = int(gauss.shape[0])
        _want(gauss, torch.float32, (n_gauss, GAUSS_FLOATS), "gauss")
        if self.ws is None or n_gauss != self.n_gauss:
            raise RuntimeError("Binning.run_async needs prepare(n_gauss) first (no allocation while capturing)")
        if n_pairs_dev is not None:
            _want(n_pairs_dev, torch.int64, (1,), "n_pairs_dev")
        cv = self.canvas.c()
        _check("bs_bin_tiles_async", lib.bs_bin_tiles_async(_ptr(gauss), n_gauss, ctypes.byref(cv), _ptr(self.ws),
                                                             self.ws.numel(), self.capacity, _ptr(n_pairs_dev),
                                                             _ptr(self.keys), _ptr(self.ranges), _stream()))
        self.n_pairs = None
        self._binned = True
        return self

    def result(self):
        """(status, P) of the last binning (synchronises): BS_OK or
        BS_ERR_CAPACITY, and the pairs it found; sets n_pairs.  When the
        buffers were allocated anew since the last binning (prepare, fit),
        the workspace holds none: the last synchronising run's pairs are
        reported against the new capacity."""
        if not self._binned:
            self.n_pairs = self._last_pairs
            return (BS_OK if self._last_pairs <= self.capacity else BS_ERR_CAPACITY), self._last_pairs
        st, n = c_int32(0), c_int64(0)
        _check("bs_bin_tiles_result", lib.bs_bin_tiles_result(_ptr(self.ws), self.ws.numel(), ctypes.byref(st),
                                                               ctypes.byref(n), _stream()))
        self.n_pairs = int(n.value)
        return int(st.value), int(n.value)

    def device_status(self) -> int:
        if not self._binned:   # buffers allocated anew since the last binning: nothing recorded
            return BS_OK
        out = c_int32(0)
        _check("bs_device_status", lib.bs_device_status(_ptr(self.ws), self.ws.numel(), ctypes.byref(out),
                                                         _stream()))
        return int(out.value)


def sync_status(clear: bool = True) -> int:
    """bs_sync_status: BS_OK, or BS_ERR_NOT_FINITE when a sampling or
    backward kernel wrote a non-finite record or gradient since the last
    clear (synchronises the current stream)."""
    out = c_int32(0)
    _check("bs_sync_status", lib.bs_sync_status(1 if clear else 0, ctypes.byref(out), _stream()))
    return int(out.value)


def bin_tiles_static(gauss: torch.Tensor, canvas: Canvas, tile_keys: torch.Tensor, tile_ranges: torch.Tensor):
    """bs_bin_tiles_static: binning with the library's fixed scratch (no
    workspace argument).  tile_keys [pair_capacity] and tile_ranges
    [n_tiles, 2] int32 are the caller's; returns the pair count."""
    n_gauss = int(gauss.shape[0])
    _want(gauss, torch.float32, (n_gauss, GAUSS_FLOATS), "gauss")
    _want(tile_keys, torch.int32, None, "tile_keys")
    _want(tile_ranges, torch.int32, (canvas.n_tiles, 2), "tile_ranges")
    cv = canvas.c()
    n_pairs = c_int64(0)
    _check("bs_bin_tiles_static", lib.bs_bin_tiles_static(_ptr(gauss), n_gauss, ctypes.byref(cv),
                                                           tile_keys.numel(), ctypes.byref(n_pairs),
                                                           _ptr(tile_keys), _ptr(tile_ranges), _stream()))
    return int(n_pairs.value)


def render_fwd(gauss: torch.Tensor, canvas: Canvas, binning: Binning, out=None):
    W, H = canvas.width, canvas.height
    dev = gauss.device
    if out is None:
        out = (torch.empty(3, H, W, dtype=torch.float32, device=dev),
               torch.empty(H, W, dtype=torch.float32, device=dev),
               torch.empty(H, W, dtype=torch.int32, device=dev))
    img, T, nc = out
    cv = canvas.c()
    _check("bs_render_fwd", lib.bs_render_fwd(_ptr(gauss), int(gauss.shape[0]), ctypes.byref(cv),
                                               _ptr(binning.keys), _ptr(binning.ranges), _ptr(img), _ptr(T),
                                               _ptr(nc), _stream()))
    return img, T, nc


def render_fwd_l2(gauss: torch.Tensor, canvas: Canvas, binning: Binning, target: torch.Tensor, out=None,
                  dimg=None, loss=None):
    """Forward blend and the L2 loss gradient in one pass: (img, T_final,
    n_contrib), dL/dimg, loss (device double)."""
    W, H = canvas.width, canvas.height
    dev = gauss.device
    _want(target, torch.float32, (3, H, W), "target")
    if out is None:
        out = (torch.empty(3, H, W, dtype=torch.float32, device=dev),
               torch.empty(H, W, dtype=torch.float32, device=dev),
               torch.empty(H, W, dtype=torch.int32, device=dev))
    img, T, nc = out
    dimg = dimg if dimg is not None else torch.empty_like(img)
    loss = loss if loss is not None else torch.empty((), dtype=torch.float64, device=dev)
    cv = canvas.c()
    _check("bs_render_fwd_l2", lib.bs_render_fwd_l2(_ptr(gauss), int(gauss.shape[0]), ctypes.byref(cv),
                                                     _ptr(binning.keys), _ptr(binning.ranges), _ptr(target),
                                                     _ptr(img), _ptr(T), _ptr(nc), _ptr(dimg),
                                                     c_void_p(loss.data_ptr()), _stream()))
    return (img, T, nc), dimg, loss


def render_stats(gauss: torch.Tensor, canvas: Canvas, binning: Binning):
    """Work counters of a forward blend: dict(evals (performed), blended,
    tile_px_entries, visits (entries up to each pixel's stop point),
    n_contrib_sum)."""
    W, H = canvas.width, canvas.height
    dev = gauss.device
    img = torch.empty(3, H, W, dtype=torch.float32, device=dev)
    T = torch.empty(H, W, dtype=torch.float32, device=dev)
    nc = torch.empty(H, W, dtype=torch.int32, device=dev)
    st = torch.zeros(4, dtype=torch.int64, device=dev)
    cv = canvas.c()
    _check("bs_render_stats", lib.bs_render_stats(_ptr(gauss), int(gauss.shape[0]), ctypes.byref(cv),
                                                   _ptr(binning.keys), _ptr(binning.ranges), _ptr(img), _ptr(T),
                                                   _ptr(nc), _ptr(st), _stream()))
    v = st.cpu().tolist()
    return dict(evals=v[0], blended=v[1], tile_px_entries=v[2], visits=v[3], n_contrib_sum=int(nc.sum().item()))


def l2_loss_grad(img: torch.Tensor, target: torch.Tensor, dimg=None, loss=None):
    _want(img, torch.float32, None, "img")
    _want(target, torch.float32, tuple(img.shape), "target")
    dimg = dimg if dimg is not None else torch.empty_like(img)
    loss = loss if loss is not None else torch.empty((), dtype=torch.float64, device=img.device)
    _check("bs_l2_loss_grad", lib.bs_l2_loss_grad(_ptr(img), _ptr(target), img.numel(), _ptr(dimg),
                                                   c_void_p(loss.data_ptr()), _stream()))
    return loss, dimg


def render_bwd(gauss, canvas: Canvas, binning: Binning, T_final, n_contrib, dimg, dgauss=None,
               curves: CurveSet = None, cfg: SampleCfg = None, first=None, grad: CurveSet = None):
    """Per-Gaussian gradients, and (when curves is given) curve gradients."""
    ng = int(gauss.shape[0])
    dgauss = dgauss if dgauss is not None else torch.empty(ng, DGAUSS_FLOATS, dtype=torch.float32,
                                                           device=gauss.device)
    cv = canvas.c()
    if curves is not None:
        grad = grad if grad is not None else curves.zeros_like()
        c, k, g = curves.c(first), cfg.c(), grad.grad_c()
        cp, kp, gp = ctypes.byref(c), ctypes.byref(k), ctypes.byref(g)
    else:
        cp = kp = gp = None
    _check("bs_render_bwd", lib.bs_render_bwd(_ptr(gauss), ng, ctypes.byref(cv), _ptr(binning.keys),
                                               _ptr(binning.ranges), _ptr(T_final), _ptr(n_contrib),
                                               _ptr(dimg), _ptr(dgauss), cp, kp, gp, _stream()))
    return dgauss, grad


@dataclass
class PDCfg:
    """Parameters of one pruning/densification pass (bs_pd_cfg)."""
    op_start: float = 0.2
    op_end: float = 0.02
    step: int = 0
    t_end: int = 1
    area_min: float = 4.0
    color_eps: float = 0.03
    iou_min: float = 0.9
    err_thresh: float = 0.1
    split_drop: float = 0.5
    new_opacity: float = 0.5
    new_width: float = 2.0

    def c(self):
        return bs_pd_cfg(self.op_start, self.op_end, self.step, self.t_end, self.area_min, self.color_eps,
                         self.iou_min, self.err_thresh, self.split_drop, self.new_opacity, self.new_width)


def prune_densify_workspace(n_open: int, n_closed: int, canvas: Canvas) -> int:
    cv = canvas.c()
    nb = c_size_t(0)
    _check("bs_prune_densify_workspace", lib.bs_prune_densify_workspace(n_open, n_closed, ctypes.byref(cv),
                                                                         ctypes.byref(nb)))
    return int(nb.value)


def prune_densify(curves: CurveSet, img: torch.Tensor, target: torch.Tensor, cfg: PDCfg, canvas: Canvas,
                  ws: torch.Tensor = None, changed: torch.Tensor = None):
    """One pruning/densification pass, in place on `curves`.  Returns the
    per-curve changed mask (uint8) and the pass's counts.  Synchronises."""
    curves.check()
    n = curves.n_open + curves.n_closed
    shape = (3, canvas.height, canvas.width)
    _want(img, torch.float32, shape, "img")
    _want(target, torch.float32, shape, "target")
    dev = img.device
    nbytes = prune_densify_workspace(curves.n_open, curves.n_closed, canvas)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    changed = changed if changed is not None else torch.empty(max(1, n), dtype=torch.uint8, device=dev)
    c, k, cv = curves.mut_c(), cfg.c(), canvas.c()
    st = bs_pd_stats()
    _check("bs_prune_densify", lib.bs_prune_densify(ctypes.byref(c), ctypes.byref(k), ctypes.byref(cv), _ptr(img),
                                                     _ptr(target), _ptr(ws), ws.numel(), _ptr(changed),
                                                     ctypes.byref(st), _stream()))
    return changed[:n], {f: int(getattr(st, f)) for f, _ in bs_pd_stats._fields_}


def debug_umma_wait(first_wait: int = -1):
    """Test hook: the tries of the tensor-core GEMM's wait for its last MMA
    commit (< 0 restores the default; 0 gives up at once, which makes the
    network calls return BS_ERR_TIMEOUT)."""
    _check("bs_debug_umma_wait", lib.bs_debug_umma_wait(first_wait))


def debug_retry_limit(max_attempts: int = -1):
    """Test hook: bound the device-side retry loops (the union step of the
    region labelling) to max_attempts linking attempts (< 0 restores the
    default bound; 0 makes every union with anything to link give up)."""
    _check("bs_debug_retry_limit", lib.bs_debug_retry_limit(max_attempts))


# ---------------------------------------------------------------------------
# Batches of images (bs_batch_*) and the Adam step (bs_adam_step)

@dataclass
class BatchImage:
    """One image of a batch: canvas, curve counts, sampling, background."""
    width: int
    height: int
    n_open: int
    n_closed: int
    sample: SampleCfg
    bg: tuple = (0.0, 0.0, 0.0)

    def c(self):
        return bs_batch_image(self.width, self.height, self.n_open, self.n_closed, self.sample.c(),
                              (c_float * 3)(*self.bg))


def batch_sizes(images, tile: int = 16, pair_capacity: int = 1 << 20) -> dict:
    """bs_batch_plan (host arithmetic only, no device needed): the totals of
    a batch of BatchImage and its workspace bytes."""
    arr = (bs_batch_image * len(images))(*(im.c() for im in images))
    b = bs_batch(ctypes.cast(arr, c_void_p), len(images), int(tile), int(pair_capacity), None, 0)
    sz = bs_batch_sizes()
    _check("bs_batch_plan", lib.bs_batch_plan(ctypes.byref(b), ctypes.byref(sz)))
    return {f: int(getattr(sz, f)) for f, _ in bs_batch_sizes._fields_}


class Batch:
    """The layout of a batch and its device workspace (bs_batch_plan,
    bs_batch_setup).  Host-side offsets of every image's curves, Gaussians,
    pixels and tiles in the concatenated arrays are kept for slicing."""

    def __init__(self, images, tile: int = 16, pair_capacity: int = 1 << 22, device="cuda"):
        self.images = list(images)
        self.tile = int(tile)
        self.device = device
        self._arr = (bs_batch_image * len(self.images))(*(im.c() for im in self.images))
        self._plan(pair_capacity)
        no = [im.n_open for im in self.images]
        nc = [im.n_closed for im in self.images]
        ng = [im.n_open * im.sample.g_open + im.n_closed * im.sample.rows_closed * im.sample.k_closed
              for im in self.images]
        npx = [im.width * im.height for im in self.images]
        nt = [(-(-im.width // self.tile)) * (-(-im.height // self.tile)) for im in self.images]

        def prefix(v):
            out, acc = [], 0
            for x in v:
                out.append(acc)
                acc += x
            return out
        self.open0, self.closed0, self.gauss0 = prefix(no), prefix(nc), prefix(ng)
        self.pix0, self.tile0 = prefix(npx), prefix(nt)
        self.n_gauss_of = ng

    def _plan(self, pair_capacity):
        self.pair_capacity = int(pair_capacity)
        sz = bs_batch_sizes()
        b = bs_batch(ctypes.cast(self._arr, c_void_p), len(self.images), self.tile, self.pair_capacity, None, 0)
        _check("bs_batch_plan", lib.bs_batch_plan(ctypes.byref(b), ctypes.byref(sz)))
        self.sizes = sz
        self.n_open, self.n_closed = int(sz.n_open), int(sz.n_closed)
        self.n_gauss, self.n_pixels, self.n_tiles = int(sz.n_gauss), int(sz.n_pixels), int(sz.n_tiles)
        self.ws = torch.empty(int(sz.ws_bytes), dtype=torch.uint8, device=self.device)
        _check("bs_batch_setup", lib.bs_batch_setup(ctypes.byref(self.c()), _stream()))

    def grow(self, pair_capacity: int):
        """Re-plan with a larger pair capacity (new workspace, new table)."""
        self._plan(pair_capacity)

    def c(self):
        return bs_batch(ctypes.cast(self._arr, c_void_p), len(self.images), self.tile, self.pair_capacity,
                        _ptr(self.ws), self.ws.numel())

    def image(self, t: torch.Tensor, b: int):
        """Image b's [3, H, W] view of a batch image buffer [3 n_pixels]."""
        im = self.images[b]
        n = im.width * im.height
        return t[3 * self.pix0[b]:3 * (self.pix0[b] + n)].view(3, im.height, im.width)

    def pixel_map(self, t: torch.Tensor, b: int):
        """Image b's [H, W] view of a per-pixel buffer [n_pixels]."""
        im = self.images[b]
        return t[self.pix0[b]:self.pix0[b] + im.width * im.height].view(im.height, im.width)

    def curve_order(self, curves: CurveSet, rank=None, first=None):
        n = curves.n_open + curves.n_closed
        rank = rank if rank is not None else torch.empty(n, dtype=torch.int32, device=self.device)
        first = first if first is not None else torch.empty(n, dtype=torch.int32, device=self.device)
        c, b = curves.c(), self.c()
        _check("bs_batch_curve_order", lib.bs_batch_curve_order(ctypes.byref(b), ctypes.byref(c), _ptr(rank),
                                                                 _ptr(first), _stream()))
        return rank, first

    def sample_curves(self, curves: CurveSet, first, out=None):
        gauss = out if out is not None else torch.empty(self.n_gauss, GAUSS_FLOATS, dtype=torch.float32,
                                                        device=self.device)
        _want(gauss, torch.float32, (self.n_gauss, GAUSS_FLOATS), "gauss")
        c, b = curves.c(first), self.c()
        _check("bs_batch_sample_curves", lib.bs_batch_sample_curves(ctypes.byref(b), ctypes.byref(c), _ptr(gauss),
                                                                     _stream()))
        return gauss

    def bin_tiles(self, gauss, vals, ranges):
        _want(vals, torch.int32, None, "tile_vals")
        _want(ranges, torch.int32, (self.n_tiles, 2), "tile_ranges")
        if vals.numel() < self.pair_capacity:
            raise ValueError("tile_vals must hold pair_capacity entries")
        b = self.c()
        _check("bs_batch_bin_tiles", lib.bs_batch_bin_tiles(ctypes.byref(b), _ptr(gauss), _ptr(vals), _ptr(ranges),
                                                             _stream()))

    def render_fwd(self, gauss, vals, ranges, img, T, nc, target=None, dimg=None, loss=None):
        b = self.c()
        _check("bs_batch_render_fwd", lib.bs_batch_render_fwd(
            ctypes.byref(b), _ptr(gauss), _ptr(vals), _ptr(ranges), _ptr(target), _ptr(img), _ptr(T), _ptr(nc),
            _ptr(dimg), c_void_p(loss.data_ptr()) if loss is not None else c_void_p(0), _stream()))

    def render_bwd(self, gauss, vals, ranges, T, nc, dimg, dgauss, curves: CurveSet = None, first=None,
                   grad: CurveSet = None):
        b = self.c()
        if grad is not None:
            c, g = curves.c(first), grad.grad_c()
            cp, gp = ctypes.byref(c), ctypes.byref(g)
        else:
            cp = gp = None
        _check("bs_batch_render_bwd", lib.bs_batch_render_bwd(
            ctypes.byref(b), _ptr(gauss), _ptr(vals), _ptr(ranges), _ptr(T), _ptr(nc), _ptr(dimg), _ptr(dgauss),
            cp, gp, _stream()))

    def status(self):
        """(status, pairs found by the last binning); synchronises."""
        st, n = c_int32(0), c_int64(0)
        b = self.c()
        _check("bs_batch_status", lib.bs_batch_status(ctypes.byref(b), ctypes.byref(st), ctypes.byref(n), _stream()))
        return int(st.value), int(n.value)


@dataclass
class AdamGroup:
    """One parameter group of bs_adam_step: param, grad, and its moments (all
    float32 device tensors of the same size), lr, box [lo, hi], optional
    per-row lr multipliers."""
    param: torch.Tensor
    grad: torch.Tensor
    m: torch.Tensor
    v: torch.Tensor
    lr: float
    lo: float = -3.0e38
    hi: float = 3.0e38
    row_scale: torch.Tensor = None
    row_len: int = 1

    def c(self):
        for k in ("param", "grad", "m", "v"):
            _want(getattr(self, k), torch.float32, None, k)
        n = self.param.numel()
        if any(getattr(self, k).numel() != n for k in ("grad", "m", "v")):
            raise ValueError("param, grad, m and v must have the same size")
        return bs_adam_group(_ptr(self.param), _ptr(self.grad), _ptr(self.m), _ptr(self.v), n, self.lr, self.lo,
                             self.hi, _ptr(self.row_scale), int(self.row_len))


def adam_step(groups, step: torch.Tensor, beta1=0.9, beta2=0.999, eps=1e-8):
    """bs_adam_step over up to 16 groups; step is a device int32 scalar
    (advanced by one on the device)."""
    if not 1 <= len(groups) <= ADAM_MAX_GROUPS:
        raise ValueError("1 to 16 groups")
    _want(step, torch.int32, None, "step")
    arr = (bs_adam_group * len(groups))(*(g.c() for g in groups))
    cfg = bs_adam_cfg(beta1, beta2, eps)
    _check("bs_adam_step", lib.bs_adam_step(arr, len(groups), ctypes.byref(cfg), _ptr(step), _stream()))


# ---------------------------------------------------------------------------
# The learned initialiser's network (bs_net_*)

def net_param_count(layer: int) -> int:
    n = lib.bs_net_param_count(layer)
    if n < 0:
        raise ValueError("layer out of range")
    return int(n)


def net_workspace(n: int, side: int) -> int:
    nb = c_size_t(0)
    _check("bs_net_workspace", lib.bs_net_workspace(n, side, ctypes.byref(nb)))
    return int(nb.value)


def _net_c(w, w_bf16):
    return bs_net((c_void_p * NET_LAYERS)(*(t.data_ptr() for t in w)),
                  (c_void_p * NET_LAYERS)(*(t.data_ptr() for t in w_bf16)))


def net_sync_weights(w, w_bf16):
    """w: 6 float32 master tensors, w_bf16: 6 int16 tensors (bf16 bits)."""
    net = _net_c(w, w_bf16)
    _check("bs_net_sync_weights", lib.bs_net_sync_weights(ctypes.byref(net), _stream()))


NET_CURVE_SHAPES = dict(ctrl=(12, 2), color=(3,), opac=(), open_ctrl=(10, 2), open_width=(), open_color=(3,),
                        open_opac=(3,))


def _net_curves_c(curves: dict, n: int, cells: int, need_all: bool):
    """bs_net_curves of a dict of float32 device tensors [n, cells, ...]
    (missing keys NULL unless need_all)."""
    ptrs = {}
    for k in NET_CURVE_KEYS:
        t = curves.get(k)
        if t is None:
            if need_all:
                raise ValueError(f"target {k} is missing")
            ptrs[k] = None
            continue
        _want(t, torch.float32, (n, cells) + NET_CURVE_SHAPES[k], k)
        ptrs[k] = t.data_ptr()
    return bs_net_curves(**ptrs)


def net_forward(w, w_bf16, patches, ws, head=None, curves: dict = None):
    """Head outputs to `head` [n, cells, 64] and proposals into the tensors
    of `curves` (keys NET_CURVE_KEYS, any subset)."""
    _want(patches, torch.float32, None, "patches")
    n, side = int(patches.shape[0]), int(patches.shape[-1])
    net = _net_c(w, w_bf16)
    c = _net_curves_c(curves, n, (side // 32) ** 2, False) if curves else None
    _check("bs_net_forward", lib.bs_net_forward(ctypes.byref(net), _ptr(patches), n, side, _ptr(ws), ws.numel(),
                                                 _ptr(head), ctypes.byref(c) if c is not None else None, _stream()))


def net_train_step(w, w_bf16, grads, patches, targets: dict, ws, loss):
    """targets: every key of NET_CURVE_KEYS, float32 device [n, cells, ...]."""
    _want(patches, torch.float32, None, "patches")
    n, side = int(patches.shape[0]), int(patches.shape[-1])
    net = _net_c(w, w_bf16)
    t = _net_curves_c(targets, n, (side // 32) ** 2, True)
    g = bs_net_grad((c_void_p * NET_LAYERS)(*(x.data_ptr() for x in grads)))
    _check("bs_net_train_step", lib.bs_net_train_step(ctypes.byref(net), _ptr(patches), n, side, ctypes.byref(t),
                                                       _ptr(ws), ws.numel(), ctypes.byref(g),
                                                       c_void_p(loss.data_ptr()), _stream()))


# ---------------------------------------------------------------------------
# Xing loss (bs_xing_loss) and SVG export (bs_svg_export)

def xing_loss(curves: CurveSet, lam: float, grad_closed_ctrl: torch.Tensor = None, loss=None):
    """lambda * mean Xing loss of the closed curves (device double); adds its
    gradient to grad_closed_ctrl when given."""
    loss = loss if loss is not None else torch.empty((), dtype=torch.float64, device=curves.closed_ctrl.device)
    c = curves.c()
    if grad_closed_ctrl is not None:
        _want(grad_closed_ctrl, torch.float32, tuple(curves.closed_ctrl.shape), "grad_closed_ctrl")
    _check("bs_xing_loss", lib.bs_xing_loss(ctypes.byref(c), lam, c_void_p(loss.data_ptr()), _ptr(grad_closed_ctrl),
                                             _stream()))
    return loss


def svg_export(arrays: dict, width: int, height: int, rank=None, own_opacity: bool = False) -> str:
    """The SVG document of host curve arrays (numpy, the CurveSet fields,
    optionally closed_color2 / closed_opac2), back to front by draw rank."""
    import numpy as np
    keep = []

    def hp(k, dtype=np.float32):
        v = arrays.get(k)
        if v is None:
            return c_void_p(0)
        a = np.ascontiguousarray(np.asarray(v, dtype=dtype))
        keep.append(a)
        return c_void_p(a.ctypes.data) if a.size else c_void_p(0)
    no = int(np.asarray(arrays["open_ctrl"]).shape[0])
    nc = int(np.asarray(arrays["closed_ctrl"]).shape[0])
    c = bs_curves(no, nc, *(hp(k) for k in CURVE_FIELDS), c_void_p(0), *(hp(k) for k in FILL_FIELDS))
    r = c_void_p(0)
    if rank is not None:
        ra = np.ascontiguousarray(np.asarray(rank, dtype=np.uint32))
        keep.append(ra)
        r = c_void_p(ra.ctypes.data)
    need = c_size_t(0)
    flags = 1 if own_opacity else 0
    _check("bs_svg_export", lib.bs_svg_export(ctypes.byref(c), r, width, height, flags, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check("bs_svg_export", lib.bs_svg_export(ctypes.byref(c), r, width, height, flags, buf, need.value,
                                               ctypes.byref(need)))
    return buf.value.decode()


def debug_gemm_engine(engine: int):
    """Test hook: the network GEMM engine for later calls (1 tcgen05, 0
    mma.sync); returns the tcgen05 tiles that gave up a bounded wait so far."""
    t = c_int64(0)
    _check("bs_debug_gemm_engine", lib.bs_debug_gemm_engine(engine, ctypes.byref(t)))
    return int(t.value)
