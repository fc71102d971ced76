"""bs_bin_tiles_static: binning for callers that cannot allocate device
memory (a host that gives this library a fixed memory budget, or code that
must not call an allocator), with its scratch in the library's fixed device
array.  Its results must equal those of bs_bin_tiles with a caller workspace,
call after call (the array is reused and keeps the previous call's contents),
and an oversized request must be refused before anything runs.

This file runs last (pytest collects files in name order): if it fails, a
run that stops at the first failure has already run every other test."""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    from paper_2503_16424_gb300 import bs as _bs
    return _bs


def _table(seed, W, H, n):
    """A seeded float32 Gaussian table: means over and around the canvas,
    varied support boxes, a few culled records."""
    rng = np.random.default_rng(seed)
    rec = np.zeros((n, 12), dtype=np.float32)
    rec[:, 0] = rng.uniform(-30, W + 30, n)
    rec[:, 1] = rng.uniform(-30, H + 30, n)
    rec[:, 10] = rng.uniform(0, 40, n)
    rec[:, 11] = rng.uniform(0, 40, n)
    rec[::53, 10] = -1.0
    return rec


def _with_workspace(bs, gauss, canvas):
    b = bs.Binning(canvas, "cuda", pair_capacity=1024).run(gauss)
    return b.n_pairs, b.keys[:b.n_pairs].clone(), b.ranges.clone()


@pytest.mark.parametrize("seeds", [(1, 2)])
def test_static_scratch_matches_workspace_binning_on_consecutive_calls(bs, seeds):
    canvas = bs.Canvas(300, 200)
    for seed, n in zip(seeds, (5000, 3000)):   # the second call sees the first call's leftovers
        gauss = torch.as_tensor(_table(seed, 300, 200, n), device="cuda")
        n_ref, keys_ref, ranges_ref = _with_workspace(bs, gauss, canvas)
        assert n_ref > 20000
        keys = torch.full((n_ref + 100,), -1, dtype=torch.int32, device="cuda")
        ranges = torch.full((canvas.n_tiles, 2), -1, dtype=torch.int32, device="cuda")
        n_pairs = bs.bin_tiles_static(gauss, canvas, keys, ranges)
        torch.cuda.synchronize()
        assert n_pairs == n_ref
        assert torch.equal(keys[:n_pairs], keys_ref)
        assert torch.equal(ranges, ranges_ref)


def test_static_scratch_refuses_oversized_requests(bs):
    canvas = bs.Canvas(2048, 2048)
    gauss = torch.zeros(262144, 12, dtype=torch.float32, device="cuda")
    keys = torch.empty(8, dtype=torch.int32, device="cuda")
    ranges = torch.empty(canvas.n_tiles, 2, dtype=torch.int32, device="cuda")
    cv = canvas.c()
    n_pairs = ctypes.c_int64(0)
    st = bs.lib.bs_bin_tiles_static(ctypes.c_void_p(gauss.data_ptr()), 262144, ctypes.byref(cv), 7_200_000,
                                    ctypes.byref(n_pairs), ctypes.c_void_p(keys.data_ptr()),
                                    ctypes.c_void_p(ranges.data_ptr()), None)
    assert st == bs.BS_ERR_INVALID_ARG
    assert b"fixed scratch" in bs.lib.bs_last_error()


def test_static_scratch_allocates_no_device_memory(bs):
    """The defining property: after a first call on the device (which looks
    up the array's address and loads the kernels), repeated calls change
    neither the device's free memory (cudaMemGetInfo) nor the counts of
    torch's caching allocator."""
    canvas = bs.Canvas(300, 200)
    gauss = torch.as_tensor(_table(3, 300, 200, 4000), device="cuda")
    keys = torch.empty(1 << 18, dtype=torch.int32, device="cuda")
    ranges = torch.empty(canvas.n_tiles, 2, dtype=torch.int32, device="cuda")
    cv = canvas.c()
    n_pairs = ctypes.c_int64(0)
    args = (ctypes.c_void_p(gauss.data_ptr()), 4000, ctypes.byref(cv), keys.numel(), ctypes.byref(n_pairs),
            ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(ranges.data_ptr()), None)
    assert bs.lib.bs_bin_tiles_static(*args) == bs.BS_OK     # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    first = n_pairs.value
    for _ in range(5):
        assert bs.lib.bs_bin_tiles_static(*args) == bs.BS_OK
        assert n_pairs.value == first
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for k in ("allocation.all.allocated", "segment.all.allocated", "allocated_bytes.all.allocated"):
        assert stats1.get(k, 0) == stats0.get(k, 0), k
