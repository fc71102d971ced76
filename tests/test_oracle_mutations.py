"""Planted mistakes in the oracle (on the CPU, via monkeypatch) must each be
caught by one of the pins, showing the pins are not vacuous."""

import pytest
import torch

import oracle.curves as curves_mod
import oracle.raster as raster_mod
import tests.test_oracle_geometry as tg
import tests.test_oracle_raster as tr


def _expect_fail(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_flipped_rotation_is_caught(monkeypatch):
    orig = raster_mod._alpha_raw

    def bad(tab, px, py):
        t = dict(tab)
        t["uy"] = -tab["uy"]
        return orig(t, px, py)
    monkeypatch.setattr(raster_mod, "_alpha_raw", bad)
    _expect_fail(tr.test_single_rotated_gaussian_matches_density_ratio)


def test_dropped_transmittance_is_caught(monkeypatch):
    orig_cumprod = torch.cumprod

    def bad_cumprod(x, dim):
        return torch.ones_like(x)            # T = 1 for every Gaussian
    monkeypatch.setattr(raster_mod.torch, "cumprod", bad_cumprod)
    try:
        _expect_fail(tr.test_scan_form_equals_sequential_loop, 0)
    finally:
        monkeypatch.setattr(raster_mod.torch, "cumprod", orig_cumprod)


def test_reversed_boundary_is_caught(monkeypatch):
    def bad(ctrl):
        A = ctrl[:, 0:7]
        B = torch.cat([ctrl[:, 0:1], ctrl[:, [7, 8, 9, 10, 11, 6]]], dim=1)
        return A, B
    monkeypatch.setattr(curves_mod, "closed_boundaries", bad)
    monkeypatch.setattr(tg.oracle, "closed_boundaries", bad)
    _expect_fail(tg.test_closed_boundaries_order)


def test_swapped_scales_are_caught(monkeypatch):
    orig = raster_mod._alpha_raw

    def bad(tab, px, py):
        t = dict(tab)
        t["isx"], t["isy"] = tab["isy"], tab["isx"]
        return orig(t, px, py)
    monkeypatch.setattr(raster_mod, "_alpha_raw", bad)
    _expect_fail(tr.test_single_rotated_gaussian_matches_density_ratio)


def test_swapped_sigma_axes_is_caught(monkeypatch):
    orig = curves_mod.covariance

    def bad(theta, sx, sy, eps):
        return orig(theta, sy, sx, eps)
    monkeypatch.setattr(tg.oracle, "covariance", bad)
    _expect_fail(tg.test_covariance_eigen_structure)


def test_wrong_segment_opacity_is_caught(monkeypatch):
    orig = curves_mod.chain_sample_params

    def bad(K, S):
        s, t = orig(K, S)
        return s[::-1].copy(), t
    monkeypatch.setattr(curves_mod, "chain_sample_params", bad)
    _expect_fail(tg.test_open_straight_line_closed_form, 16)
