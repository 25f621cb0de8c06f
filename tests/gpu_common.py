"""Shared helpers of the GPU parity tests: run libpam and the oracle on the
same seeded inputs and compare them element by element.

Tolerances (FP32 path vs FP64 oracle):
  energy maps (I_TAX, I_AS, backprop energy): relative L2 <= 1e-5
  NCC maps (rho_pairs, rho_n): max |difference| <= 1e-5
  brightest pixel: identical
"""
from __future__ import annotations

import numpy as np

import oracle

REL_L2_TOL = 1e-5
NCC_TOL = 1e-5


def rel_l2(got, want) -> float:
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = np.linalg.norm(want.ravel())
    return float(np.linalg.norm((got - want).ravel()) / (den if den > 0 else 1.0))


def peak(a):
    a = np.asarray(a)
    return tuple(int(v) for v in np.unravel_index(np.argmax(a), a.shape))


def peak_margin(a) -> float:
    """Relative gap between the largest and second-largest pixel."""
    v = np.sort(np.asarray(a, dtype=np.float64).ravel())
    return float((v[-1] - v[-2]) / v[-1]) if v[-1] > 0 else 0.0


def geometry_of(w, bins=None, evanescent_zero=False):
    return oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz,
                           w.bins() if bins is None else bins, evanescent_zero=evanescent_zero)


def compare_xcorr(gpu: dict, orc: dict, f: int = 0, check_peak: bool = True) -> dict:
    """Compare one frame of a libpam xcorr result (torch tensors) with the oracle."""
    m = {}
    img = gpu["image"][f].cpu().numpy()
    m["image_rel_l2"] = rel_l2(img, orc["image"])
    if "image_as" in gpu:
        m["image_as_rel_l2"] = rel_l2(gpu["image_as"][f].cpu().numpy(), orc["image_as"])
    if "rho_pairs" in gpu:
        m["rho_pairs_max_abs"] = float(np.max(np.abs(gpu["rho_pairs"][f].cpu().numpy() - orc["rho_pairs"])))
    if "rho_n" in gpu:
        m["rho_n_max_abs"] = float(np.max(np.abs(gpu["rho_n"][f].cpu().numpy() - orc["rho_n"])))
    assert m["image_rel_l2"] <= REL_L2_TOL, m
    if "image_as_rel_l2" in m:
        assert m["image_as_rel_l2"] <= REL_L2_TOL, m
    if "rho_pairs_max_abs" in m:
        assert m["rho_pairs_max_abs"] <= NCC_TOL, m
    if "rho_n_max_abs" in m:
        assert m["rho_n_max_abs"] <= NCC_TOL, m
    if check_peak:
        m["peak"] = peak(img)
        m["peak_margin"] = peak_margin(orc["image"])
        assert m["peak"] == peak(orc["image"]), m
    return m
