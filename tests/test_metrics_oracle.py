"""Pins of oracle/metrics.py: hand-computed maps (ESA, Eq. 12 ISNR, Eq. 13
centroid), a symmetric blob, the degenerate maps, and Eq. 20's closed forms."""
import math

import numpy as np

from oracle import metrics


def test_hand_computed_map():
    img = np.array([[0, 1, 0], [1, 4, 3], [0, 1, 0]], dtype=np.float32)
    r = metrics.measures(img, x0=-1e-3, dx=1e-3, z0=10e-3, dz=2e-3, alpha=0.7)
    # half max = 2: inside {4, 3}; outside 7 pixels summing to 3
    assert r["n_inside"] == 2
    assert math.isclose(r["esa_m2"], 2 * 1e-3 * 2e-3)
    assert math.isclose(r["isnr_db"], 10 * math.log10(3.5 / (3 / 7)), rel_tol=1e-12)
    # alpha max = 2.8: pixels 4 at (x=0, z=12 mm) and 3 at (x=1 mm, z=12 mm)
    assert math.isclose(r["cx_m"], (4 * 0.0 + 3 * 1e-3) / 7, rel_tol=1e-12)
    assert math.isclose(r["cz_m"], 12e-3, rel_tol=1e-12)
    assert r["max"] == 4.0


def test_symmetric_blob_centroid_is_its_centre():
    z, x = np.mgrid[0:41, 0:31]
    img = np.exp(-((x - 17) ** 2 / 18.0 + (z - 23) ** 2 / 30.0)).astype(np.float32)
    r = metrics.measures(img, x0=-4.5e-3, dx=0.3e-3, z0=5e-3, dz=0.1e-3, alpha=0.7)
    assert math.isclose(r["cx_m"], -4.5e-3 + 17 * 0.3e-3, rel_tol=1e-9)
    assert math.isclose(r["cz_m"], 5e-3 + 23 * 0.1e-3, rel_tol=1e-9)
    # the half-max area of exp(-x^2/a - z^2/b) is pi sqrt(ab) ln 2 pixels (to discretisation)
    assert abs(r["n_inside"] - math.pi * math.sqrt(18 * 30) * math.log(2)) < 4


def test_degenerate_maps():
    r = metrics.measures(np.zeros((4, 5)), 0, 1, 0, 1)
    assert r["n_inside"] == 0 and math.isnan(r["isnr_db"]) and math.isnan(r["cx_m"])
    r = metrics.measures(np.ones((4, 5)), 0, 1, 0, 1)
    assert r["n_inside"] == 20 and r["isnr_db"] == math.inf
    r = metrics.measures(np.array([[0, 0], [0, 2.0]]), 0, 1, 0, 1)   # zeros outside
    assert r["isnr_db"] == math.inf and r["cx_m"] == 1 and r["cz_m"] == 1


def test_isnr_is_scale_invariant_and_as3_closed_forms():
    rng = np.random.default_rng(3)
    img = rng.uniform(0, 1, (17, 9)).astype(np.float32)
    a = metrics.measures(img, 0, 1e-3, 0, 1e-3)
    b = metrics.measures(img * np.float32(8.0), 0, 1e-3, 0, 1e-3)   # power of 2: exact scaling
    assert a["n_inside"] == b["n_inside"] and math.isclose(a["isnr_db"], b["isnr_db"], rel_tol=1e-12)
    e = rng.uniform(0, 1, (5, 6))
    e[2, 3] = 1.0
    assert np.allclose(metrics.as3(e), e ** 3)                        # max = 1: AS^3 = e^3
    assert np.allclose(metrics.as3(3.0 * e), 3.0 * metrics.as3(e))    # degree-1 homogeneous
    assert np.all(metrics.as3(e) <= e + 1e-15)
    assert np.array_equal(metrics.as3(np.zeros((2, 2))), np.zeros((2, 2)))
