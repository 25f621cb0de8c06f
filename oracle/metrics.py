"""FP64 reference of the paper's image measures and of the AS^3 image
(test infrastructure: only tests/ and the bench's baseline leg import it).

* A_0.5, the energy spread area (Sec. II-D): the pixels whose value exceeds
  half of the image maximum, times the pixel area.
* ISNR (Eq. 12): 10 log10 of the mean pixel value inside A_0.5 over the mean
  outside it.
* Centroid (Eq. 13): sum_i I_i r_i / sum_i I_i over the pixels with
  I_i > alpha max I (alpha = 0.7 for images, 0.9 for NCC maps).
* AS^3 (Eq. 20): (I_AS / max I_AS)^2 I_AS.

The threshold decisions are taken in float32, the precision of the maps,
so that pixel membership is decided the same way the GPU decides it.
Parity pins: tests/test_metrics_oracle.py (hand-computed maps, a symmetric
blob, scaling laws).
"""
from __future__ import annotations

import math

import numpy as np


def measures(img, x0: float, dx: float, z0: float, dz: float, alpha: float = 0.7) -> dict:
    """img [nz][nx]; pixel (j, i) at x = x0 + i dx, z = z0 + j dz."""
    f = np.asarray(img, dtype=np.float32)
    m = f.max()
    inside = f > np.float32(0.5) * m
    n_in = int(inside.sum())
    n_out = f.size - n_in
    v = f.astype(np.float64)
    s_in, s_out = float(v[inside].sum()), float(v[~inside].sum())
    if not m > 0 or n_in == 0:
        isnr = math.nan
    elif n_out == 0 or s_out <= 0:
        isnr = math.inf
    else:
        isnr = 10.0 * math.log10((s_in / n_in) / (s_out / n_out))
    sel = f > np.float32(alpha) * m
    w = v[sel]
    jj, ii = np.nonzero(sel)
    if w.sum() > 0:
        cx = float(np.sum(w * (x0 + ii * dx)) / w.sum())
        cz = float(np.sum(w * (z0 + jj * dz)) / w.sum())
    else:
        cx = cz = math.nan
    return {"esa_m2": n_in * abs(dx * dz), "isnr_db": isnr, "cx_m": cx, "cz_m": cz, "max": float(m),
            "n_inside": n_in}


def as3(energy):
    """Eq. 20 from the AS energy map [nz][nx]."""
    e = np.asarray(energy, dtype=np.float64)
    m = e.max()
    return (e / m) ** 2 * e if m > 0 else np.zeros_like(e)
