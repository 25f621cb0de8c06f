"""AS^3 (pam_as3) and the image measures (pam_image_metrics) on the GPU
against oracle/metrics.py and the method oracle."""
import math

import numpy as np
import pytest

import oracle
from gpu_common import REL_L2_TOL, rel_l2
from oracle import metrics
from paper_2412_02413_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pam():
    from paper_2412_02413_gb300 import pam
    return pam


def _grid(w):
    return -(w.n_elem - 1) / 2 * w.pitch, w.pitch, w.z0, w.dz


def test_as3_matches_oracle():
    w = synth.workload(1)
    w.nz = 40
    pam = _pam()
    plan = pam.Plan.from_workload(w, max_frames=2)
    rf = np.stack([synth.make_frame(w, 11)[0], synth.make_frame(w, 12)[0]])
    img = plan.as3(torch.from_numpy(rf).cuda()).cpu().numpy()
    g = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, w.bins())
    for f in range(2):
        want = metrics.as3(oracle.as_backprop(g, rf[f]))
        assert rel_l2(img[f], want) <= REL_L2_TOL
        assert np.argmax(img[f]) == np.argmax(want)
    plan.close()


@pytest.mark.parametrize("alpha", [0.7, 0.9])
def test_measures_match_oracle(alpha):
    w = synth.workload(1)
    w.nz = 40
    pam = _pam()
    plan = pam.Plan.from_workload(w, max_frames=3)
    rf = torch.from_numpy(np.stack([synth.make_frame(w, 20 + i)[0] for i in range(3)])).cuda()
    out = plan.as_tax(rf, rho_n=True, image_as=True)
    maps = torch.cat([out["image"], out["image_as"], out["rho_n"],
                      torch.zeros(1, w.nz, w.nx, device="cuda"),          # all zero: NaN ISNR, NaN centroid
                      torch.ones(1, w.nz, w.nx, device="cuda")])          # nothing outside A_0.5: +inf ISNR
    x0, dx, z0, dz = _grid(w)
    got = pam.image_metrics(maps, x0, dx, z0, dz, alpha)
    host = maps.cpu().numpy()
    for k in range(host.shape[0]):
        want = metrics.measures(host[k], x0, dx, z0, dz, alpha)
        g = got[k]
        assert g["n_inside"] == want["n_inside"], k
        assert g["max"] == want["max"]
        assert math.isclose(g["esa_m2"], want["esa_m2"], rel_tol=1e-6)
        for key in ("isnr_db", "cx_m", "cz_m"):
            if math.isnan(want[key]) or math.isinf(want[key]):
                assert (math.isnan(g[key]) and math.isnan(want[key])) or g[key] == want[key], (k, key)
            else:
                assert math.isclose(g[key], want[key], rel_tol=1e-6, abs_tol=1e-9), (k, key, g[key], want[key])
    # AS-TAX suppresses artefacts: higher ISNR and smaller A_0.5 than AS on these frames
    for f in range(3):
        assert got[f]["isnr_db"] > got[3 + f]["isnr_db"]
        assert got[f]["esa_m2"] <= got[3 + f]["esa_m2"]
    plan.close()


def _probe_rate(packed):
    import ctypes
    import os

    from paper_2412_02413_gb300 import build
    lib = ctypes.CDLL(build.PROBE_LIB)
    lib.pam_probe_fp32_fma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.pam_probe_fp32_fma_rate.restype = ctypes.c_int
    v = ctypes.c_double(0.0)
    assert os.path.exists(build.PROBE_LIB)
    assert lib.pam_probe_fp32_fma_rate(1024, int(packed), ctypes.byref(v)) == 0
    return v.value


def test_fp32_fma_rate_is_plausible():
    """The benchmark's FMA probe (its own library, not libpam): the scalar and
    the packed two-wide rates lie between a quarter of the unit-count peak at
    1 GHz and twice that peak at 2.2 GHz (128 FP32 lanes per SM, 2 flops per
    FMA)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for packed in (0, 1):
        rate = _probe_rate(packed)
        assert 0.25 * sms * 128 * 2 * 1.0e9 / 1e12 < rate < 2 * sms * 128 * 2 * 2.2e9 / 1e12, (packed, rate)
