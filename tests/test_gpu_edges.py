"""Size extremes and degenerate inputs against the oracle:
* a deep grid (2048 rows) at 128 elements, checked on sampled rows;
* many bins (every bin of 0.5-10 MHz at nt = 8192, about 1,900 of them);
* an all-zero frame through the learned form (no NaN; the gate passes and
  the image is zero, as the plain method gives)."""
import numpy as np
import pytest

import oracle
from gpu_common import NCC_TOL, REL_L2_TOL, compare_xcorr, rel_l2
from paper_2412_02413_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pam():
    from paper_2412_02413_gb300 import pam
    return pam


def test_deep_grid_sampled_rows():
    w = synth.Workload(name="deep", n_elem=128, pitch=0.3e-3, fs=40e6, nt=1024, c=1540.0, nz=2048,
                       z_first=5e-3, z_last=5e-3 + 2047 * 0.05e-3, f_lo=0.5e6, f_hi=8e6, n_bins=None, pattern_m=16,
                       source_z=(10e-3, 100e-3))
    rf = synth.make_frame(w, 1)[0]
    plan = _pam().Plan.from_workload(w)
    out = plan.as_tax(torch.from_numpy(rf).cuda(), rho_n=True, image_as=True)
    ia = out["image_as"][0].cpu().numpy().astype(np.float64)
    rn = out["rho_n"][0].cpu().numpy().astype(np.float64)
    apod = oracle.pattern(128, 3, 16)
    for j in (0, 1000, 2047):
        g = oracle.Geometry(128, w.nt, w.fs, w.c, w.pitch, 1, w.z0 + j * w.dz, 1e-4, w.bins())
        orc = oracle.as_xcorr(g, rf, apod)
        assert rel_l2(ia[j], orc["image_as"][0]) <= REL_L2_TOL, j
        assert np.max(np.abs(rn[j] / rn[j].max() - orc["rho_n"][0])) <= NCC_TOL, j
    plan.close()


def test_many_bins():
    w = synth.Workload(name="wide", n_elem=32, pitch=0.3e-3, fs=40e6, nt=8192, c=1540.0, nz=6, z_first=8e-3,
                       z_last=8e-3 + 5 * 2e-3, f_lo=0.5e6, f_hi=10e6, n_bins=None, pattern_m=2)
    assert len(w.bins()) > 1800
    rf = synth.random_rf(32, 8192, seed=41)
    pam = _pam()
    plan = pam.Plan.from_workload(w)
    out = plan.as_tax(torch.from_numpy(rf).cuda(), rho_n=True, rho_pairs=True, image_as=True)
    g = oracle.Geometry(32, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, w.bins())
    orc = oracle.as_tax(g, rf, oracle.pattern(32, 3, 2))
    compare_xcorr(out, orc, check_peak=False)
    plan.close()


def test_learned_zero_frame():
    from paper_2412_02413_gb300 import learn
    w = synth.workload(1)
    w.nz = 24
    pam = _pam()
    L = pam.Learned.from_workload(w, max_frames=2)
    L.set_params(learn.init_params(5))
    L.configure(gate_tol=0.25)
    rf = torch.zeros((2, w.n_elem, w.nt), dtype=torch.float32, device="cuda")
    rf[1] = torch.from_numpy(synth.make_frame(w, 90)[0]).cuda()
    out = L.as_tax(rf)
    torch.cuda.synchronize()
    img = out["image"].cpu().numpy()
    assert np.all(np.isfinite(img)) and np.all(np.isfinite(out["rho_n"].cpu().numpy()))
    assert np.all(img[0] == 0.0)
    assert int(out["gate_pass"][0].item()) == 1 and float(out["gate_err"][0].item()) == 0.0
    L.close()
