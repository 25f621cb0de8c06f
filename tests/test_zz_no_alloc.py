"""pam_as_tax_static: AS-TAX for callers that cannot allocate GPU memory.

Such callers cannot create a plan, which calls cudaMalloc. Examples are code
inside a framework that owns every device allocation and real-time loops
with a fixed memory footprint. The entry point keeps its tables and
workspace in a fixed device array inside the library. These tests call it
through the C ABI and compare it with pam_as_tax on a plan, with the
tolerances of the other parity tests. It runs two calls in a row, because
the second call must not be affected by what the first left in the shared
array. This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import NCC_TOL, REL_L2_TOL, rel_l2
from paper_2412_02413_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _desc(pam, w, bins):
    L = pam.load()
    d = pam.PlanDesc()
    L.pam_plan_desc_init(ctypes.byref(d))
    d.n_elem, d.pitch_m, d.fs_hz, d.c_mps = w.n_elem, w.pitch, w.fs, w.c
    d.n_samples, d.nz, d.z0_m, d.dz_m = w.nt, w.nz, w.z0, w.dz
    d.bins = bins.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d.n_bins = int(bins.size)
    d.n_apod, d.pattern_m = 3, w.pattern_m
    return d


@pytest.mark.parametrize("wid", [2, 1])
def test_static_entry_matches_plan_entry(wid):
    from paper_2412_02413_gb300 import pam
    L = pam.load()
    w = synth.workload(wid)
    bins = np.ascontiguousarray(w.bins(), dtype=np.int32)
    d = _desc(pam, w, bins)
    plan = pam.Plan.from_workload(w)
    stream = torch.cuda.current_stream()
    for frame in (0, 1):   # two calls in a row
        rf = torch.from_numpy(synth.make_frame(w, frame)[0]).cuda()
        img = torch.full((1, w.nz, w.nx), float("nan"), device="cuda")
        rho = torch.full((1, w.nz, w.nx), float("nan"), device="cuda")
        st = L.pam_as_tax_static(ctypes.byref(d), rf.data_ptr(), 1, img.data_ptr(), rho.data_ptr(),
                                 stream.cuda_stream)
        assert st == 0, L.pam_last_error()
        ref = plan.as_tax(rf)
        torch.cuda.synchronize()
        a, b = img[0].cpu().numpy(), ref["image"][0].cpu().numpy()
        assert rel_l2(a, b) <= REL_L2_TOL
        assert float(torch.max(torch.abs(rho - ref["rho_n"]))) <= NCC_TOL
        assert np.argmax(a) == np.argmax(b)
    plan.close()


def test_static_entry_rejects_oversize_geometry():
    from paper_2412_02413_gb300 import pam
    L = pam.load()
    w = synth.workload(2)
    w.nz = 32768                     # 32768 x 128 pixels need far more than the fixed array
    bins = np.ascontiguousarray(w.bins(), dtype=np.int32)
    d = _desc(pam, w, bins)
    rf = torch.zeros(1, w.n_elem, w.nt, device="cuda")
    img = torch.zeros(1, w.nz, w.nx, device="cuda")
    st = L.pam_as_tax_static(ctypes.byref(d), rf.data_ptr(), 1, img.data_ptr(), None, None)
    assert st == 1
    assert b"static scratch" in L.pam_last_error()
