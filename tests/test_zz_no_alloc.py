"""pam_as_tax_static: AS-TAX for callers that cannot allocate GPU memory.

Such callers cannot create a plan, which calls cudaMalloc. Examples are code
inside a framework that owns every device allocation and real-time loops
with a fixed memory footprint. The entry point keeps its tables and
workspace in a fixed device array inside the library. These tests call it
through the C ABI and compare it with pam_as_tax on a plan, with the
tolerances of the other parity tests. They run calls in a row, because a
call must not be affected by what the previous one left in the shared array,
and check that a call leaves the device's free memory unchanged. This file is
collected last.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import NCC_TOL, REL_L2_TOL, rel_l2
from paper_2412_02413_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAM_ERR_INVALID_ARG, PAM_ERR_UNSUPPORTED = 1, 2


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


def _static(L, d, rf, img, rho, stream):
    return L.pam_as_tax_static(ctypes.byref(d), rf.data_ptr(), rf.shape[0], img.data_ptr(),
                               None if rho is None else rho.data_ptr(), stream.cuda_stream)


def _check_frames(img, rho, ref):
    for f in range(img.shape[0]):
        a, b = img[f].cpu().numpy(), ref["image"][f].cpu().numpy()
        assert rel_l2(a, b) <= REL_L2_TOL, f
        assert float(torch.max(torch.abs(rho[f] - ref["rho_n"][f]))) <= NCC_TOL, f
        assert np.argmax(a) == np.argmax(b), f


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
        rf = torch.from_numpy(synth.make_frame(w, frame)[0]).cuda()[None]
        img = torch.full((1, w.nz, w.nx), float("nan"), device="cuda")
        rho = torch.full((1, w.nz, w.nx), float("nan"), device="cuda")
        assert _static(L, d, rf, img, rho, stream) == 0, L.pam_last_error()
        ref = plan.as_tax(rf)
        torch.cuda.synchronize()
        _check_frames(img, rho, ref)
    plan.close()


def test_static_entry_allocates_nothing():
    """After a first call on the device (its one-time set-up) a call leaves
    the device's free memory exactly where it was."""
    from paper_2412_02413_gb300 import pam
    L = pam.load()
    w = synth.workload(2)
    bins = np.ascontiguousarray(w.bins(), dtype=np.int32)
    d = _desc(pam, w, bins)
    stream = torch.cuda.current_stream()
    rf = torch.from_numpy(synth.make_frame(w, 3)[0]).cuda()[None]
    img = torch.empty((1, w.nz, w.nx), device="cuda")
    rho = torch.empty((1, w.nz, w.nx), device="cuda")
    assert _static(L, d, rf, img, rho, stream) == 0, L.pam_last_error()
    torch.cuda.synchronize()
    first = img.clone()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert _static(L, d, rf, img, rho, stream) == 0, L.pam_last_error()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
    assert torch.equal(img, first)   # same input, same bits


def test_static_entry_several_frames():
    """n_frames = 3 distinct frames in one call: the per-frame offsets of the
    input and outputs, and the reuse of the tables and workspace across frames."""
    from paper_2412_02413_gb300 import pam
    L = pam.load()
    w = synth.workload(1)
    bins = np.ascontiguousarray(w.bins(), dtype=np.int32)
    d = _desc(pam, w, bins)
    stream = torch.cuda.current_stream()
    rf = torch.from_numpy(np.stack([synth.make_frame(w, f)[0] for f in (4, 5, 6)])).cuda()
    img = torch.full((3, w.nz, w.nx), float("nan"), device="cuda")
    rho = torch.full((3, w.nz, w.nx), float("nan"), device="cuda")
    assert _static(L, d, rf, img, rho, stream) == 0, L.pam_last_error()
    plan = pam.Plan.from_workload(w, max_frames=3)
    ref = plan.as_tax(rf)
    torch.cuda.synchronize()
    _check_frames(img, rho, ref)
    assert not torch.equal(img[0], img[1])
    plan.close()


def test_static_entry_caps_split_at_cluster_size():
    """32 rows at 128 elements: the automatic bin split of a plan is far above
    the cluster size of 8 (it sums partials in global memory), while the static
    entry point caps it at 8 and reduces on chip. The images agree."""
    from paper_2412_02413_gb300 import pam
    L = pam.load()
    w = synth.workload(2)
    w.nz = 32
    bins = np.ascontiguousarray(w.bins(), dtype=np.int32)
    d = _desc(pam, w, bins)
    stream = torch.cuda.current_stream()
    rf = torch.from_numpy(synth.make_frame(w, 7)[0]).cuda()[None]
    img = torch.full((1, w.nz, w.nx), float("nan"), device="cuda")
    rho = torch.full((1, w.nz, w.nx), float("nan"), device="cuda")
    assert _static(L, d, rf, img, rho, stream) == 0, L.pam_last_error()
    plan = pam.Plan.from_workload(w)
    ref = plan.as_tax(rf)
    torch.cuda.synchronize()
    _check_frames(img, rho, ref)
    plan.close()


def test_static_entry_reports_expired_wait_as_nan(monkeypatch):
    """A bounded wait that gives up (injected from the host: a wait nothing
    completes, about one second) turns every output element into NaN; the next
    call, without the injection, is exact again."""
    from paper_2412_02413_gb300 import pam
    L = pam.load()
    w = synth.workload(1)
    w.nz = 16
    bins = np.ascontiguousarray(w.bins(), dtype=np.int32)
    d = _desc(pam, w, bins)
    stream = torch.cuda.current_stream()
    rf = torch.from_numpy(synth.make_frame(w, 8)[0]).cuda()[None]
    img = torch.zeros((1, w.nz, w.nx), device="cuda")
    rho = torch.zeros((1, w.nz, w.nx), device="cuda")
    monkeypatch.setenv("PAM_FAULT", "static_wait")
    assert _static(L, d, rf, img, rho, stream) == 0, L.pam_last_error()
    torch.cuda.synchronize()
    monkeypatch.delenv("PAM_FAULT")
    assert bool(torch.isnan(img).all()) and bool(torch.isnan(rho).all())
    assert _static(L, d, rf, img, rho, stream) == 0, L.pam_last_error()
    plan = pam.Plan.from_workload(w)
    ref = plan.as_tax(rf)
    torch.cuda.synchronize()
    _check_frames(img, rho, ref)
    plan.close()


def test_static_entry_refuses_capturing_stream():
    """The per-call uploads come from pageable memory, which stream capture
    does not allow: on a capturing stream the call is refused before anything
    is queued, and the capture itself stays usable."""
    from paper_2412_02413_gb300 import pam
    L = pam.load()
    w = synth.workload(1)
    w.nz = 16
    bins = np.ascontiguousarray(w.bins(), dtype=np.int32)
    d = _desc(pam, w, bins)
    rf = torch.zeros((1, w.n_elem, w.nt), device="cuda")
    img = torch.zeros((1, w.nz, w.nx), device="cuda")
    x = torch.zeros(4, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            x.add_(1.0)
            codes.append(_static(L, d, rf, img, None, s))
    assert codes == [PAM_ERR_UNSUPPORTED], codes
    assert b"capturing" in L.pam_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, torch.ones(4, device="cuda"))


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
    assert st == PAM_ERR_INVALID_ARG
    assert b"static scratch" in L.pam_last_error()
