"""Failure detection without a GPU fault.

* A kernel whose bounded mbarrier wait can never complete (nothing arrives)
  gives up after about one second, reports through the plan's status word,
  and pam_sync returns PAM_ERR_TIMEOUT; the next call on the same plan works.
* Host-side fault injection (PAM_FAULT=alloc): plan creation fails part way
  with PAM_ERR_OOM and leaves no device memory behind.
* PAM_FAULT=launch: a compute call fails with PAM_ERR_CUDA before queueing
  anything, and the same plan then gives the same result bit for bit.
No test here traps, faults or hangs the GPU.
"""
import time

import numpy as np
import pytest

import oracle
from gpu_common import REL_L2_TOL, rel_l2
from paper_2412_02413_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _small():
    w = synth.workload(1)
    w.nz = 24
    return w


def test_expired_wait_reports_timeout_and_the_context_survives():
    from paper_2412_02413_gb300 import pam
    w = _small()
    plan = pam.Plan.from_workload(w)
    rf, _ = synth.make_frame(w, 70)
    rft = torch.from_numpy(rf).cuda()
    plan.as_tax(rft)
    plan.sync()                                   # clean before
    t0 = time.perf_counter()
    plan.debug_expire_wait()
    with pytest.raises(pam.PamError) as exc:
        plan.sync()
    elapsed = time.perf_counter() - t0
    assert exc.value.status == 5                  # PAM_ERR_TIMEOUT
    assert 0.2 < elapsed < 30.0, elapsed          # the wait is bounded (about one second of SM cycles)
    plan.sync()                                   # the status word was cleared
    out = plan.as_tax(rft, rho_n=True)            # the context is still usable
    plan.sync()
    g = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, w.bins())
    orc = oracle.as_tax(g, rf, oracle.pattern(w.n_elem, 3, w.pattern_m))
    assert rel_l2(out["image"][0].cpu().numpy(), orc["image"]) <= REL_L2_TOL
    plan.close()


def test_injected_allocation_failure_leaves_nothing(monkeypatch):
    from paper_2412_02413_gb300 import pam
    w = _small()
    warm = pam.Plan.from_workload(w, max_frames=64)   # loads the library and the context
    warm.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    monkeypatch.setenv("PAM_FAULT", "alloc")
    with pytest.raises(pam.PamError) as exc:
        pam.Plan.from_workload(w, max_frames=64)
    assert exc.value.status == 3                  # PAM_ERR_OOM
    assert "injected" in str(exc.value)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) <= 2 * 1024 * 1024, (free0, free1)
    monkeypatch.delenv("PAM_FAULT")
    plan = pam.Plan.from_workload(w, max_frames=64)   # creation works again
    plan.close()


def test_injected_launch_failure_leaves_the_plan_usable(monkeypatch):
    from paper_2412_02413_gb300 import pam
    w = _small()
    plan = pam.Plan.from_workload(w)
    rft = torch.from_numpy(synth.make_frame(w, 71)[0]).cuda()
    ref = plan.as_tax(rft, rho_n=True)
    ref_e = plan.as_backprop(rft)
    plan.sync()
    monkeypatch.setenv("PAM_FAULT", "launch")
    for call in (lambda: plan.as_tax(rft), lambda: plan.as_backprop(rft)):
        with pytest.raises(pam.PamError) as exc:
            call()
        assert exc.value.status == 4              # PAM_ERR_CUDA
        assert "injected" in str(exc.value)
    monkeypatch.delenv("PAM_FAULT")
    out = plan.as_tax(rft, rho_n=True)
    e = plan.as_backprop(rft)
    plan.sync()
    assert torch.equal(out["image"], ref["image"]) and torch.equal(out["rho_n"], ref["rho_n"])
    assert torch.equal(e, ref_e)
    plan.close()
