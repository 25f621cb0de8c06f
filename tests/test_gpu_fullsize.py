"""Full-size cases of the configured workloads, in the launch configuration
the bench times, against the oracle on sampled outputs: the oracle evaluates
single depth rows (a one-row geometry at that depth), which it can do in a
fraction of a second at 128 elements and 300 bins.

* precision form: FP16 hi + lo split, 64 frames per call (two frame groups),
  128 x 512, 300 bins; frames of different scales;
* learned form: band energies from the BF16 GEMM variant and the tcgen05
  network at 128 x 512; the gate closed gives the plain method.
"""
import numpy as np
import pytest

import oracle
from gpu_common import rel_l2
from paper_2412_02413_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROWS = (0, 255, 511)


def _row_geometry(w, j, bins=None):
    return oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, 1, w.z0 + j * w.dz, 1e-4,
                           w.bins() if bins is None else bins)


@pytest.fixture(scope="module")
def w2_base():
    w = synth.workload(2)
    return w, [synth.make_frame(w, 300 + i)[0] for i in range(4)]


def test_fp16split_64_frames_sampled_rows(w2_base):
    from paper_2412_02413_gb300 import pam
    w, base = w2_base
    scale = lambda f: float(1 + f)                       # frames of different scales (power-of-2 scaling per frame)
    rf = np.stack([base[f % 4] * np.float32(scale(f)) for f in range(64)])
    plan = pam.Plan.from_workload(w, max_frames=64, form="fp16split")
    out = plan.as_tax(torch.from_numpy(rf).cuda(), rho_n=True, image_as=True)
    torch.cuda.synchronize()
    apod = oracle.pattern(w.n_elem, 3, w.pattern_m)
    for f in (0, 31, 32, 63):
        e_gpu = out["image_as"][f].cpu().numpy().astype(np.float64)
        rn = out["rho_n"][f].cpu().numpy().astype(np.float64)
        for j in ROWS:
            orc = oracle.as_xcorr(_row_geometry(w, j), base[f % 4], apod)
            # energies scale with the square of the frame scale; NCC maps do not
            assert rel_l2(e_gpu[j], orc["image_as"][0] * scale(f) ** 2) <= 1e-5, (f, j)
            assert np.max(np.abs(rn[j] / rn[j].max() - orc["rho_n"][0])) <= 1e-5, (f, j)
    plan.close()


def test_learned_full_size(w2_base):
    from paper_2412_02413_gb300 import learn, pam
    w, base = w2_base
    params, _ = learn.load_checkpoint()
    L = pam.Learned.from_workload(w, max_frames=2)
    L.set_params(params)
    L.configure(gate_tol=0.25, tensor_cores=True)
    rf = torch.from_numpy(np.stack(base[:2])).cuda()
    feats, _, en = L.example(rf, target=False, energy=True)
    e = en.cpu().numpy().astype(np.float64)
    for f in range(2):
        for j in ROWS:
            want = oracle.as_backprop(_row_geometry(w, j), base[f])[0]
            assert rel_l2(e[f, j], want) <= 2e-3, (f, j)      # BF16 form: about 6e-4
    rho_tc = L.forward(feats).cpu().numpy()
    L.configure(gate_tol=0.25, tensor_cores=False)
    rho_cc = L.forward(feats).cpu().numpy()
    assert rel_l2(rho_tc, rho_cc) <= 1e-3
    L.configure(gate_tol=-1.0, tensor_cores=True)            # gate closed: the plain method
    out = L.as_tax(rf)
    plan = pam.Plan.from_workload(w, max_frames=2)
    plan.set_split(1)
    ref = plan.as_tax(rf, rho_n=True)
    torch.cuda.synchronize()
    for f in range(2):
        assert rel_l2(out["image"][f].cpu().numpy(), ref["image"][f].cpu().numpy()) <= 1e-6
    L.configure(gate_tol=0.25, tensor_cores=True)            # the bench setting
    out = L.as_tax(rf)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out["image"].cpu().numpy()))
    assert np.all(np.isfinite(out["gate_err"].cpu().numpy()))
    plan.close()
    L.close()
