"""Learned form (pam_learn_*) on the GPU against the FP64 oracle of the
network (oracle/cnn_oracle.py) and of the method (oracle/pam_oracle.c).

The network's operands are BF16 with FP32 sums, so two references are used:
* the plain FP64 oracle, given the BF16-rounded inputs and weights the GPU
  uses; the tolerance comes from BF16 rounding of the activations and
  gradients between layers (unit roundoff 2^-9 per rounding, a few per layer);
* the same oracle steps with the GPU's rounding points restated (activations,
  dL/dz and each layer's input gradient rounded to BF16): this pins the
  kernels' index and transpose logic far below the BF16 noise.
"""
import numpy as np
import pytest

import oracle
from gpu_common import NCC_TOL, REL_L2_TOL, rel_l2
from oracle import cnn_oracle as co
from paper_2412_02413_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 1e-3


def _pam():
    from paper_2412_02413_gb300 import pam
    return pam


def bf16(x):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    r = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def flat(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def unflat(v, channels=co.CHANNELS):
    out, o = [], 0
    for cin, cout in zip(channels[:-1], channels[1:]):
        n = cout * cin * 9
        w = v[o:o + n].reshape(cout, cin, 3, 3)
        b = v[o + n:o + n + cout]
        out.append((np.asarray(w, np.float64), np.asarray(b, np.float64)))
        o += n + cout
    return out


def rand_params(seed):
    p = co.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    return [(w, rng.uniform(-0.1, 0.1, b.shape)) for w, b in p]


def gpu_weights(params):
    """The parameters as the GPU sees them: BF16 weights, FP32 biases."""
    return [(bf16(w), np.asarray(b, np.float32).astype(np.float64)) for w, b in params]


def forward_rounded(params, x):
    """Oracle forward with the GPU's rounding points (activations to BF16)."""
    h = x
    for li, (w, b) in enumerate(params):
        z = co.conv3x3(h, w, b)
        if li < len(params) - 1:
            h = bf16(np.maximum(z, 0.0))
        else:
            return EPS + (1.0 - EPS) * co.sigmoid(z)


def grads_rounded(params, x, target):
    """Oracle gradients with the GPU's rounding points: activations, dL/dz and
    every masked input gradient in BF16; sums in FP64."""
    acts, h = [x], x
    for li, (w, b) in enumerate(params):
        z = co.conv3x3(h, w, b)
        if li < len(params) - 1:
            h = bf16(np.maximum(z, 0.0))
            acts.append(h)
    s = co.sigmoid(z)
    diff = EPS + (1.0 - EPS) * s - target[:, None]
    n = diff.size
    wgt = co.loss_weights(x)
    loss = float(np.sum(wgt * diff ** 2) / n)
    dy = bf16(2.0 * wgt * diff / n * (1.0 - EPS) * s * (1.0 - s))
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        w, _ = params[li]
        dx, dw, db = co.conv3x3_backward(acts[li], w, dy)
        grads[li] = (dw, db)
        if li > 0:
            dy = bf16(dx * (acts[li] > 0.0))
    return loss, grads


def _learned(ne, nt, nz, max_frames=2, n_bins=None, fs=20e6):
    pam = _pam()
    w = synth.Workload(name="t", n_elem=ne, pitch=0.3e-3, fs=fs, nt=nt, c=1540.0, nz=nz, z_first=4e-3,
                       z_last=4e-3 + (nz - 1) * 0.45e-3, f_lo=1e6, f_hi=8e6, n_bins=n_bins, pattern_m=2)
    return pam.Learned.from_workload(w, max_frames=max_frames), w


def _features(n, nz, nx, seed):
    rng = np.random.default_rng(seed)
    x = bf16(rng.uniform(-1.0, 0.0, (n, 5, nz, nx)))
    return x, torch.from_numpy(_pam().pack_features(x)).cuda()


# ------------------------------------------------------------------ forward --
@pytest.mark.parametrize("ne,nz", [(16, 21), (32, 9)])
def test_forward_matches_oracle(ne, nz):
    L, _ = _learned(ne, 128, nz)
    params = rand_params(1)
    L.set_params(flat(params))
    x, feats = _features(2, nz, ne, 2)
    rho = L.forward(feats).cpu().numpy().astype(np.float64)
    gw = gpu_weights(params)
    plain, _ = co.forward(gw, x, EPS)
    rounded = forward_rounded(gw, x)
    e_plain = rel_l2(rho, plain[:, 0])
    e_round = rel_l2(rho, rounded[:, 0])
    e_bf = rel_l2(rounded[:, 0], plain[:, 0])
    print(f"forward ne={ne} nz={nz}: rel L2 vs FP64 oracle {e_plain:.2e} (BF16 rounding alone {e_bf:.2e}), "
          f"vs BF16-rounding oracle {e_round:.2e}")
    assert e_plain <= 1.5 * e_bf + 1e-4
    assert e_round <= 1e-4
    assert np.all(rho >= EPS) and np.all(rho < 1.0)
    L.close()


# ---------------------------------------------------------------- gradients --
def test_gradients_match_oracle():
    nz, ne = 21, 16
    L, _ = _learned(ne, 128, nz)
    params = rand_params(3)
    L.set_params(flat(params))
    x, feats = _features(2, nz, ne, 4)
    target = np.random.default_rng(5).uniform(EPS, 1.0, (2, nz, ne))
    g, loss = L.grads(feats, torch.from_numpy(target.astype(np.float32)).cuda())
    g = unflat(g.cpu().numpy().astype(np.float64))
    gw = gpu_weights(params)
    # target as the GPU sees it (FP32)
    t32 = target.astype(np.float32).astype(np.float64)
    loss_o, grads_o = co.loss_and_grads(gw, x, t32, EPS)
    loss_r, grads_r = grads_rounded(gw, x, t32)
    assert abs(float(loss.item()) - loss_o) <= 1e-2 * loss_o
    assert abs(float(loss.item()) - loss_r) <= 1e-5 * loss_r
    for li in range(5):
        for k, name in ((0, "w"), (1, "b")):
            ep = rel_l2(g[li][k], grads_o[li][k])
            er = rel_l2(g[li][k], grads_r[li][k])
            # what the BF16 rounding points alone do to this gradient (the
            # deep layers' weight gradients sum products whose terms cancel,
            # so their relative error is a multiple of 2^-9)
            e_bf = rel_l2(grads_r[li][k], grads_o[li][k])
            print(f"layer {li + 1} d{name}: rel L2 vs FP64 oracle {ep:.2e} (BF16 rounding alone {e_bf:.2e}), "
                  f"vs BF16-rounding oracle {er:.2e}")
            assert ep <= 1.5 * e_bf + 1e-3, (li, name, ep, e_bf)
            assert er <= 2e-3, (li, name, er)
    L.close()


def test_adam_first_step_is_lr_times_sign():
    nz, ne = 9, 16
    L, _ = _learned(ne, 128, nz)
    params = rand_params(6)
    p0 = flat(params).astype(np.float32)
    L.set_params(p0)
    x, feats = _features(2, nz, ne, 7)
    target = np.random.default_rng(8).uniform(EPS, 1.0, (2, nz, ne)).astype(np.float32)
    lr = 1e-3
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    L.train_step(feats, torch.from_numpy(target).cuda(), lr, loss=loss)
    torch.cuda.synchronize()
    p1 = L.get_params().astype(np.float64)
    _, grads_o = co.loss_and_grads(gpu_weights(params), x, target.astype(np.float64), EPS)
    g = flat(grads_o)
    p1_o = co.adam_step(p0.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr=lr)[0]
    big = np.abs(g) > 0.05 * np.abs(g).max()
    assert big.sum() > 100
    # Adam's first step is lr * sign(g) wherever |g| >> eps
    assert np.allclose(p1[big], p1_o[big], atol=1e-6 * lr + 1e-7)
    assert L.info()["adam_steps"] == 1
    L.close()


# ------------------------------------------------- features and the target --
def test_example_features_and_target_match_oracle():
    w = synth.workload(1)
    w.nz = 40
    rf, _ = synth.make_frame(w, 3)
    pam = _pam()
    L = pam.Learned.from_workload(w, max_frames=2)
    rf2 = np.stack([rf, synth.make_frame(w, 4)[0]])
    feats, tgt, en = L.example(torch.from_numpy(rf2).cuda(), energy=True)
    got = pam.unpack_features(feats, w.nz, w.n_elem)
    bins = w.bins()
    nb = len(bins)
    for f in range(2):
        g = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, bins)
        e_full = oracle.as_backprop(g, rf2[f])
        e_bands = []
        for b in range(4):
            sub = bins[nb * b // 4: nb * (b + 1) // 4]
            gb = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, sub)
            e_bands.append(oracle.as_backprop(gb, rf2[f]))
        want = co.features(np.stack(e_bands))
        # BF16 rounding of values in [-1, 0]: at most half an ulp, 2^-9
        assert np.max(np.abs(got[f] - want)) <= 2.5e-3
        assert rel_l2(en[f].cpu().numpy(), e_full) <= REL_L2_TOL
        orc = oracle.as_tax(g, rf2[f], oracle.pattern(w.n_elem, 3, w.pattern_m))
        rho_tax = np.cbrt(np.prod(orc["rho_pairs"], axis=0))
        assert np.max(np.abs(tgt[f].cpu().numpy() - rho_tax)) <= NCC_TOL
    L.close()


def test_tensor_core_band_energies_match_oracle():
    """With tensor cores on, the band energies come from the BF16 GEMM form:
    relative error about 6e-4, below the BF16 rounding of the features."""
    w = synth.workload(2)
    w.nz = 40
    rf, _ = synth.make_frame(w, 5)
    pam = _pam()
    L = pam.Learned.from_workload(w, max_frames=1)
    L.configure(tensor_cores=True)
    feats, _, en = L.example(torch.from_numpy(rf[None]).cuda(), target=False, energy=True)
    got = pam.unpack_features(feats, w.nz, w.n_elem)[0]
    bins = w.bins()
    nb = len(bins)
    g = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, bins)
    e_full = oracle.as_backprop(g, rf)
    e_bands = []
    for b in range(4):
        gb = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, bins[nb * b // 4: nb * (b + 1) // 4])
        e_bands.append(oracle.as_backprop(gb, rf))
    err = rel_l2(en[0].cpu().numpy(), e_full)
    print(f"tensor-core band energies: rel L2 of E {err:.2e}")
    assert err <= 2e-3
    want = co.features(np.stack(e_bands))
    # half a BF16 ulp plus the form's error through log10 (|d log10(x)| <= 2e-3 / ln 10 relative)
    assert np.max(np.abs(got - want)) <= 5e-3
    L.close()


# --------------------------------------------------------------- the gate --
def test_gate_closed_gives_the_plain_method():
    w = synth.workload(1)
    w.nz = 40
    pam = _pam()
    L = pam.Learned.from_workload(w, max_frames=2)
    L.set_params(flat(rand_params(9)))
    L.configure(gate_tol=-1.0)
    rf2 = np.stack([synth.make_frame(w, 5)[0], synth.make_frame(w, 6)[0]])
    out = L.as_tax(torch.from_numpy(rf2).cuda())
    plan = pam.Plan.from_workload(w, max_frames=2)
    plan.set_split(1)
    ref = plan.as_tax(torch.from_numpy(rf2).cuda(), rho_n=True)
    torch.cuda.synchronize()
    assert out["gate_pass"].cpu().numpy().tolist() == [0, 0]
    for f in range(2):
        assert rel_l2(out["image"][f].cpu().numpy(), ref["image"][f].cpu().numpy()) <= 1e-6
        assert np.max(np.abs(out["rho_n"][f].cpu().numpy() - ref["rho_n"][f].cpu().numpy())) <= 1e-6
        g = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, w.bins())
        orc = oracle.as_tax(g, rf2[f], oracle.pattern(w.n_elem, 3, w.pattern_m))
        assert rel_l2(out["image"][f].cpu().numpy(), orc["image"]) <= REL_L2_TOL
    plan.close()
    L.close()


def test_learned_call_larger_than_the_batch():
    """A call of 5 frames on a learned form built for 2 runs in batches of 2;
    with the gate closed every frame equals the plain method."""
    w = synth.workload(1)
    w.nz = 24
    pam = _pam()
    L = pam.Learned.from_workload(w, max_frames=2)
    L.set_params(flat(rand_params(14)))
    L.configure(gate_tol=-1.0)
    rf = torch.from_numpy(np.stack([synth.make_frame(w, 40 + i)[0] for i in range(5)])).cuda()
    out = L.as_tax(rf)
    plan = pam.Plan.from_workload(w, max_frames=5)
    plan.set_split(1)
    ref = plan.as_tax(rf, rho_n=True)
    torch.cuda.synchronize()
    assert out["gate_pass"].cpu().numpy().tolist() == [0] * 5
    for f in range(5):
        assert rel_l2(out["image"][f].cpu().numpy(), ref["image"][f].cpu().numpy()) <= 1e-6
    plan.close()
    L.close()


def test_gate_catches_an_untrained_network():
    """At the bench's gate tolerance (0.25) an untrained network's maps miss the
    gate, and those frames come out as the plain method."""
    w = synth.workload(1)
    w.nz = 40
    pam = _pam()
    L = pam.Learned.from_workload(w, max_frames=4)
    L.set_params(flat(co.init_params(21)))
    L.configure(gate_tol=0.25)
    rf = torch.from_numpy(np.stack([synth.make_frame(w, 60 + i)[0] for i in range(4)])).cuda()
    out = L.as_tax(rf)
    plan = pam.Plan.from_workload(w, max_frames=4)
    plan.set_split(1)
    ref = plan.as_tax(rf, rho_n=True)
    torch.cuda.synchronize()
    passed = out["gate_pass"].cpu().numpy()
    errs = out["gate_err"].cpu().numpy()
    print(f"untrained network: gate errors {np.round(errs, 3).tolist()}")
    assert passed.sum() == 0 and np.all(errs > 0.25)
    for f in range(4):
        assert rel_l2(out["image"][f].cpu().numpy(), ref["image"][f].cpu().numpy()) <= 1e-6
    plan.close()
    L.close()


def test_gate_open_gives_the_network_image():
    w = synth.workload(1)
    w.nz = 40
    pam = _pam()
    L = pam.Learned.from_workload(w, max_frames=2)
    L.set_params(flat(rand_params(10)))
    L.configure(gate_tol=float("inf"))
    rf2 = torch.from_numpy(np.stack([synth.make_frame(w, 7)[0], synth.make_frame(w, 8)[0]])).cuda()
    out = L.as_tax(rf2)
    feats, _, en = L.example(rf2, target=False, energy=True)
    rho = L.forward(feats)
    torch.cuda.synchronize()
    assert out["gate_pass"].cpu().numpy().tolist() == [1, 1]
    assert np.all(np.isfinite(out["gate_err"].cpu().numpy()))
    for f in range(2):
        r = rho[f].cpu().numpy().astype(np.float64)
        want = (r / r.max()) ** 2 * en[f].cpu().numpy()
        assert rel_l2(out["image"][f].cpu().numpy(), want) <= 1e-6
    L.close()


def test_gate_error_is_the_tile_distance():
    """gate_err equals the relative L2 distance, on the predicted peak's row
    tile, between rho_pred^2 E and the exact rho^2 E (computed here from the
    oracle)."""
    w = synth.workload(1)
    w.nz = 40
    pam = _pam()
    L = pam.Learned.from_workload(w, max_frames=1)
    L.set_params(flat(rand_params(11)))
    L.configure(gate_tol=float("inf"))
    rf = synth.make_frame(w, 9)[0]
    rft = torch.from_numpy(rf[None]).cuda()
    out = L.as_tax(rft)
    feats, _, en = L.example(rft, target=False, energy=True)
    rho = L.forward(feats)[0].cpu().numpy().astype(np.float64)
    e = en[0].cpu().numpy().astype(np.float64)
    g = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, w.bins())
    orc = oracle.as_tax(g, rf, oracle.pattern(w.n_elem, 3, w.pattern_m))
    rho_x = np.cbrt(np.prod(orc["rho_pairs"], axis=0))
    rows = 4096 // w.n_elem                         # row tile of the persistent kernel: 16 warps x 256 / nx rows
    i_pred = rho ** 2 * e
    r0 = (int(np.argmax(i_pred)) // w.n_elem) // rows * rows
    sl = slice(r0, min(w.nz, r0 + rows))
    ip, ix = i_pred[sl], rho_x[sl] ** 2 * orc["image_as"][sl]
    want = np.linalg.norm(ip - ix) / np.linalg.norm(ix)
    got = float(out["gate_err"][0].item())
    assert abs(got - want) <= 1e-4 * max(want, 1e-3)
    L.close()


# ------------------------------------------------------------ tensor cores --
def test_tensor_core_forward_matches():
    nz, ne = 40, 128                                 # 16-row strips: two full, one ragged
    L, _ = _learned(ne, 256, nz, n_bins=10)
    params = rand_params(12)
    L.set_params(flat(params))
    x, feats = _features(2, nz, ne, 13)
    rho_cc = L.forward(feats).cpu().numpy().astype(np.float64)
    L.configure(tensor_cores=True)
    rho_tc = L.forward(feats).cpu().numpy().astype(np.float64)
    L.sync()
    rounded = forward_rounded(gpu_weights(params), x)[:, 0]
    e_cc, e_tc, e_x = rel_l2(rho_tc, rounded), rel_l2(rho_cc, rounded), rel_l2(rho_tc, rho_cc)
    print(f"tensor-core forward: rel L2 vs oracle {e_tc:.2e} (CUDA cores {e_cc:.2e}), tc vs cc {e_x:.2e}")
    assert e_tc <= 1e-4 and e_x <= 1e-4
    L.close()


def test_training_resumes_bit_exactly(tmp_path):
    """12 Adam steps straight through equal 6 steps, a saved training state, a
    new learned form restored from it, and 6 more steps: bit for bit."""
    from paper_2412_02413_gb300 import learn
    w = synth.workload(1)
    w.nz = 24
    pam = _pam()
    B = 4
    rf = torch.from_numpy(np.stack([synth.make_frame(w, 80 + i)[0] for i in range(2 * B)])).cuda()
    La = pam.Learned.from_workload(w, max_frames=2 * B)
    La.set_params(learn.init_params(3))
    feats, tgt, _ = La.example(rf)
    sched = learn.batch_schedule(2, 6, 7)          # 12 steps over 2 batches
    lrs = [learn.lr_at(k, 12, 2e-3, 5e-5) for k in range(12)]

    def run(L, steps):
        for k in steps:
            b = sched[k]
            L.train_step(feats[b * B:(b + 1) * B], tgt[b * B:(b + 1) * B], lrs[k])
        L.sync()

    run(La, range(12))
    p_straight = La.get_params()
    Lb = pam.Learned.from_workload(w, max_frames=2 * B)
    Lb.set_params(learn.init_params(3))
    run(Lb, range(6))
    path = str(tmp_path / "state.npz")
    learn.save_training_state(path, Lb, 6, {"test": True})
    Lb.close()
    state, adam_steps, step, _ = learn.load_training_state(path)
    assert step == 6 and adam_steps == 6
    Lc = pam.Learned.from_workload(w, max_frames=2 * B)
    Lc.set_state(state, adam_steps)
    run(Lc, range(6, 12))
    assert np.array_equal(Lc.get_params(), p_straight)
    assert Lc.info()["adam_steps"] == 12
    La.close()
    Lc.close()


# --------------------------------------------------------------- training --
def _isnr_esa(img, pix_area):
    """Eq. 12: ISNR = 10 log10(mean inside A_0.5 / mean outside), and the
    area A_0.5 of the pixels above half the maximum (ESA)."""
    m = img > 0.5 * img.max()
    inside, outside = img[m].mean(), img[~m].mean()
    return 10.0 * np.log10(inside / outside), m.sum() * pix_area


def test_training_gains_over_plain_as():
    """A short training run on frames the method generates: the loss falls,
    and on held-out frames the learned image has a far higher ISNR than the
    plain AS image (no cross-correlation weight), close to exact AS-TAX."""
    w = synth.workload(1)
    pam = _pam()
    n_train, n_test, B = 192, 16, 16
    L = pam.Learned.from_workload(w, max_frames=B)
    L.set_params(flat(co.init_params(0)))
    feats = L.empty_features(n_train + n_test)
    target = torch.empty((n_train + n_test, w.nz, w.n_elem), dtype=torch.float32, device="cuda")
    energy = torch.empty_like(target)
    rf_all = np.stack([synth.make_frame(w, 2000 + i)[0] for i in range(n_train + n_test)])
    rf_t = torch.from_numpy(rf_all).cuda()
    for s in range(0, n_train + n_test, B):
        L.example(rf_t[s:s + B], features=feats[s:s + B], target=target[s:s + B], energy=energy[s:s + B])
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    losses = []
    gen = torch.Generator().manual_seed(0)
    for step in range(400):
        idx = torch.randint(0, n_train // B, (1,), generator=gen).item() * B
        L.train_step(feats[idx:idx + B], target[idx:idx + B], 2e-3, loss=loss)
        if step % 50 == 0 or step == 399:
            losses.append(float(loss[0].item()))
    L.configure(gate_tol=float("inf"))
    out = L.as_tax(rf_t[n_train:])
    plan = pam.Plan.from_workload(w, max_frames=n_test)
    ref = plan.as_tax(rf_t[n_train:], rho_n=True, image_as=True)
    torch.cuda.synchronize()
    pix = w.pitch * w.dz * 1e6
    gains, gaps, errs_l, errs_as = [], [], [], []
    for f in range(n_test):
        il = out["image"][f].cpu().numpy().astype(np.float64)
        it = ref["image"][f].cpu().numpy().astype(np.float64)
        ia = ref["image_as"][f].cpu().numpy().astype(np.float64)
        s_l, _ = _isnr_esa(il, pix)
        s_t, _ = _isnr_esa(it, pix)
        s_a, _ = _isnr_esa(ia, pix)
        gains.append(s_l - s_a)
        gaps.append(s_t - s_l)
        errs_l.append(rel_l2(il / il.max(), it / it.max()))
        errs_as.append(rel_l2(ia / ia.max(), it / it.max()))
    print(f"training loss {losses[0]:.4f} -> {losses[-1]:.4f}; held-out ISNR gain over AS "
          f"{np.mean(gains):.1f} dB (exact AS-TAX {np.mean(gaps) + np.mean(gains):.1f} dB); rel L2 to AS-TAX "
          f"learned {np.mean(errs_l):.3f} vs AS {np.mean(errs_as):.3f}")
    assert losses[-1] < 0.5 * losses[0]
    assert np.mean(gains) > 3.0
    assert np.mean(errs_l) < np.mean(errs_as)
    plan.close()
    L.close()
