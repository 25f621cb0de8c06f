"""libpam (CUDA, FP32) against the FP64 oracle on the same seeded inputs,
called through the C ABI via the Python binding. The tests cover:
* small grids spanning several CTA tiles with ragged tails;
* both full workloads (64-element and 128-element);
* multi-frame batching;
* AS-DAX and the evanescent-zero flag;
* edge cases: zero input, one bin, one row, the largest nt;
* error handling.
"""
import numpy as np
import pytest

import oracle
from gpu_common import NCC_TOL, REL_L2_TOL, compare_xcorr, geometry_of, peak, rel_l2
from paper_2412_02413_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C = 1540.0


def _pam():
    from paper_2412_02413_gb300 import pam
    return pam


def _tiny(ne, nt, nz, bins=None, fs=20e6, pattern_m=2, z0=4e-3, dz=0.45e-3, f_lo=1e6, f_hi=8e6):
    w = synth.Workload(name="t", n_elem=ne, pitch=0.3e-3, fs=fs, nt=nt, c=C, nz=nz, z_first=z0,
                       z_last=z0 + (nz - 1) * dz if nz > 1 else z0 + dz, f_lo=f_lo, f_hi=f_hi,
                       n_bins=bins, pattern_m=pattern_m)
    if nz == 1:
        w.z_last = z0 + dz  # keeps dz positive; only row 0 is imaged
    return w


def _plan(w, n_apod=3, **kw):
    pam = _pam()
    dz = w.dz if w.nz > 1 else (w.z_last - w.z_first)
    return pam.Plan(n_elem=w.n_elem, pitch=w.pitch, fs=w.fs, c=w.c, n_samples=w.nt, nz=w.nz, z0=w.z0, dz=dz,
                    bins=w.bins(), n_apod=n_apod, pattern_m=w.pattern_m, **kw)


def _geom(w, **kw):
    dz = w.dz if w.nz > 1 else (w.z_last - w.z_first)
    return oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, dz, w.bins(), **kw)


def _run_tax(plan, rf):
    return plan.as_tax(torch.from_numpy(np.ascontiguousarray(rf)).cuda(), rho_n=True, rho_pairs=True,
                       image_as=True)


# ------------------------------------------------------------- small grids --
@pytest.mark.parametrize("ne,nt,nz,nbins", [
    (16, 128, 7, None),     # one CTA tile (256 rows) with a short tail
    (16, 128, 300, None),   # 256 rows per CTA: two tiles, ragged
    (32, 256, 150, None),   # 128 rows per CTA: two tiles, ragged
    (64, 512, 90, None),    # 64 rows per CTA: two tiles, ragged
    (128, 256, 77, 10),     # 32 rows per CTA: three tiles, ragged
])
def test_small_tax_parity(ne, nt, nz, nbins):
    w = _tiny(ne, nt, nz, bins=nbins)
    rf = synth.random_rf(ne, nt, seed=100 + ne)
    plan = _plan(w)
    assert np.array_equal(plan.apod, oracle.pattern(ne, 3, w.pattern_m).astype(np.float32))
    assert np.array_equal(plan.bins, w.bins())
    out = _run_tax(plan, rf)
    torch.cuda.synchronize()
    orc = oracle.as_tax(_geom(w), rf, oracle.pattern(ne, 3, w.pattern_m))
    compare_xcorr(out, orc, check_peak=False)


@pytest.mark.parametrize("apod_index,split", [(-1, 0), (1, 0), (-1, 2)])
def test_backprop_energy_and_fields(apod_index, split):
    w = _tiny(16, 128, 9)
    rf = synth.random_rf(16, 128, seed=7)
    plan = _plan(w)
    plan.set_split(split)
    e, fl = plan.as_backprop(torch.from_numpy(rf).cuda(), apod_index=apod_index, fields=True)
    torch.cuda.synchronize()
    a = None if apod_index < 0 else oracle.pattern(16, 3, 2)[apod_index]
    g = _geom(w)
    want_f = oracle.fields(g, rf, a)
    want_e = oracle.as_backprop(g, rf, a)
    got_f = fl[0].cpu().numpy()
    assert rel_l2(np.abs(got_f), np.abs(want_f)) < REL_L2_TOL
    assert np.max(np.abs(got_f - want_f)) / np.max(np.abs(want_f)) < 1e-5
    assert rel_l2(e[0].cpu().numpy(), want_e) < REL_L2_TOL


def test_gpu_fields_obey_composition():
    """F_x of the GPU field at row j+m equals F_x at row j times exp(i kz m dz)
    for every propagating component (Eq. 2 composes)."""
    w = _tiny(32, 256, 12, z0=2e-3, dz=0.6e-3)
    rf = synth.random_rf(32, 256, seed=9)
    plan = _plan(w)
    _, fl = plan.as_backprop(torch.from_numpy(rf).cuda(), fields=True)
    F = fl[0].cpu().numpy().astype(np.complex128)
    worst = 0.0
    for b, k in enumerate(plan.bins):
        kx, kz = oracle.kz(k * w.fs / w.nt, C, w.pitch, w.n_elem)
        prop = np.abs(kz.imag) == 0
        P0 = np.fft.fft(F[b, 2])
        P1 = np.fft.fft(F[b, 9])
        pred = P0 * np.exp(1j * kz * 7 * w.dz)
        scale = np.max(np.abs(P0))
        worst = max(worst, float(np.max(np.abs(P1[prop] - pred[prop])) / scale))
    assert worst < 1e-5, worst


# ---------------------------------------------------------- full workloads --
@pytest.fixture(scope="module")
def w1_frames():
    w = synth.workload(1)
    frames = [synth.make_frame(w, f) for f in range(3)]
    g = geometry_of(w)
    A = oracle.pattern(w.n_elem, 3, w.pattern_m)
    orc = [oracle.as_tax(g, rf, A) for rf, _ in frames]
    return w, frames, orc


def test_workload1_parity(w1_frames):
    w, frames, orc = w1_frames
    plan = _pam().Plan.from_workload(w)
    for f in range(2):
        out = _run_tax(plan, frames[f][0])
        m = compare_xcorr(out, orc[f])
        assert m["peak_margin"] > 10 * REL_L2_TOL, m


@pytest.mark.parametrize("split", [1, 3, 8, 12])
def test_split_paths_match_oracle(w1_frames, split):
    """Splits up to 8 reduce inside a thread-block cluster, larger ones through
    global partial sums; both must agree with the oracle."""
    w, frames, orc = w1_frames
    plan = _pam().Plan.from_workload(w)
    plan.set_split(split)
    compare_xcorr(_run_tax(plan, frames[0][0]), orc[0])
    e = plan.as_backprop(torch.from_numpy(frames[0][0]).cuda())
    assert rel_l2(e[0].cpu().numpy(), orc[0]["image_as"]) < REL_L2_TOL


@pytest.mark.parametrize("radix", [4, 8])
@pytest.mark.parametrize("nt", [64, 128, 256, 1024])
def test_time_fft_radix_matches_oracle(radix, nt):
    """The time FFT with radix-8 stages (then radix 4 and 2) and with radix-4
    stages (then radix 2), over sequence lengths nt/2 = 32 ... 512 that end in
    each kind of last stage."""
    w = _tiny(16, nt, 9, fs=20e6 * nt / 128)
    rf = synth.random_rf(w.n_elem, w.nt, 40 + nt)
    plan = _plan(w)
    plan.set_fft_radix(radix)
    orc = oracle.as_tax(_geom(w), rf, oracle.pattern(w.n_elem, 3, w.pattern_m))
    compare_xcorr(_run_tax(plan, rf), orc, check_peak=False)


@pytest.mark.parametrize("lane_rows", [1, 2])
@pytest.mark.parametrize("grid", [0, 1, 37, 100, 151])
def test_fused_grid_matches_oracle_and_is_deterministic(w2_frame, grid, lane_rows):
    """The even division over any number of CTAs (one per SM, down to one)
    agrees with the oracle, and a given count reproduces its bits, with one
    or two depth rows per lane."""
    w, rf, src, orc = w2_frame
    plan = _pam().Plan.from_workload(w, max_frames=1)
    plan.set_grid(grid)
    plan.set_lane_rows(lane_rows)
    a = _run_tax(plan, rf)
    compare_xcorr(a, orc)
    b = _run_tax(plan, rf)
    assert torch.equal(a["image"], b["image"]) and torch.equal(a["rho_pairs"], b["rho_pairs"])


@pytest.mark.parametrize("ne,nt,nz,nbins", [
    (16, 128, 300, None),   # nx 16: 256-row tiles, ragged
    (32, 256, 77, 20),      # nx 32
    (64, 256, 70, 33),      # nx 64: 64-row tiles, 96 with two rows per lane
    (128, 512, 45, 17),     # nx 128: 32-row tiles, 48 with two rows per lane
])
def test_two_rows_per_lane_matches_one_row(ne, nt, nz, nbins):
    """Two depth rows per lane run each row's arithmetic exactly as one row per
    lane. With one CTA (every tile in one pass over the bins) the AS, AS-DAX
    and AS-TAX maps are bit-identical; over the full grid, where the larger
    row tiles of nx >= 64 group the bins' partial sums differently (bit-identical
    below nx = 64), both match the oracle, over ragged tiles, several frames
    and a split of the bins across CTAs."""
    w = _tiny(ne, nt, nz, bins=nbins, fs=40e6, pattern_m=max(2, ne // 8))
    frames = synth.random_rf(ne, nt, seed=60 + ne, n_frames=3)
    rf = torch.from_numpy(frames).cuda()
    for n_apod, call in ((3, "as_tax"), (2, "as_dax")):
        plan = _plan(w, n_apod=n_apod, max_frames=3)
        for grid in (1, 0, 5):
            plan.set_grid(grid)
            plan.set_lane_rows(1)
            one = {k: v.clone() for k, v in getattr(plan, call)(rf, rho_pairs=True, image_as=True).items()}
            plan.set_lane_rows(2)
            two = getattr(plan, call)(rf, rho_pairs=True, image_as=True)
            torch.cuda.synchronize()
            if grid == 1 or ne < 64:
                for k in one:
                    assert torch.equal(one[k], two[k]), (n_apod, grid, k)
            A = oracle.pattern(ne, n_apod, w.pattern_m)
            orc = (oracle.as_tax if n_apod == 3 else oracle.as_xcorr)(_geom(w), frames[2], A)
            compare_xcorr({k: v[2:3] for k, v in two.items()}, orc, check_peak=False)
        plan.close()
    plan = _plan(w, n_apod=1, max_frames=3)
    plan.set_grid(1)
    plan.set_lane_rows(1)
    e1 = plan.as_backprop(rf).clone()
    plan.set_lane_rows(2)
    e2 = plan.as_backprop(rf)
    torch.cuda.synchronize()
    assert torch.equal(e1, e2)
    with pytest.raises(_pam().PamError):
        plan.set_lane_rows(3)
    plan.close()


def test_workload1_batched_frames(w1_frames):
    """Three frames in one call with max_frames = 2 (two kernel batches)."""
    w, frames, orc = w1_frames
    plan = _pam().Plan.from_workload(w, max_frames=2)
    rf = np.stack([fr[0] for fr in frames])
    out = _run_tax(plan, rf)
    for f in range(3):
        compare_xcorr(out, orc[f], f=f)


@pytest.fixture(scope="module")
def w2_frame():
    w = synth.workload(2)
    rf, src = synth.make_frame(w, 0)
    orc = oracle.as_tax(geometry_of(w), rf, oracle.pattern(w.n_elem, 3, w.pattern_m))
    return w, rf, src, orc


def test_workload2_parity(w2_frame):
    """The 128-element, 128 x 512, 300-bin frame in the one-frame launch
    configuration that bench.py times."""
    w, rf, src, orc = w2_frame
    plan = _pam().Plan.from_workload(w, max_frames=1)
    out = _run_tax(plan, rf)
    m = compare_xcorr(out, orc)
    assert m["peak_margin"] > 10 * REL_L2_TOL, m
    jz, ix = m["peak"]
    assert any(abs(ix - s.ix) <= 1 and abs(jz - s.iz) <= 2 for s in src), (m["peak"], src)


def test_workload2_backprop_matches_image_as(w2_frame):
    """Eq. 3 full-aperture energy equals the summed-aperture energy of the TAX
    call (Pattern-16 masks sum to one)."""
    w, rf, src, orc = w2_frame
    plan = _pam().Plan.from_workload(w)
    e = plan.as_backprop(torch.from_numpy(rf).cuda())
    assert rel_l2(e[0].cpu().numpy(), orc["image_as"]) < REL_L2_TOL


# ----------------------------------------------------------------- variants --
def test_dax_parity(w1_frames):
    w, frames, _ = w1_frames
    pam = _pam()
    plan = pam.Plan.from_workload(w, n_apod=2)
    rf = frames[0][0]
    out = plan.as_dax(torch.from_numpy(rf).cuda(), rho_n=True, rho_pairs=True, image_as=True)
    orc = oracle.as_xcorr(geometry_of(w), rf, oracle.pattern(w.n_elem, 2, w.pattern_m))
    compare_xcorr(out, orc)


def test_evanescent_zero_parity():
    w = _tiny(32, 256, 20, f_lo=0.3e6, f_hi=4e6)
    rf = synth.random_rf(32, 256, seed=21)
    plan = _plan(w, evanescent_zero=True)
    out = _run_tax(plan, rf)
    orc = oracle.as_tax(_geom(w, evanescent_zero=True), rf, oracle.pattern(32, 3, 2))
    compare_xcorr(out, orc, check_peak=False)


def _zero_stuffed(w, rf, apod):
    """Oracle inputs for 2x zero-stuffing in the channel direction (Sec. II-D):
    2 n_elem channels at pitch/2, element e on channel 2e, odd channels zero,
    and each aperture's weight of element e on channel 2e."""
    ne = w.n_elem
    rf2 = np.zeros((2 * ne, rf.shape[-1]), np.float32)
    rf2[0::2] = rf
    a2 = np.zeros((apod.shape[0], 2 * ne))
    a2[:, 0::2] = apod
    dz = w.dz if w.nz > 1 else (w.z_last - w.z_first)
    g = oracle.Geometry(2 * ne, w.nt, w.fs, w.c, w.pitch / 2, w.nz, w.z0, dz, w.bins())
    return g, rf2, a2


@pytest.mark.parametrize("ne,nt,nz", [(16, 256, 21), (64, 1024, 40)])
def test_lateral_upsample2x_parity(ne, nt, nz):
    w = _tiny(ne, nt, nz, pattern_m=4 if ne == 16 else 8)
    w.source_z = (w.z0, w.z0 + (nz - 1) * w.dz)
    rf = synth.make_frame(w, 3)[0] if ne == 64 else synth.random_rf(ne, nt, seed=31)
    plan = _plan(w, upsample2x=True)
    assert plan.nx == 2 * ne
    out = _run_tax(plan, rf)
    apod = oracle.pattern(ne, 3, w.pattern_m)
    g, rf2, a2 = _zero_stuffed(w, rf, apod)
    orc = oracle.as_tax(g, rf2, a2)
    compare_xcorr(out, orc, check_peak=(ne == 64))
    # the full-aperture back-propagation on the same virtual array
    e = plan.as_backprop(torch.from_numpy(np.ascontiguousarray(rf)).cuda())
    want = oracle.as_backprop(g, rf2, np.where(np.arange(2 * ne) % 2 == 0, 1.0, 0.0))
    assert rel_l2(e[0].cpu().numpy(), want) <= REL_L2_TOL
    plan.close()


@pytest.mark.parametrize("ne,nt,nz", [(16, 256, 21), (64, 1024, 40)])
def test_lateral_pad2x_parity(ne, nt, nz):
    """2x lateral padding (Sec. II-D): transforms over 2 n_elem points, maps
    cropped to the element columns, rho_n normalised over the crop."""
    w = _tiny(ne, nt, nz, pattern_m=4 if ne == 16 else 8)
    w.source_z = (w.z0, w.z0 + (nz - 1) * w.dz)
    rf = synth.make_frame(w, 4)[0] if ne == 64 else synth.random_rf(ne, nt, seed=33)
    plan = _plan(w, pad2x=True)
    assert plan.nx == ne
    out = _run_tax(plan, rf)
    assert tuple(out["image"].shape) == (1, nz, ne)
    apod = oracle.pattern(ne, 3, w.pattern_m)
    orc = oracle.as_xcorr_pad2x(_geom(w), rf, apod)
    compare_xcorr(out, orc, check_peak=(ne == 64))
    assert float(out["rho_n"].max()) == 1.0
    rft = torch.from_numpy(np.ascontiguousarray(rf)).cuda()
    e = plan.as_backprop(rft)
    assert rel_l2(e[0].cpu().numpy(), oracle.as_backprop_pad2x(_geom(w), rf)) <= REL_L2_TOL
    # the padding matters: the unpadded maps differ well above the tolerance
    plain = _plan(w)
    assert rel_l2(plain.as_backprop(rft)[0].cpu().numpy(), oracle.as_backprop_pad2x(_geom(w), rf)) > 1e-3
    plain.close()
    plan.close()


def test_lateral_pad2x_dax_host_and_frames():
    """AS-DAX, several frames per call (max_frames 2, so two chunks) and the
    host-buffer entry point, all with 2x lateral padding."""
    w = _tiny(32, 256, 9, pattern_m=4)
    rfs = np.stack([synth.random_rf(32, 256, seed=40 + f) for f in range(3)])
    A = oracle.pattern(32, 2, 4)
    plan = _plan(w, n_apod=2, pad2x=True, max_frames=2)
    out = plan.as_dax(torch.from_numpy(rfs).cuda(), rho_n=True, rho_pairs=True, image_as=True)
    img_h = np.zeros((3, w.nz, 32), np.float32)
    rho_h = np.zeros_like(img_h)
    plan.as_xcorr_host(rfs, img_h, rho_h)
    for f in range(3):
        orc = oracle.as_xcorr_pad2x(_geom(w), rfs[f], A)
        compare_xcorr(out, orc, f=f, check_peak=False)
        assert rel_l2(img_h[f], orc["image"]) <= REL_L2_TOL
        assert np.max(np.abs(rho_h[f] - orc["rho_n"])) <= NCC_TOL
    plan.close()


def test_lateral_pad2x_rejections():
    pam = _pam()
    with pytest.raises(pam.PamError):          # 2 n_elem = 256 is not built
        _plan(_tiny(128, 256, 8), pad2x=True)
    with pytest.raises(pam.PamError):          # tensor-core forms run without it
        _plan(_tiny(64, 256, 8), pad2x=True, form="bf16")
    with pytest.raises(pam.PamError):          # not together with zero-stuffing
        _plan(_tiny(16, 256, 8), pad2x=True, upsample2x=True)
    with pytest.raises(pam.PamError):          # the image is n_elem wide
        _plan(_tiny(16, 256, 8), pad2x=True, nx=32)
    plan = _plan(_tiny(16, 256, 8), pad2x=True)
    with pytest.raises(pam.PamError):          # no fields output
        plan.as_backprop(torch.zeros((1, 16, 256), device="cuda"), fields=True)
    plan.close()


def test_lateral_upsample2x_rejections():
    pam = _pam()
    w = _tiny(16, 256, 8)
    with pytest.raises(pam.PamError):          # nx = 2 n_elem = 256 is not built
        _plan(_tiny(128, 256, 8), upsample2x=True)
    with pytest.raises(pam.PamError):          # tensor-core forms run without it
        _plan(_tiny(64, 256, 8), upsample2x=True, form="bf16")
    with pytest.raises(pam.PamError):          # nx must be 2 n_elem
        _plan(w, upsample2x=True, nx=16)


def test_identical_apertures_give_unit_ncc():
    w = _tiny(64, 512, 40)
    rf = synth.random_rf(64, 512, seed=22)
    plan = _plan(w, apod=np.ones((3, 64), np.float32))
    out = _run_tax(plan, rf)
    assert float(torch.max(torch.abs(out["rho_pairs"] - 1))) <= NCC_TOL
    assert float(torch.max(torch.abs(out["rho_n"] - 1))) <= NCC_TOL


def test_point_source_lands_on_its_pixel():
    from oracle_pins import as_point_source_rf
    ne, nt, fs = 64, 512, 20e6
    w = _tiny(ne, nt, 40, f_lo=2e6, f_hi=8e6, z0=4e-3, dz=0.4e-3)
    rf = as_point_source_rf(ne, nt, fs, 0.3e-3, w.bins(), 23, w.z0 + 17 * w.dz)
    plan = _plan(w)
    out = _run_tax(plan, rf)
    assert peak(out["image"][0].cpu().numpy()) == (17, 23)
    assert peak(out["image_as"][0].cpu().numpy()) == (17, 23)


# --------------------------------------------------------------- edge cases --
def test_zero_input():
    w = _tiny(32, 256, 10)
    plan = _plan(w)
    out = _run_tax(plan, np.zeros((32, 256), np.float32))
    assert float(out["image"].abs().max()) == 0.0
    assert torch.all(out["rho_n"] == 1.0)
    assert torch.all(out["rho_pairs"] == np.float32(1e-3))


def test_one_bin_one_row():
    w = _tiny(64, 512, 1, bins=1, f_lo=3e6, f_hi=3.02e6)
    assert w.bins().size == 1
    rf = synth.random_rf(64, 512, seed=23)
    plan = _plan(w)
    out = _run_tax(plan, rf)
    orc = oracle.as_tax(_geom(w), rf, oracle.pattern(64, 3, 2))
    compare_xcorr(out, orc, check_peak=False)


def test_largest_nt():
    w = _tiny(128, 8192, 20, bins=12, fs=40e6, f_lo=0.5e6, f_hi=8e6, pattern_m=16)
    rf = synth.random_rf(128, 8192, seed=24)
    plan = _plan(w)
    out = _run_tax(plan, rf)
    orc = oracle.as_tax(_geom(w), rf, oracle.pattern(128, 3, 16))
    compare_xcorr(out, orc, check_peak=False)


def test_empty_call_and_determinism():
    w = _tiny(32, 256, 30)
    rf = torch.from_numpy(synth.random_rf(32, 256, seed=25)).cuda()
    plan = _plan(w)
    a = plan.as_tax(rf, rho_pairs=True)
    b = plan.as_tax(rf, rho_pairs=True)
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k
    plan.sync()


def test_bad_pointers_are_rejected():
    pam = _pam()
    w = _tiny(32, 256, 10)
    plan = _plan(w)
    L = pam.load()
    rf = torch.zeros(1, 32, 256, device="cuda")
    img = torch.zeros(1, 10, 32, device="cuda")
    base = int(rf.data_ptr())
    assert L.pam_as_tax(plan.handle, base + 4, 1, int(img.data_ptr()), None, None, None, None) == 1
    host = np.zeros((32, 256), np.float32)
    assert L.pam_as_tax(plan.handle, host.ctypes.data, 1, int(img.data_ptr()), None, None, None, None) == 1
    assert L.pam_as_tax(plan.handle, base, 0, int(img.data_ptr()), None, None, None, None) == 0
    assert L.pam_as_tax(plan.handle, base, -1, int(img.data_ptr()), None, None, None, None) == 1
    assert L.pam_as_backprop(plan.handle, base, 1, 3, int(img.data_ptr()), None, None) == 1
    with pytest.raises(TypeError):
        plan.as_tax(torch.zeros(1, 32, 256))


def test_host_entry_point_matches_device(w1_frames):
    w, frames, orc = w1_frames
    plan = _pam().Plan.from_workload(w, max_frames=2)
    rf = np.stack([fr[0] for fr in frames])
    img = np.zeros((3, w.nz, w.nx), np.float32)
    rho = np.zeros((3, w.nz, w.nx), np.float32)
    plan.as_xcorr_host(rf, img, rho)
    dev = plan.as_tax(torch.from_numpy(rf).cuda())
    assert np.array_equal(img, dev["image"].cpu().numpy())
    assert np.array_equal(rho, dev["rho_n"].cpu().numpy())
    for f in range(3):
        assert rel_l2(img[f], orc[f]["image"]) <= REL_L2_TOL


def test_async_host_entry_point_pipelined(w1_frames):
    """pam_as_xcorr_host_async on two plans and two streams, results read after
    each stream's event: identical to the blocking entry point."""
    w, frames, _ = w1_frames
    pam = _pam()
    plans = [pam.Plan.from_workload(w), pam.Plan.from_workload(w)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    rf = [np.ascontiguousarray(fr[0]) for fr in frames]
    pinned = [torch.from_numpy(r).pin_memory().numpy() for r in rf]
    outs = [(torch.zeros(1, w.nz, w.nx).pin_memory().numpy(), torch.zeros(1, w.nz, w.nx).pin_memory().numpy())
            for _ in rf]
    for i, r in enumerate(pinned):
        plans[i % 2].as_xcorr_host_async(r, outs[i][0], outs[i][1], stream=streams[i % 2])
    torch.cuda.synchronize()
    for i, r in enumerate(rf):
        img = np.zeros((1, w.nz, w.nx), np.float32)
        rho = np.zeros((1, w.nz, w.nx), np.float32)
        plans[0].as_xcorr_host(r, img, rho)
        assert np.array_equal(outs[i][0], img) and np.array_equal(outs[i][1], rho)
    for p in plans:
        p.close()


def test_plans_of_different_sizes_coexist():
    """A plan with a smaller time FFT created later must not break an earlier
    plan with a larger one (kernel attributes are process-wide)."""
    big = _tiny(32, 4096, 10, bins=5, fs=40e6, f_lo=1e6, f_hi=8e6)
    small = _tiny(32, 256, 10)
    pb = _plan(big)
    rf_big = synth.random_rf(32, 4096, seed=27)
    ref = _run_tax(pb, rf_big)["image"].clone()
    ps = _plan(small)
    _run_tax(ps, synth.random_rf(32, 256, seed=28))
    again = _run_tax(pb, rf_big)["image"]
    torch.cuda.synchronize()
    assert torch.equal(ref, again)


def test_profile_counters():
    w = _tiny(32, 256, 10)
    plan = _plan(w)
    rf = torch.from_numpy(synth.random_rf(32, 256, seed=26)).cuda()
    for split, kernels in ((4, 4), (16, 5)):   # cluster path / global-partials path
        plan.set_split(split)
        plan.profile_enable(True)
        for _ in range(3):
            plan.as_tax(rf)
        ms, n, k = plan.profile_read()
        assert n == 3 and k == 3 * kernels and ms > 0
    plan.profile_enable(False)


# ------------------------------------------------------ tensor-core form --
# The propagation as a tcgen05 GEMM with 16-bit operands. Tolerances are those
# stated for the chosen forms: relative L2 <= 1e-2 on the energy maps and the
# same brightest pixel; NCC deviations are reported. The hi + lo split recovers
# close to FP32 agreement.
FORM_TOL = {"bf16": (1e-2, 5e-2), "fp16": (1e-2, 2e-2), "bf16split": (1e-4, 1e-3), "fp16split": (1e-5, 1e-5)}


@pytest.mark.parametrize("form", ["bf16", "fp16", "bf16split", "fp16split"])
def test_gemm_form_workload2(w2_frame, form):
    w, rf, src, orc = w2_frame
    plan = _pam().Plan.from_workload(w, max_frames=1, form=form)
    out = _run_tax(plan, rf)
    img = out["image"][0].cpu().numpy()
    err = {k: rel_l2(out[k][0].cpu().numpy(), orc[k]) for k in ("image", "image_as")}
    ncc = float(np.max(np.abs(out["rho_pairs"][0].cpu().numpy() - orc["rho_pairs"])))
    rn = float(np.max(np.abs(out["rho_n"][0].cpu().numpy() - orc["rho_n"])))
    print(f"\n{form}: rel L2 image {err['image']:.3e} image_as {err['image_as']:.3e} "
          f"max|dNCC| {ncc:.3e} max|d rho_n| {rn:.3e}")
    l2_tol, ncc_tol = FORM_TOL[form]
    assert err["image"] <= l2_tol and err["image_as"] <= l2_tol, err
    assert ncc <= ncc_tol and rn <= ncc_tol, (ncc, rn)
    assert peak(img) == peak(orc["image"])


@pytest.mark.parametrize("form", ["bf16", "fp16", "fp16split"])
def test_gemm_form_frame_groups(form):
    """20 frames: two groups of 16 frames (the second one ragged) in one call,
    each frame against the oracle."""
    w = _tiny(128, 512, 24, bins=12, fs=40e6, f_lo=1e6, f_hi=8e6, pattern_m=16)
    frames = synth.random_rf(128, 512, seed=31, n_frames=20)
    frames[3] *= 1000.0                # frame scale must not matter (per-frame power-of-2 scaling)
    plan = _plan(w, max_frames=20, form=form)
    out = _run_tax(plan, frames)
    g = _geom(w)
    A = oracle.pattern(128, 3, 16)
    worst = 0.0
    for f in (0, 3, 15, 16, 19):
        orc = oracle.as_tax(g, frames[f], A)
        worst = max(worst, rel_l2(out["image_as"][f].cpu().numpy(), orc["image_as"]))
    assert worst <= FORM_TOL[form][0], worst


@pytest.mark.parametrize("form", ["bf16", "bf16split", "fp16split"])
def test_gemm_form_overlapping_apertures(form):
    """AS-DAX with two overlapping apertures of non-uniform weight whose edges
    are not on 8-element boundaries: the element blocks an aperture touches
    carry weight 0 outside it, and a shared element sits in both K ranges."""
    w = _tiny(128, 512, 40, bins=16, fs=40e6, f_lo=1e6, f_hi=8e6, pattern_m=16)
    e = np.arange(128)
    A = np.zeros((2, 128), np.float32)
    A[0, :70] = 0.5 + 0.5 * np.cos(np.pi * e[:70] / 71.0)
    A[1, 37:] = 0.75 + 0.25 * np.sin(e[37:] / 9.0)
    rf = synth.random_rf(128, 512, seed=33)
    plan = _plan(w, n_apod=2, apod=A, form=form)
    out = plan.as_dax(torch.from_numpy(rf).cuda(), rho_n=True, rho_pairs=True, image_as=True)
    orc = oracle.as_xcorr(_geom(w), rf, A)
    err = {k: rel_l2(out[k][0].cpu().numpy(), orc[k]) for k in ("image", "image_as")}
    ncc = float(np.max(np.abs(out["rho_pairs"][0].cpu().numpy() - orc["rho_pairs"])))
    l2_tol, ncc_tol = FORM_TOL[form]
    assert err["image"] <= l2_tol and err["image_as"] <= l2_tol, err
    assert ncc <= ncc_tol, ncc


def test_gemm_tile_and_frames_options_on_dax():
    """The two-aperture kernels under every (M tile, frames per CTA) pair:
    AS-DAX with overlapping, unaligned apertures, 18 frames (a ragged group of
    16 and of 32) and 13 rows (a pair with one row), bit-identical to the
    default and within the split form's tolerance of the oracle."""
    w = _tiny(128, 512, 13, bins=10, fs=40e6, f_lo=1e6, f_hi=8e6, pattern_m=16)
    e = np.arange(128)
    A = np.zeros((2, 128), np.float32)
    A[0, :70] = 0.5 + 0.5 * np.cos(np.pi * e[:70] / 71.0)
    A[1, 37:] = 0.75 + 0.25 * np.sin(e[37:] / 9.0)
    frames = synth.random_rf(128, 512, seed=37, n_frames=18)
    rf = torch.from_numpy(frames).cuda()
    plan = _plan(w, n_apod=2, apod=A, max_frames=18, form="fp16split")
    kw = dict(rho_n=True, rho_pairs=True, image_as=True)
    ref = {k: v.clone() for k, v in plan.as_dax(rf, **kw).items()}
    for m, fg in ((256, 32), (128, 16), (256, 16)):
        plan.set_gemm_tile(m)
        plan.set_gemm_frames(fg)
        out = plan.as_dax(rf, **kw)
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(ref[k], out[k]), (m, fg, k)
    orc = oracle.as_xcorr(_geom(w), frames[17], A)
    assert rel_l2(out["image"][17].cpu().numpy(), orc["image"]) <= FORM_TOL["fp16split"][0]
    assert float(np.max(np.abs(out["rho_pairs"][17].cpu().numpy() - orc["rho_pairs"]))) <= FORM_TOL["fp16split"][1]


def test_gemm_form_rejects_unsupported():
    pam = _pam()
    with pytest.raises(pam.PamError):
        _plan(_tiny(64, 512, 8), form="bf16")                       # nx must be 128
    w = _tiny(128, 512, 8, pattern_m=16)
    with pytest.raises(pam.PamError):
        _plan(w, apod=np.ones((3, 128), np.float32), form="bf16")    # 3 x 16 element blocks: K too deep


@pytest.mark.parametrize("form", ["bf16", "fp16split"])
def test_gemm_tile_pairs_match_single_rows(form):
    """The 2-CTA tile (M = 256, cta_group::2: one MMA covers two depth rows)
    and 16 frames per CTA (N = 32) sum the same products in the same order as
    one CTA per row with 32 frames, so the maps are bit-identical; 23 rows
    leave the last pair with one row, and 20 frames make a ragged last frame
    group (of 16 and of 32)."""
    w = _tiny(128, 512, 23, bins=12, fs=40e6, f_lo=1e6, f_hi=8e6, pattern_m=16)
    frames = torch.from_numpy(synth.random_rf(128, 512, seed=35, n_frames=20)).cuda()
    plan = _plan(w, max_frames=20, form=form)
    kw = dict(rho_n=True, rho_pairs=True, image_as=True)
    plan.set_gemm_tile(128)
    plan.set_gemm_frames(32)
    one = {k: v.clone() for k, v in plan.as_tax(frames, **kw).items()}
    for m, fg in ((256, 32), (128, 16), (256, 16)):
        plan.set_gemm_tile(m)
        plan.set_gemm_frames(fg)
        two = plan.as_tax(frames, **kw)
        torch.cuda.synchronize()
        for k in one:
            assert torch.equal(one[k], two[k]), (m, fg, k)
    orc = oracle.as_tax(_geom(w), frames[19].cpu().numpy(), oracle.pattern(128, 3, 16))
    assert rel_l2(two["image_as"][19].cpu().numpy(), orc["image_as"]) <= FORM_TOL[form][0]
    with pytest.raises(_pam().PamError):
        plan.set_gemm_tile(64)
    with pytest.raises(_pam().PamError):
        plan.set_gemm_frames(8)
