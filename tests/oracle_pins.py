"""Pins of the FP64 oracle to facts that do not come from the oracle itself:
values printed in the paper, closed forms, invariants, and special cases that
reduce to a library routine. Each pin is a plain function that raises
AssertionError when it fails. ``test_oracle_pins.py`` runs them all on the
correct oracle. ``test_oracle_mutations.py`` runs them against deliberately
broken oracles and requires that every planted mistake trips at least one.
"""
from __future__ import annotations

import os

import numpy as np

import oracle
from paper_2412_02413_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
EPS = 1e-3
C = 1540.0


def _geom(ne=16, nt=128, fs=20e6, nz=6, z0=3e-3, dz=0.7e-3, bins=None, pitch=0.3e-3, evz=False):
    if bins is None:
        bins = oracle.band_bins(nt, fs, 1e6, 8e6)
    return oracle.Geometry(ne, nt, fs, C, pitch, nz, z0, dz, bins, evanescent_zero=evz)


def _rand_rf(ne, nt, seed):
    return synth.random_rf(ne, nt, seed)


# ------------------------------------------------------------ apodization --
def pin_golden_patterns():
    """Sec. II-A and II-C print the Pattern-2 vectors for 8 elements (n=2) and
    12 elements (n=3)."""
    rows = {}
    with open(os.path.join(GOLDEN, "apodization_patterns.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, w = line.split(":")
            ne, na, m, q = map(int, head.split())
            rows[(ne, na, m, q)] = np.array([float(v) for v in w.split()])
    assert len(rows) == 5
    for (ne, na, m, q), want in rows.items():
        got = oracle.pattern(ne, na, m)[q]
        assert np.array_equal(got, want), (ne, na, m, q, got, want)


# -------------------------------------------------------------- time DFT --
def pin_time_dft_is_rfft():
    """Eq. 1 F_t reduces to numpy's real FFT at the selected bins."""
    rf = _rand_rf(6, 128, 11)
    bins = np.arange(1, 64)
    got = oracle.time_dft(rf, bins)
    want = np.fft.rfft(rf.astype(np.float64), axis=1)[:, bins].T
    assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))


def pin_time_dft_tone():
    """A cos(2 pi k0 t/nt + theta) has spectrum (nt/2) A e^{i theta} at k0 and
    nothing at other bins (forward convention exp(-i w t))."""
    nt, k0, A, th = 256, 37, 0.75, 0.4
    t = np.arange(nt)
    rf = np.stack([A * np.cos(2 * np.pi * k0 * t / nt + th + 0.3 * e) for e in range(4)]).astype(np.float32)
    S = oracle.time_dft(rf, [k0, k0 + 1, 5])
    for e in range(4):
        want = nt / 2 * A * np.exp(1j * (th + 0.3 * e))
        assert abs(S[0, e] - want) < 2e-4 * abs(want), (S[0, e], want)
        assert abs(S[1, e]) < 2e-4 * abs(want) and abs(S[2, e]) < 2e-4 * abs(want)


def pin_time_parseval():
    """sum_t x^2 = (2/nt) sum_{0<k<nt/2} |X_k|^2 for a signal with no DC and no
    Nyquist content."""
    nt = 128
    rng = np.random.default_rng(5)
    spec = np.zeros(nt // 2 + 1, complex)
    spec[1:nt // 2] = rng.standard_normal(nt // 2 - 1) + 1j * rng.standard_normal(nt // 2 - 1)
    x = np.fft.irfft(spec, nt).astype(np.float32)
    S = oracle.time_dft(x[None, :], np.arange(1, nt // 2))
    lhs = float(np.sum(x.astype(np.float64) ** 2))
    rhs = 2.0 / nt * float(np.sum(np.abs(S) ** 2))
    assert abs(lhs - rhs) < 1e-10 * lhs


# ----------------------------------------------------------- lateral DFT --
def pin_lateral_dft_is_fft():
    """Eq. 1 F_x of the apodized row reduces to numpy's FFT."""
    rng = np.random.default_rng(3)
    s = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    a = rng.uniform(-1, 1, 16)
    got = oracle.lateral_dft(s, a)
    want = np.fft.fft(a * s)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def pin_lateral_parseval_and_roundtrip():
    """Inverse lateral DFT: sum_i |p_i|^2 = (1/nx) sum_u |P_u|^2, and it undoes
    the forward DFT."""
    rng = np.random.default_rng(4)
    P = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    p = oracle.lateral_idft(P)
    assert abs(np.sum(np.abs(p) ** 2) - np.sum(np.abs(P) ** 2) / 32) < 1e-12 * np.sum(np.abs(P) ** 2)
    s = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    back = oracle.lateral_idft(oracle.lateral_dft(s))
    assert np.max(np.abs(back - s)) < 1e-12 * np.max(np.abs(s))


# ----------------------------------------------------------- propagation --
def _plane_wave_case(u0, k0=20, ne=16, nt=128, fs=20e6, pitch=0.3e-3):
    """rf_e(t) = cos(w0 t + kx0 x_e) with w0 on bin k0 and kx0 on lateral bin u0.
    Closed form under Eq. 1-2: p~(x_i, z) = (nt/2) exp(i (kx0 x_i + kz0 z))."""
    up = u0 - ne if 2 * u0 >= ne else u0
    kx0 = 2 * np.pi * up / (ne * pitch)
    f0 = k0 * fs / nt
    k = 2 * np.pi * f0 / C
    kz0 = np.sqrt(complex(k * k - kx0 * kx0))
    xe = (np.arange(ne) - (ne - 1) / 2) * pitch
    t = np.arange(nt) / fs
    rf = np.cos(2 * np.pi * f0 * t[None, :] + kx0 * xe[:, None]).astype(np.float64)
    return rf, kx0, kz0, xe


def pin_plane_wave_exact_phase():
    """Eq. 2 moves a single plane-wave component by exactly kz0*z in phase, and
    decays an evanescent one by exp(-kappa z)."""
    ne, nt, fs, pitch = 16, 128, 20e6, 0.3e-3
    for u0, k0 in ((3, 20), (13, 20), (2, 40), (7, 8)):
        rf, kx0, kz0, xe = _plane_wave_case(u0, k0, ne, nt, fs, pitch)
        g = oracle.Geometry(ne, nt, fs, C, pitch, 5, 1e-3, 0.9e-3, [k0])
        F = oracle.fields(g, rf.astype(np.float32), None)[0]  # [nz][nx]
        z = 1e-3 + np.arange(5) * 0.9e-3
        want = nt / 2 * np.exp(1j * (kx0 * xe[None, :] + kz0 * z[:, None]))
        err = np.max(np.abs(F - want)) / (nt / 2)
        assert err < 5e-5, (u0, k0, err)   # float32 rf limits the agreement


def pin_evanescent_zero_plane_waves():
    """The evanescent-zero reading of Eq. 2: a plane wave whose lateral
    wavenumber exceeds w/c (kz imaginary) is removed at every depth, while a
    propagating one keeps the exact phase shift kz0*z of the closed form."""
    ne, nt, fs, pitch = 16, 128, 20e6, 0.3e-3
    z = 1e-3 + np.arange(5) * 0.9e-3
    # (4, 8): f0 = 1.25 MHz, |kx0| = 5236 rad/m > w/c = 5100 rad/m -> evanescent
    # (kappa = 1190 rad/m, so the principal branch still leaves 0.4% at 4.6 mm)
    rf, kx0, kz0, xe = _plane_wave_case(4, 8, ne, nt, fs, pitch)
    assert kz0.imag > 0 and kz0.real == 0
    g = oracle.Geometry(ne, nt, fs, C, pitch, 5, 1e-3, 0.9e-3, [8], evanescent_zero=True)
    F = oracle.fields(g, rf.astype(np.float32), None)[0]
    # float32 rf leaks about 1e-7 of the amplitude into the other lateral bins;
    # those are evanescent too at 1.25 MHz except u = 0, +-1 (|kx| <= 2094 rad/m)
    lead = np.max(np.abs(F))
    assert lead < 1e-5 * nt / 2, lead
    g0 = oracle.Geometry(ne, nt, fs, C, pitch, 5, 1e-3, 0.9e-3, [8], evanescent_zero=False)
    F0 = oracle.fields(g0, rf.astype(np.float32), None)[0]
    decay = nt / 2 * np.exp(-kz0.imag * z)
    assert np.allclose(np.max(np.abs(F0), axis=1), decay, rtol=1e-3), "principal branch keeps the decay"
    # (3, 20): f0 = 3.125 MHz, |kx0| = 3927 rad/m < w/c = 12750 rad/m -> propagating
    rf, kx0, kz0, xe = _plane_wave_case(3, 20, ne, nt, fs, pitch)
    assert kz0.imag == 0
    g = oracle.Geometry(ne, nt, fs, C, pitch, 5, 1e-3, 0.9e-3, [20], evanescent_zero=True)
    F = oracle.fields(g, rf.astype(np.float32), None)[0]
    want = nt / 2 * np.exp(1j * (kx0 * xe[None, :] + kz0.real * z[:, None]))
    assert np.max(np.abs(F - want)) / (nt / 2) < 5e-5


def pin_evanescent_zero_propagator():
    """Eq. 2 with evanescent components dropped, on a random spectrum at a bin
    that holds both kinds: the propagating entries equal Q exp(i kz z) and the
    evanescent entries are exactly zero."""
    rng = np.random.default_rng(31)
    nx, z = 32, 3.3e-3
    _, kzv = oracle.kz(1.6e6, C, 0.3e-3, nx)
    ev = kzv.imag > 0
    assert ev.any() and (~ev).any()
    Q = rng.standard_normal(nx) + 1j * rng.standard_normal(nx)
    P = oracle.propagate(Q, kzv, z, evanescent_zero=True)
    assert np.all(P[ev] == 0)
    assert np.max(np.abs(P[~ev] - Q[~ev] * np.exp(1j * kzv[~ev].real * z))) < 1e-12 * np.max(np.abs(Q))


def pin_composition_law():
    """Eq. 2 composes: propagating by z1 then z2 equals propagating by z1+z2,
    for propagating and evanescent components alike."""
    rng = np.random.default_rng(8)
    nx = 32
    for f in (0.8e6, 3.0e6, 7.5e6):
        _, kzv = oracle.kz(f, C, 0.3e-3, nx)
        Q = rng.standard_normal(nx) + 1j * rng.standard_normal(nx)
        z1, z2 = 4.1e-3, 2.7e-3
        two = oracle.propagate(oracle.propagate(Q, kzv, z1), kzv, z2)
        one = oracle.propagate(Q, kzv, z1 + z2)
        assert np.max(np.abs(two - one)) < 1e-12 * np.max(np.abs(Q)), f


def pin_depth_parseval():
    """With no evanescent component in a bin, sum_x |p~(x, z)|^2 is the same at
    every depth (unit-modulus propagator + lateral Parseval)."""
    ne, nt, fs = 16, 128, 20e6
    fmin = C / (2 * 0.3e-3)  # all |kx| <= pi/pitch propagate above this
    bins = [k for k in range(1, nt // 2) if k * fs / nt > fmin * 1.01][:3]
    g = oracle.Geometry(ne, nt, fs, C, 0.3e-3, 7, 2e-3, 1.3e-3, bins)
    F = oracle.fields(g, _rand_rf(ne, nt, 21), None)
    e = np.sum(np.abs(F) ** 2, axis=2)  # [bins][nz]
    assert np.max(np.abs(e - e[:, :1]) / e[:, :1]) < 1e-11


def pin_z0_identity():
    """At the array face (z = 0) with nx = n_elem the field is the apodized
    channel spectrum itself: p~_q(x_i, 0, w_k) = a_q[i] S[k][i]."""
    ne, nt = 16, 128
    rf = _rand_rf(ne, nt, 9)
    bins = [9, 17, 30]
    g = oracle.Geometry(ne, nt, 20e6, C, 0.3e-3, 2, 0.0, 1e-3, bins)
    a = oracle.pattern(ne, 3, 2)[1]
    F = oracle.fields(g, rf, a)
    S = oracle.time_dft(rf, bins)
    assert np.max(np.abs(F[:, 0, :] - a[None, :] * S)) < 1e-11 * np.max(np.abs(S))


def pin_linearity_complementary():
    """Fields are linear in the apodization: with a_1 + a_2 + a_3 = 1 the
    sub-aperture fields add up to the full-aperture field."""
    ne, nt = 16, 128
    rf = _rand_rf(ne, nt, 10)
    g = _geom(ne, nt, nz=3)
    A = oracle.pattern(ne, 3, 2)
    full = oracle.fields(g, rf, None)
    s = sum(oracle.fields(g, rf, A[q]) for q in range(3))
    assert np.max(np.abs(full - s)) < 1e-10 * np.max(np.abs(full))


# ------------------------------------------------------------------ NCC --
def pin_energy_identity():
    """sum_k |p1+p2+p3|^2 = A11 + A22 + A33 + 2 (C12 + C23 + C31)."""
    ne, nt = 16, 128
    g = _geom(ne, nt)
    out = oracle.as_tax(g, _rand_rf(ne, nt, 12), oracle.pattern(ne, 3, 2))
    acc = out["acc"]
    lhs = acc[6]
    rhs = acc[0] + acc[1] + acc[2] + 2 * (acc[3] + acc[4] + acc[5])
    assert np.max(np.abs(lhs - rhs)) < 1e-10 * np.max(lhs)
    assert np.allclose(out["image_as"], lhs, rtol=0, atol=0)


def pin_ncc_identical_fields():
    """Identical apertures give identical fields, so every NCC is 1 and rho_n = 1
    (Eq. 4, 10)."""
    ne, nt = 16, 128
    g = _geom(ne, nt)
    A = np.ones((3, ne))
    out = oracle.as_tax(g, _rand_rf(ne, nt, 13), A)
    assert np.max(np.abs(out["rho_pairs"] - 1.0)) < 1e-12
    assert np.max(np.abs(out["rho_n"] - 1.0)) < 1e-12


def pin_ncc_bounds_and_max():
    """Cauchy-Schwarz: C_qr^2 <= A_qq A_rr, so rho lies in [-1, 1] before the
    clamp and in [eps, 1] after. The maximum of rho_n is exactly 1. Images are
    non-negative."""
    ne, nt = 16, 128
    g = _geom(ne, nt)
    out = oracle.as_tax(g, _rand_rf(ne, nt, 14), oracle.pattern(ne, 3, 2))
    acc = out["acc"]
    for (c, a, b) in ((3, 0, 1), (4, 1, 2), (5, 2, 0)):
        assert np.all(acc[c] ** 2 <= acc[a] * acc[b] * (1 + 1e-12))
    rp = out["rho_pairs"]
    assert rp.min() >= EPS and rp.max() <= 1.0 + 1e-12
    assert out["rho_n"].max() == 1.0
    assert out["rho_n"].min() > 0 and out["image"].min() >= 0


def pin_clamp_each_pair():
    """With a_2 = -a_1 and a_3 = a_1, rho_12 = rho_23 = -1 and rho_31 = 1.
    Clamping each pair at eps (Sec. II-A) gives (eps, eps, 1)."""
    ne, nt = 16, 128
    g = _geom(ne, nt)
    a = oracle.pattern(ne, 2, 2)[0]
    A = np.stack([a, -a, a])
    out = oracle.as_tax(g, _rand_rf(ne, nt, 15), A)
    rp = out["rho_pairs"]
    assert np.max(np.abs(rp[0] - EPS)) < 1e-15 and np.max(np.abs(rp[1] - EPS)) < 1e-15
    assert np.max(np.abs(rp[2] - 1.0)) < 1e-12


def pin_tax_cube_root_vs_dax():
    """An empty third aperture has A33 = 0, so rho_23 = rho_31 = eps. Eq. 10
    then gives rho_TAX = cbrt(rho_12 eps^2), and after normalisation
    rho_n(TAX) = cbrt(rho_n(DAX)) for the same first two apertures."""
    ne, nt = 16, 128
    g = _geom(ne, nt)
    rf = _rand_rf(ne, nt, 16)
    P = oracle.pattern(ne, 2, 2)
    tax = oracle.as_tax(g, rf, np.stack([P[0], P[1], np.zeros(ne)]))
    dax = oracle.as_xcorr(g, rf, P)
    assert np.max(np.abs(tax["rho_n"] - np.cbrt(dax["rho_n"]))) < 1e-12


def pin_appendix_a_time_domain_ncc():
    """Appendix A: with the negative frequencies completed as conjugates, the
    zero-lag time-domain NCC (Eq. 8 with zero means) of the band-limited
    fields equals the frequency-domain rho of Eq. 4."""
    ne, nt = 16, 128
    rf = _rand_rf(ne, nt, 17)
    bins = oracle.band_bins(nt, 20e6, 1e6, 8e6)
    g = _geom(ne, nt, nz=4, bins=bins)
    A = oracle.pattern(ne, 3, 2)
    out = oracle.as_tax(g, rf, A)
    f1 = oracle.fields(g, rf, A[0])
    f2 = oracle.fields(g, rf, A[1])
    checked = 0
    for j in range(g.nz):
        for i in range(g.nx):
            X = np.zeros(nt, complex)
            Y = np.zeros(nt, complex)
            X[bins] = f1[:, j, i]
            X[nt - bins] = np.conj(f1[:, j, i])
            Y[bins] = f2[:, j, i]
            Y[nt - bins] = np.conj(f2[:, j, i])
            x = np.fft.ifft(X)
            y = np.fft.ifft(Y)
            assert np.max(np.abs(x.imag)) < 1e-12 * np.max(np.abs(x.real))
            x, y = x.real - x.real.mean(), y.real - y.real.mean()
            rtd = float(x @ y / np.sqrt((x @ x) * (y @ y)))
            if rtd > 2 * EPS:
                assert abs(rtd - out["rho_pairs"][0, j, i]) < 1e-11, (j, i, rtd)
                checked += 1
    assert checked > 10


# ------------------------------------------------------------ point sources --
def as_point_source_rf(ne, nt, fs, pitch, bins, ix, zs):
    """Channel data whose array-plane angular spectrum is exactly that of a
    point at (x_ix, zs) under the paper's model. Every propagating kx carries
    exp(-i kx x_s) exp(-i kz zs), so Eq. 2 refocuses it at depth zs. Built
    directly from spectra: this is a test input, not the method."""
    u = np.arange(ne)
    up = np.where(2 * u >= ne, u - ne, u)
    kx = 2 * np.pi * up / (ne * pitch)
    S = np.zeros((len(bins), ne), complex)
    for b, k in enumerate(bins):
        kk = 2 * np.pi * (k * fs / nt) / C
        d = kk * kk - kx * kx
        prop = d > 0
        P = np.zeros(ne, complex)
        P[prop] = np.exp(-2j * np.pi * u[prop] * ix / ne) * np.exp(-1j * np.sqrt(d[prop]) * zs)
        S[b] = np.fft.ifft(P)          # element-domain spectrum at z = 0
    t = np.arange(nt)
    rf = np.zeros((ne, nt))
    for b, k in enumerate(bins):
        rf += (2.0 / nt) * np.real(S[b][:, None] * np.exp(2j * np.pi * k * t[None, :] / nt))
    return rf.astype(np.float32)


def pin_point_source_exact_pixel():
    """A source synthesised from the angular-spectrum model lands on its own
    pixel: both the AS energy (Eq. 3) and the AS-TAX image (Eq. 11) peak
    exactly at (x_s, z_s)."""
    ne, nt, fs, pitch = 32, 256, 20e6, 0.3e-3
    bins = oracle.band_bins(nt, fs, 2e6, 8e6)
    nz, z0, dz = 24, 4e-3, 0.5e-3
    for ix, jz in ((11, 13), (20, 6)):
        zs = z0 + jz * dz
        rf = as_point_source_rf(ne, nt, fs, pitch, bins, ix, zs)
        g = oracle.Geometry(ne, nt, fs, C, pitch, nz, z0, dz, bins)
        E = oracle.as_backprop(g, rf, None)
        assert np.unravel_index(np.argmax(E), E.shape) == (jz, ix)
        out = oracle.as_tax(g, rf, oracle.pattern(ne, 3, 2))
        assert np.unravel_index(np.argmax(out["image"]), E.shape) == (jz, ix)


def pin_green_sources_near_truth():
    """Green's-function channel data (delay r/c, 1/r spreading, 20 dB SNR) of
    the 64-element workload: the brightest AS-TAX pixel lies within 1 column
    and 2 rows of a true source, and so does the brightest AS pixel."""
    w = synth.workload(1)
    rf, src = synth.make_frame(w, 0)
    g = oracle.Geometry(w.n_elem, w.nt, w.fs, w.c, w.pitch, w.nz, w.z0, w.dz, w.bins())
    out = oracle.as_tax(g, rf, oracle.pattern(w.n_elem, 3, w.pattern_m))
    for key in ("image", "image_as"):
        jz, ix = np.unravel_index(np.argmax(out[key]), out[key].shape)
        assert any(abs(ix - s.ix) <= 1 and abs(jz - s.iz) <= 2 for s in src), (key, jz, ix, src)


# ---------------------------------------------------------- brute force --
def numpy_as_xcorr(rf, fs, pitch, nz, z0, dz, bins, A, eps=EPS, pad=1, evz=False):
    """Independent tiny-case implementation with numpy's FFT routines. With
    pad = 2 the lateral transforms use numpy's zero padding to 2 n_elem points
    (``fft(..., n=2 ne)``) and the fields are cropped to the n_elem element
    columns before the sums. With evz the propagator of every component whose
    kz is imaginary is zero."""
    ne, nt = rf.shape
    nf = pad * ne
    S = np.fft.rfft(rf.astype(np.float64), axis=1)[:, bins].T         # [nb][ne]
    kx = 2 * np.pi * np.fft.fftfreq(nf, d=pitch)
    k = 2 * np.pi * (np.asarray(bins) * fs / nt) / C
    kz = np.sqrt((k[:, None] ** 2 - kx[None, :] ** 2).astype(complex))  # principal branch
    z = z0 + np.arange(nz) * dz
    ph = np.exp(1j * kz[:, None, :] * z[None, :, None])                # [nb][nz][nf]
    if evz:
        ph = np.where(np.imag(kz)[:, None, :] > 0, 0.0, ph)
    p = [np.fft.ifft(np.fft.fft(a[None, :] * S, n=nf, axis=1)[:, None, :] * ph, axis=2)[..., :ne] for a in A]
    Aq = [np.sum(np.abs(x) ** 2, axis=0) for x in p]
    pairs = [(0, 1), (1, 2), (2, 0)] if len(A) == 3 else [(0, 1)]
    rho = []
    for q, r in pairs:
        cqr = np.sum(np.real(np.conj(p[q]) * p[r]), axis=0)
        rr = cqr / np.sqrt(Aq[q] * Aq[r])
        rho.append(np.maximum(rr, eps))
    rt = np.cbrt(rho[0] * rho[1] * rho[2]) if len(A) == 3 else rho[0]
    rn = rt / rt.max()
    E = np.sum(np.abs(sum(p)) ** 2, axis=0)
    return dict(image=rn ** 2 * E, rho_n=rn, rho_pairs=np.stack(rho), image_as=E)


def pin_numpy_brute_force():
    """The whole AS-TAX and AS-DAX chain against an independent numpy
    implementation on a tiny case."""
    ne, nt, fs, pitch = 16, 128, 20e6, 0.3e-3
    rf = _rand_rf(ne, nt, 19)
    bins = oracle.band_bins(nt, fs, 1e6, 8e6)
    nz, z0, dz = 5, 2e-3, 0.8e-3
    g = oracle.Geometry(ne, nt, fs, C, pitch, nz, z0, dz, bins)
    for na in (3, 2):
        A = oracle.pattern(ne, na, 2)
        got = oracle.as_xcorr(g, rf, A)
        want = numpy_as_xcorr(rf, fs, pitch, nz, z0, dz, bins, A)
        for key in ("image", "rho_n", "rho_pairs", "image_as"):
            err = np.max(np.abs(got[key] - want[key])) / np.max(np.abs(want[key]))
            assert err < 1e-10, (na, key, err)


def pin_numpy_brute_force_evanescent_zero():
    """AS-TAX and plain AS with evanescent components dropped, against the
    numpy implementation with the imaginary-kz propagators set to zero. The
    band starts at 0.5 MHz, where most lateral components are evanescent, so
    the result differs clearly from the principal-branch reading."""
    ne, nt, fs, pitch = 16, 128, 20e6, 0.3e-3
    rf = _rand_rf(ne, nt, 29)
    bins = oracle.band_bins(nt, fs, 0.5e6, 8e6)
    nz, z0, dz = 5, 0.2e-3, 0.3e-3
    g = oracle.Geometry(ne, nt, fs, C, pitch, nz, z0, dz, bins, evanescent_zero=True)
    A = oracle.pattern(ne, 3, 2)
    got = oracle.as_xcorr(g, rf, A)
    want = numpy_as_xcorr(rf, fs, pitch, nz, z0, dz, bins, A, evz=True)
    for key in ("image", "rho_n", "rho_pairs", "image_as"):
        err = np.max(np.abs(got[key] - want[key])) / np.max(np.abs(want[key]))
        assert err < 1e-10, (key, err)
    keep = numpy_as_xcorr(rf, fs, pitch, nz, z0, dz, bins, A, evz=False)
    assert np.max(np.abs(keep["image_as"] - want["image_as"])) > 1e-3 * np.max(want["image_as"])
    e = oracle.as_backprop(g, rf)
    assert np.max(np.abs(e - want["image_as"])) < 1e-10 * np.max(want["image_as"])


def pin_pad2x_numpy_brute_force():
    """2x lateral padding (Sec. II-D): AS-TAX and AS-DAX of the padded,
    cropped oracle against numpy's zero-padded FFTs on a tiny case."""
    ne, nt, fs, pitch = 16, 128, 20e6, 0.3e-3
    rf = _rand_rf(ne, nt, 23)
    bins = oracle.band_bins(nt, fs, 1e6, 8e6)
    nz, z0, dz = 5, 2e-3, 0.8e-3
    g = oracle.Geometry(ne, nt, fs, C, pitch, nz, z0, dz, bins)
    for na in (3, 2):
        A = oracle.pattern(ne, na, 2)
        got = oracle.as_xcorr_pad2x(g, rf, A)
        want = numpy_as_xcorr(rf, fs, pitch, nz, z0, dz, bins, A, pad=2)
        for key in ("image", "rho_n", "rho_pairs", "image_as"):
            assert got[key].shape == want[key].shape, key
            err = np.max(np.abs(got[key] - want[key])) / np.max(np.abs(want[key]))
            assert err < 1e-10, (na, key, err)
        assert got["rho_n"].max() == 1.0


def pin_pad2x_z0_and_effect():
    """At the array face the padded, cropped energy is the channel power of
    each element, sum_k |S[k][i]|^2 (so the crop keeps the element columns).
    At depth the padding changes the map: the wrap-around of the n_elem-point
    transforms is gone."""
    ne, nt = 16, 128
    rf = _rand_rf(ne, nt, 24)
    bins = [9, 17, 30]
    g0 = oracle.Geometry(ne, nt, 20e6, C, 0.3e-3, 1, 0.0, 1e-3, bins)
    e0 = oracle.as_backprop_pad2x(g0, rf)[0]
    S = np.fft.rfft(rf.astype(np.float64), axis=1)[:, bins]
    want = np.sum(np.abs(S) ** 2, axis=1)
    assert np.max(np.abs(e0 - want)) < 1e-11 * want.max()
    g = _geom(ne, nt, nz=4, z0=6e-3)
    ep, eu = oracle.as_backprop_pad2x(g, rf), oracle.as_backprop(g, rf)
    assert ep.shape == eu.shape
    assert np.max(np.abs(ep - eu)) > 1e-2 * eu.max()


def pin_band_bins_of_workloads():
    """Omega of the two workloads: 1-7 MHz at 20 MHz / 1024 samples is bins
    52..358 (307 bins); 0.5-8 MHz at 40 MHz / 4096 is bins 52..819 (768 bins)."""
    b1 = oracle.band_bins(1024, 20e6, 1e6, 7e6)
    assert b1[0] == 52 and b1[-1] == 358 and b1.size == 307
    b2 = oracle.band_bins(4096, 40e6, 0.5e6, 8e6)
    assert b2[0] == 52 and b2[-1] == 819 and b2.size == 768
    assert np.array_equal(synth.workload(1).bins(), b1)
    w2 = synth.workload(2).bins()
    assert w2.size == 300 and w2[0] == 52 and w2[-1] == 819 and np.all(np.diff(w2) > 0)
    assert set(w2.tolist()) <= set(b2.tolist())


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_") and callable(v)]
