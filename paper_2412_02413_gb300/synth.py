"""Seeded synthetic channel data for passive acoustic mapping workloads.

This module generates inputs only. It holds none of the mapping method's
arithmetic: no angular spectrum, propagator or correlation. It simulates
cavitation sources and a linear receive array as a forward physical model:

* each source emits a time signal q(t);
* element e receives q(t - r_e/c) * r_ref/r_e (Green's function delay and 1/r
  spreading), with r_e measured in the imaging plane;
* white Gaussian noise is added at a set channel SNR.

The paper's own phantom and in-vivo recordings are not available, so these
frames stand in for them. They use the paper's workload shapes: a linear
array, sources at 10-60 mm depth, harmonic, ultra-harmonic and broadband
emissions (Sec. II-D), and channel-major float32 RF.

Seeds: the sources of frame f in workload w use 20241203 + 1000*w + f, and
the channel noise uses that seed plus 1.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

SEED_BASE = 20241203


@dataclasses.dataclass
class Workload:
    """Geometry, band and bin list of one synthetic workload."""
    name: str
    n_elem: int
    pitch: float          # m
    fs: float             # Hz
    nt: int               # samples per channel
    c: float              # m/s
    nz: int               # depth rows
    z_first: float        # m, first row (from the array face)
    z_last: float         # m, last row
    f_lo: float           # Hz
    f_hi: float           # Hz
    n_bins: Optional[int]  # None: every bin in the band; else evenly spaced subset
    pattern_m: int        # Pattern-m of the complementary apodizations
    n_apod: int = 3
    n_sources: tuple = (2, 2)       # inclusive range of the seeded source count
    snr_db: float = 20.0
    source_z: tuple = (10e-3, 50e-3)
    harmonic_f0: tuple = (1.5e6,)
    broadband_level: float = 0.1    # broadband amplitude relative to the harmonic one
    workload_id: int = 0

    @property
    def nx(self) -> int:
        return self.n_elem

    @property
    def dz(self) -> float:
        return (self.z_last - self.z_first) / (self.nz - 1) if self.nz > 1 else 1e-4

    @property
    def z0(self) -> float:
        return self.z_first

    def bins(self) -> np.ndarray:
        """Omega: DFT bin indices k (0 < k < nt/2) inside [f_lo, f_hi]; when
        n_bins is set, n_bins of them spread evenly from the first to the last."""
        df = self.fs / self.nt
        k_lo = max(1, int(np.ceil(self.f_lo / df - 1e-9)))
        k_hi = min(self.nt // 2 - 1, int(np.floor(self.f_hi / df + 1e-9)))
        allk = np.arange(k_lo, k_hi + 1, dtype=np.int64)
        if self.n_bins is None or self.n_bins >= allk.size:
            return allk.astype(np.int32)
        K = allk.size
        n = self.n_bins
        if n == 1:
            return allk[:1].astype(np.int32)
        # floor(i (K-1)/(n-1) + 1/2) in integers (the rule libpam's batches use)
        idx = (2 * np.arange(n, dtype=np.int64) * (K - 1) + (n - 1)) // (2 * (n - 1))
        return allk[idx].astype(np.int32)

    def pixel_x(self) -> np.ndarray:
        return (np.arange(self.n_elem) - (self.n_elem - 1) / 2.0) * self.pitch

    def pixel_z(self) -> np.ndarray:
        return self.z0 + np.arange(self.nz) * self.dz


def workload(wid: int) -> Workload:
    """Workload 1: 64-element array, 1024 samples at 20 MHz, 64 x 128 grid,
    band 1-7 MHz (all 307 bins), Pattern-8, 2 sources.
    Workload 2: 128-element array, 4096 samples at 40 MHz, 128 x 512 grid over
    5-60 mm, 300 bins spread over 0.5-8 MHz, Pattern-16, 1-6 sources."""
    if wid == 1:
        return Workload(name="astax_64el_64x128_307bins", n_elem=64, pitch=0.3e-3, fs=20e6, nt=1024,
                        c=1540.0, nz=128, z_first=10e-3, z_last=50e-3, f_lo=1e6, f_hi=7e6,
                        n_bins=None, pattern_m=8, n_sources=(2, 2), snr_db=20.0,
                        source_z=(10e-3, 50e-3), harmonic_f0=(1.5e6,), workload_id=1)
    if wid == 2:
        return Workload(name="astax_128el_128x512_300bins", n_elem=128, pitch=0.3e-3, fs=40e6, nt=4096,
                        c=1540.0, nz=512, z_first=5e-3, z_last=60e-3, f_lo=0.5e6, f_hi=8e6,
                        n_bins=300, pattern_m=16, n_sources=(1, 6), snr_db=20.0,
                        source_z=(10e-3, 55e-3), harmonic_f0=(1.0e6, 1.5e6), workload_id=2)
    raise ValueError(f"unknown workload {wid}")


BATCH_DZ = 55e-3 / 511      # the 0.1076 mm depth step of the 128 x 512 workload


def batch_workload(n_frames: int = 256, seed_offset: int = 0) -> List[Workload]:
    """Workload 3 (uneven batch): frames of a 128-element array at 40 MHz.
    Each frame draws its sample count uniformly in [1024, 8192] (not a power
    of 2 in general) and its depth rows uniformly in [128, 512] from 5 mm at
    0.1076 mm, 1-8 sources, and uses 300 bins spread over 0.5-8 MHz at its own
    bin spacing fs / nt. Frame f's sources use seed 20241203 + 3000 + f."""
    rng = np.random.default_rng(SEED_BASE + 3000 + 999_983 + seed_offset)
    out = []
    for f in range(n_frames):
        nt = int(rng.integers(1024, 8193))
        nz = int(rng.integers(128, 513))
        z_last = 5e-3 + (nz - 1) * BATCH_DZ
        out.append(Workload(name=f"batch_frame{f}", n_elem=128, pitch=0.3e-3, fs=40e6, nt=nt, c=1540.0, nz=nz,
                            z_first=5e-3, z_last=z_last, f_lo=0.5e6, f_hi=8e6, n_bins=300, pattern_m=16,
                            n_sources=(1, 8), snr_db=20.0, source_z=(10e-3, min(55e-3, z_last)),
                            harmonic_f0=(1.0e6, 1.5e6), workload_id=3))
    return out


def tiny_workload(n_elem=16, nt=128, nz=8, n_bins=None, fs=20e6, pattern_m=2) -> Workload:
    """Small grids for brute-force checks (a few ms of oracle time)."""
    return Workload(name=f"tiny_{n_elem}el_{nt}t_{nz}z", n_elem=n_elem, pitch=0.3e-3, fs=fs, nt=nt,
                    c=1540.0, nz=nz, z_first=4e-3, z_last=4e-3 + (nz - 1) * 0.5e-3,
                    f_lo=1e6, f_hi=8e6, n_bins=n_bins, pattern_m=pattern_m, n_sources=(1, 2),
                    source_z=(5e-3, 4e-3 + (nz - 1) * 0.5e-3), harmonic_f0=(1.5e6,), workload_id=0)


@dataclasses.dataclass
class Source:
    x: float
    z: float
    kind: str            # "stable" (harmonic series) or "inertial" (broadband)
    f0: float
    amplitude: float
    ix: int              # pixel column the source sits on
    iz: int              # pixel row the source sits on


def _bandlimited_noise(rng, n, fs, f_lo, f_hi):
    """Periodic Gaussian noise of length n, band-limited to [f_lo, f_hi]."""
    spec = rng.standard_normal(n // 2 + 1) + 1j * rng.standard_normal(n // 2 + 1)
    f = np.fft.rfftfreq(n, 1.0 / fs)
    spec[(f < f_lo) | (f > f_hi)] = 0.0
    x = np.fft.irfft(spec, n)
    s = np.std(x)
    return x / s if s > 0 else x


def make_sources(w: Workload, seed: int) -> List[Source]:
    rng = np.random.default_rng(seed)
    lo, hi = w.n_sources
    n = int(rng.integers(lo, hi + 1))
    xs = w.pixel_x()
    zs = w.pixel_z()
    margin = max(2, w.n_elem // 16)
    out = []
    for s in range(n):
        ix = int(rng.integers(margin, w.n_elem - margin))
        jz_lo = int(np.searchsorted(zs, w.source_z[0]))
        jz_hi = max(jz_lo, int(np.searchsorted(zs, w.source_z[1], side="right")) - 1)
        iz = int(rng.integers(jz_lo, jz_hi + 1))
        kind = "stable" if (s % 2 == 0) else "inertial"
        f0 = float(w.harmonic_f0[int(rng.integers(0, len(w.harmonic_f0)))])
        amp = float(rng.uniform(0.5, 1.0))
        out.append(Source(x=float(xs[ix]), z=float(zs[iz]), kind=kind, f0=f0, amplitude=amp, ix=ix, iz=iz))
    return out


def source_signal_spectrum(src: Source, w: Workload, rng, n: int):
    """Harmonic part as (freqs, amps, phases) and a periodic broadband part of
    length n, both for source ``src``."""
    nyq = w.fs / 2
    freqs, amps, phases = [], [], []
    if src.kind == "stable":
        h = 1
        while h * src.f0 < min(nyq, w.f_hi * 1.05):
            freqs.append(h * src.f0)
            amps.append(src.amplitude / h ** 0.5)
            phases.append(rng.uniform(0, 2 * np.pi))
            # ultra-harmonic between consecutive harmonics
            fu = (h + 0.5) * src.f0
            if fu < min(nyq, w.f_hi * 1.05):
                freqs.append(fu)
                amps.append(0.3 * src.amplitude / h ** 0.5)
                phases.append(rng.uniform(0, 2 * np.pi))
            h += 1
        bb = w.broadband_level * src.amplitude
    else:
        bb = src.amplitude
    noise = _bandlimited_noise(rng, n, w.fs, max(w.f_lo * 0.8, 1.0), min(w.f_hi * 1.05, nyq)) * bb
    return np.array(freqs), np.array(amps), np.array(phases), noise


def _propagated_sources(w: Workload, sources: List[Source], rng):
    """Harmonic part of the channel signals [n_elem][nt] (analytic delays) and
    the summed, delayed spectra of the broadband parts [n_elem][nt + 1] on a
    periodic record of 2*nt samples (exact fractional delays)."""
    ne, nt = w.n_elem, w.nt
    t = np.arange(nt) / w.fs
    xe = w.pixel_x()
    rf = np.zeros((ne, nt), dtype=np.float64)
    L = 2 * nt
    fL = np.fft.rfftfreq(L, 1.0 / w.fs)
    spec = np.zeros((ne, fL.size), dtype=np.complex128)   # summed delayed broadband spectra
    for src in sources:
        freqs, amps, phases, noise = source_signal_spectrum(src, w, rng, L)
        r = np.sqrt((xe - src.x) ** 2 + src.z ** 2)
        tau = r / w.c
        gain = 10e-3 / r
        if freqs.size:
            # sin(2 pi f (t - tau_e) + phi) = cos(phi_e) sin(2 pi f t) + sin(phi_e) cos(2 pi f t)
            phi_e = phases[None, :] - 2 * np.pi * freqs[None, :] * tau[:, None]        # [ne][H]
            wt = 2 * np.pi * np.outer(freqs, t)                                         # [H][nt]
            rf += gain[:, None] * ((np.cos(phi_e) * amps) @ np.sin(wt) + (np.sin(phi_e) * amps) @ np.cos(wt))
        nspec = np.fft.rfft(noise)
        band = np.nonzero(nspec)[0]
        spec[:, band] += (gain[:, None] * nspec[band][None, :]) * np.exp(-2j * np.pi * fL[band][None, :] * tau[:, None])
    return rf, spec


def source_response(w: Workload, src: Source, seed: int) -> np.ndarray:
    """Noise-free channel signals [n_elem][nt] (float32) of one source alone.
    The receive model is linear in the sources, so a frame of several sources
    is the sum of their responses plus channel noise."""
    rf, spec = _propagated_sources(w, [src], np.random.default_rng(seed))
    rf += np.fft.irfft(spec, 2 * w.nt, axis=1)[:, :w.nt]
    return rf.astype(np.float32)


def bank_sources(w: Workload, n: int, seed: int) -> List[Source]:
    """n single sources on seeded pixels of the workload's grid (kinds
    alternate stable / inertial), as make_sources draws them."""
    one = dataclasses.replace(w, n_sources=(1, 1))
    out = []
    for i in range(n):
        src = make_sources(one, seed + i)[0]
        if i % 2:
            src = dataclasses.replace(src, kind="inertial")
        out.append(src)
    return out


def make_frame(w: Workload, frame: int = 0, sources: Optional[List[Source]] = None):
    """One frame of channel-major float32 RF [n_elem][nt] plus its sources.

    The harmonic emission delays are analytic. The broadband emission is
    periodic over a record of 2*nt samples and delayed exactly in the
    frequency domain. Amplitude falls off as 10 mm / r."""
    seed = SEED_BASE + 1000 * w.workload_id + frame
    if sources is None:
        sources = make_sources(w, seed)
    rng = np.random.default_rng(seed + 7)
    rf, spec = _propagated_sources(w, sources, rng)
    rf += np.fft.irfft(spec, 2 * w.nt, axis=1)[:, :w.nt]
    p = float(np.mean(rf ** 2))
    nrng = np.random.default_rng(seed + 1)
    if w.snr_db is not None and p > 0:
        sigma = np.sqrt(p / 10 ** (w.snr_db / 10))
        rf += nrng.standard_normal(rf.shape) * sigma
    return rf.astype(np.float32), sources


def make_batch(w: Workload, n_frames: int, first_frame: int = 0) -> np.ndarray:
    """[n_frames][n_elem][nt] float32."""
    out = np.empty((n_frames, w.n_elem, w.nt), dtype=np.float32)
    for f in range(n_frames):
        out[f], _ = make_frame(w, first_frame + f)
    return out


def random_rf(n_elem: int, nt: int, seed: int, n_frames: Optional[int] = None) -> np.ndarray:
    """Gaussian white RF (edge cases, timing pools)."""
    rng = np.random.default_rng(seed)
    shape = (n_elem, nt) if n_frames is None else (n_frames, n_elem, nt)
    return rng.standard_normal(shape).astype(np.float32)
