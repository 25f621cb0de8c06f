"""The synthetic input recipe (no GPU): workload shapes, seeded determinism,
sources snapped to pixels inside the stated depth range, and the 20 dB channel
SNR, measured against the same frame without noise."""
import dataclasses

import numpy as np
import pytest

from paper_2412_02413_gb300 import synth


@pytest.mark.parametrize("wid,ne,nt,fs,nz,zr,srcs", [
    (1, 64, 1024, 20e6, 128, (10e-3, 50e-3), (2, 2)),
    (2, 128, 4096, 40e6, 512, (10e-3, 55e-3), (1, 6)),
])
def test_workload_and_frames(wid, ne, nt, fs, nz, zr, srcs):
    w = synth.workload(wid)
    assert (w.n_elem, w.nt, w.fs, w.nz, w.nx, w.pitch, w.c) == (ne, nt, fs, nz, ne, 0.3e-3, 1540.0)
    a, s_a = synth.make_frame(w, 3)
    b, _ = synth.make_frame(w, 3)
    c, _ = synth.make_frame(w, 4)
    assert a.dtype == np.float32 and a.shape == (ne, nt)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    for f in range(6):
        _, src = synth.make_frame(w, f)
        assert srcs[0] <= len(src) <= srcs[1]
        for s in src:
            assert s.x == w.pixel_x()[s.ix] and s.z == w.pixel_z()[s.iz]
            assert zr[0] - 1e-9 <= s.z <= zr[1] + 1e-9
            assert s.kind in ("stable", "inertial")


@pytest.mark.parametrize("wid", [1, 2])
def test_channel_snr_is_20_db(wid):
    w = synth.workload(wid)
    noisy, _ = synth.make_frame(w, 5)
    clean, _ = synth.make_frame(dataclasses.replace(w, snr_db=None), 5)
    noise = noisy.astype(np.float64) - clean
    snr = 10 * np.log10(np.mean(clean.astype(np.float64) ** 2) / np.mean(noise ** 2))
    assert abs(snr - 20.0) < 0.1, snr
