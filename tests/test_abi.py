"""The C ABI without a GPU: libpam builds, loads, exports every symbol that
include/pam.h declares, and rejects bad descriptors before it touches a
device. These tests make no compute call."""
import ctypes
import os
import re

import pytest

from paper_2412_02413_gb300 import build as pam_build
from paper_2412_02413_gb300 import pam

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pam.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pam_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    pam_build.build()
    return pam.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("pam_plan_create", "pam_as_backprop", "pam_as_tax", "pam_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    assert set(pam._SIGS) == set(declared_functions())


def test_status_strings(lib):
    assert lib.pam_status_string(0) == b"PAM_OK"
    assert lib.pam_status_string(1) == b"PAM_ERR_INVALID_ARG"
    assert lib.pam_status_string(5) == b"PAM_ERR_TIMEOUT"


def _desc(lib, **kw):
    d = pam.PlanDesc()
    lib.pam_plan_desc_init(ctypes.byref(d))
    d.n_elem, d.pitch_m, d.fs_hz, d.c_mps = 64, 0.3e-3, 20e6, 1540.0
    d.n_samples, d.nz, d.z0_m, d.dz_m = 1024, 128, 10e-3, 0.3e-3
    d.f_lo_hz, d.f_hi_hz = 1e6, 7e6
    d.pattern_m = 8
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def _create(lib, d):
    h = ctypes.c_void_p(123)
    s = lib.pam_plan_create(ctypes.byref(d), ctypes.byref(h))
    return s, h


def test_desc_defaults(lib):
    d = pam.PlanDesc()
    lib.pam_plan_desc_init(ctypes.byref(d))
    assert d.n_apod == 3 and d.pattern_m == 16 and abs(d.eps - 1e-3) < 1e-9 and d.max_frames == 1


@pytest.mark.parametrize("field,value,status", [
    ("n_elem", 4, 1), ("n_elem", 300, 1), ("pitch_m", 0.0, 1), ("fs_hz", -1.0, 1),
    ("c_mps", float("nan"), 1), ("n_samples", 1000, 2), ("n_samples", 32, 1), ("n_samples", 16384, 2),
    ("nz", 0, 1), ("z0_m", -1e-3, 1), ("dz_m", 0.0, 1), ("n_apod", 4, 1), ("eps", 0.0, 1),
    ("eps", 1.5, 1), ("max_frames", 0, 1), ("flags", 0x100, 1), ("flags", 0x30, 1), ("flags", 0x10, 2),
    ("nx", 128, 2), ("pattern_m", 0, 1),
    ("flags", 0x12, 2),                           # zero-stuffing runs on the plain FP32 path only
    ("flags", 0x82, 2),
    ("f_lo_hz", 9e6, 1),
])
def test_bad_descriptor_is_rejected(lib, field, value, status):
    d = _desc(lib, **{field: value})
    s, h = _create(lib, d)
    assert s == status, (field, value, s, lib.pam_last_error())
    assert h.value is None
    assert lib.pam_last_error()


def test_bad_explicit_bins(lib):
    for bins in ([0, 5], [5, 5], [9, 4], [10, 512]):
        arr = (ctypes.c_int * len(bins))(*bins)
        d = _desc(lib, bins=ctypes.cast(arr, ctypes.POINTER(ctypes.c_int)), n_bins=len(bins))
        s, h = _create(lib, d)
        assert s == 1, bins


def test_non_finite_apodization(lib):
    w = (ctypes.c_float * (3 * 64))(*([1.0] * 191 + [float("inf")]))
    d = _desc(lib, apod=ctypes.cast(w, ctypes.POINTER(ctypes.c_float)))
    s, _ = _create(lib, d)
    assert s == 1


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.pam_plan_create(None, ctypes.byref(h)) == 1
    lib.pam_destroy(None)
    assert lib.pam_as_tax(None, None, 1, None, None, None, None, None) == 1
    assert lib.pam_as_backprop(None, None, 1, -1, None, None, None) == 1
    assert lib.pam_sync(None, None) == 1
    assert lib.pam_plan_bins(None, None) == 0


def _batch_desc(lib, **kw):
    return _desc(lib, **{"n_bins": 8, **kw})


def _frames(specs):
    arr = (pam.FrameDesc * max(1, len(specs)))()
    for i, (nt, nz) in enumerate(specs):
        arr[i].n_samples, arr[i].nz = nt, nz
    return arr


@pytest.mark.parametrize("kw,specs,status", [
    ({}, [], 1),                                  # no frames
    ({"n_apod": 1}, [(512, 16)], 1),              # batches are AS-DAX / AS-TAX
    ({"n_bins": 0}, [(512, 16)], 1),              # bins per frame are required
    ({"flags": 0x10}, [(512, 16)], 2),            # tensor-core forms are not batched
    ({}, [(512, 16), (31, 16)], 1),               # frame n_samples below 32
    ({}, [(512, 16), (20000, 16)], 1),            # frame n_samples above 16384
    ({}, [(512, 0)], 1),                          # frame with no depth rows
    ({"f_lo_hz": 5.01e6, "f_hi_hz": 5.02e6}, [(512, 16)], 1),   # band holds no bin
])
def test_bad_batch_is_rejected(lib, kw, specs, status):
    d = _batch_desc(lib, **kw)
    fr = _frames(specs)
    h = ctypes.c_void_p(123)
    s = lib.pam_batch_create(ctypes.byref(d), fr, len(specs), ctypes.byref(h))
    assert s == status, (kw, specs, s, lib.pam_last_error())
    assert h.value is None


def test_batch_rejects_common_bins(lib):
    arr = (ctypes.c_int * 2)(3, 4)
    d = _batch_desc(lib, bins=ctypes.cast(arr, ctypes.POINTER(ctypes.c_int)))
    h = ctypes.c_void_p()
    assert lib.pam_batch_create(ctypes.byref(d), _frames([(512, 16)]), 1, ctypes.byref(h)) == 1


def test_batch_rejects_bad_frame_bins(lib):
    for bins in ([0, 5], [5, 5], [9, 4], [10, 256]):
        arr = (ctypes.c_int * len(bins))(*bins)
        d = _batch_desc(lib, n_bins=len(bins))
        fr = _frames([(512, 16)])
        fr[0].bins = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int))
        h = ctypes.c_void_p()
        assert lib.pam_batch_create(ctypes.byref(d), fr, 1, ctypes.byref(h)) == 1, bins


def test_batch_null_handles(lib):
    assert lib.pam_batch_as_tax(None, None, None, None, None) == 1
    assert lib.pam_batch_sync(None, None) == 1
    assert lib.pam_batch_configure(None, 1, 0) == 1
    assert lib.pam_batch_info(None, None, None, None) == 1
    assert lib.pam_batch_layout(None, None, None, None, None) == 1
    assert lib.pam_batch_bins(None, 0, None) == 0
    lib.pam_batch_destroy(None)


def test_zero_stuffing_needs_twice_the_lateral_length(lib):
    d = _desc(lib, flags=0x2, nx=64)              # 64 elements: nx must be 128
    s, _ = _create(lib, d)
    assert s == 2


def test_new_entry_points_validate_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.pam_learn_n_params() == 29505
    assert lib.pam_learn_state_size() == 3 * 29505
    assert lib.pam_learn_create(None, ctypes.byref(h)) == 1
    d = _desc(lib, n_apod=2)
    assert lib.pam_learn_create(ctypes.byref(d), ctypes.byref(h)) == 1 and not h.value   # the TAX weight needs 3
    d = _desc(lib, flags=0x10)
    assert lib.pam_learn_create(ctypes.byref(d), ctypes.byref(h)) == 2 and not h.value   # plain path only
    lib.pam_learn_destroy(None)
    assert lib.pam_learn_set_params(None, None, 0) == 1
    assert lib.pam_learn_get_params(None, None, 0) == 1
    assert lib.pam_learn_get_state(None, None, 0, None) == 1
    assert lib.pam_learn_set_state(None, None, 0, 0) == 1
    assert lib.pam_learn_configure(None, 0.1, 0) == 1
    assert lib.pam_learn_feature_bytes(None) == 0
    assert lib.pam_learn_tax(None, None, 1, None, None, None, None, None) == 1
    assert lib.pam_learn_info(None, None, None, None) == 1
    assert lib.pam_as3(None, None, 1, None, None) == 1
    assert lib.pam_debug_expire_wait(None, None) == 1
    assert lib.pam_as_xcorr_host_async(None, None, 1, None, None, None) == 1
    assert lib.pam_image_metrics(None, 1, 8, 8, 0.0, 1.0, 0.0, 1.0, 0.7, None, None) == 1
    assert lib.pam_image_metrics(None, 1, 8, 8, 0.0, 1.0, 0.0, 1.0, 1.5, None, None) == 1   # alpha in (0, 1)
    assert lib.pam_image_metrics(None, 0, 8, 8, 0.0, 1.0, 0.0, 1.0, 0.7, None, None) == 0   # no frames: nothing to do
