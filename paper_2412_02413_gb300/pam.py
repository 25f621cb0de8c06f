"""Python binding of libpam (C ABI in ``include/pam.h``).

This module only marshals arguments. It passes tensor data pointers and the
current CUDA stream handle to the library, and every step of the
angular-spectrum path runs in the library's CUDA kernels. PyTorch is used for
device memory and streams only. There is no CPU fallback: when the library
or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

PAM_OK = 0
PAM_EVANESCENT_ZERO = 0x1
PAM_LATERAL_UPSAMPLE2X = 0x2
PAM_LATERAL_PAD2X = 0x4
# tensor-core forms of the propagation (include/pam.h PAM_FORM_GEMM_*)
FORMS = {"fp32": 0x0, "bf16": 0x10, "fp16": 0x20, "bf16split": 0x40, "fp16split": 0x80}
_STATUS = {0: "PAM_OK", 1: "PAM_ERR_INVALID_ARG", 2: "PAM_ERR_UNSUPPORTED", 3: "PAM_ERR_OOM",
           4: "PAM_ERR_CUDA", 5: "PAM_ERR_TIMEOUT", 6: "PAM_ERR_NUMERIC"}


class PamError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class PlanDesc(ctypes.Structure):
    """Mirror of ``pam_plan_desc``."""
    _fields_ = [
        ("n_elem", ctypes.c_int), ("pitch_m", ctypes.c_double), ("fs_hz", ctypes.c_double),
        ("c_mps", ctypes.c_double), ("n_samples", ctypes.c_int), ("nx", ctypes.c_int),
        ("nz", ctypes.c_int), ("z0_m", ctypes.c_double), ("dz_m", ctypes.c_double),
        ("f_lo_hz", ctypes.c_double), ("f_hi_hz", ctypes.c_double),
        ("bins", ctypes.POINTER(ctypes.c_int)), ("n_bins", ctypes.c_int),
        ("n_apod", ctypes.c_int), ("apod", ctypes.POINTER(ctypes.c_float)), ("pattern_m", ctypes.c_int),
        ("eps", ctypes.c_float), ("flags", ctypes.c_uint), ("max_frames", ctypes.c_int),
    ]


class FrameDesc(ctypes.Structure):
    """Mirror of ``pam_frame_desc``."""
    _fields_ = [("n_samples", ctypes.c_int), ("nz", ctypes.c_int), ("bins", ctypes.POINTER(ctypes.c_int))]


_lock = threading.Lock()
_lib = None

# Every symbol include/pam.h declares, with (restype, argtypes).
_VP = ctypes.c_void_p
_SIGS = {
    "pam_plan_desc_init": (None, [ctypes.POINTER(PlanDesc)]),
    "pam_plan_create": (ctypes.c_int, [ctypes.POINTER(PlanDesc), ctypes.POINTER(_VP)]),
    "pam_destroy": (None, [_VP]),
    "pam_plan_bins": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "pam_plan_apod": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "pam_plan_set_split": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pam_plan_set_grid": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pam_plan_set_fft_radix": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pam_plan_set_gemm_tile": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pam_plan_set_lane_rows": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pam_plan_set_gemm_frames": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pam_as_backprop": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP]),
    "pam_as_tax": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP]),
    "pam_as_dax": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP]),
    "pam_as_xcorr_host": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP]),
    "pam_as_xcorr_host_async": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP]),
    "pam_as_tax_static": (ctypes.c_int, [ctypes.POINTER(PlanDesc), _VP, ctypes.c_int, _VP, _VP, _VP]),
    "pam_sync": (ctypes.c_int, [_VP, _VP]),
    "pam_debug_expire_wait": (ctypes.c_int, [_VP, _VP]),
    "pam_profile_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pam_profile_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_longlong)]),
    "pam_batch_create": (ctypes.c_int, [ctypes.POINTER(PlanDesc), ctypes.POINTER(FrameDesc), ctypes.c_int,
                                        ctypes.POINTER(_VP)]),
    "pam_batch_layout": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                        ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "pam_batch_bins": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "pam_batch_as_tax": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "pam_batch_sync": (ctypes.c_int, [_VP, _VP]),
    "pam_batch_configure": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "pam_batch_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_longlong)]),
    "pam_batch_destroy": (None, [_VP]),
    "pam_as3": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP]),
    "pam_image_metrics": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_float, _VP, _VP]),
    "pam_learn_n_params": (ctypes.c_size_t, []),
    "pam_learn_create": (ctypes.c_int, [ctypes.POINTER(PlanDesc), ctypes.POINTER(_VP)]),
    "pam_learn_destroy": (None, [_VP]),
    "pam_learn_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
    "pam_learn_get_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
    "pam_learn_configure": (ctypes.c_int, [_VP, ctypes.c_float, ctypes.c_int]),
    "pam_learn_state_size": (ctypes.c_size_t, []),
    "pam_learn_get_state": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t,
                                           ctypes.POINTER(ctypes.c_longlong)]),
    "pam_learn_set_state": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t,
                                           ctypes.c_longlong]),
    "pam_learn_feature_bytes": (ctypes.c_size_t, [_VP]),
    "pam_learn_example": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "pam_learn_forward": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP]),
    "pam_learn_grads": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP]),
    "pam_learn_train_step": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_float, _VP, _VP]),
    "pam_learn_tax": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP]),
    "pam_learn_sync": (ctypes.c_int, [_VP, _VP]),
    "pam_learn_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_longlong)]),
    "pam_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pam_last_error": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Open libpam.so (building it first when absent or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libpam.so is missing at {path}; run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int):
    if status != PAM_OK:
        msg = load().pam_last_error().decode(errors="replace")
        raise PamError(status, msg)


def _require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libpam needs a CUDA GPU; no CPU fallback exists")
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _require_cuda()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _dptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def _make_desc(n_elem, pitch, fs, c, n_samples, nz, z0, dz, bins=None, f_lo=0.0, f_hi=0.0, n_apod=3, apod=None,
               pattern_m=16, eps=1e-3, evanescent_zero=False, max_frames=1, nx=0, form="fp32", upsample2x=False,
               pad2x=False):
    """A filled ``pam_plan_desc`` and the host arrays it points to (keep them alive)."""
    L = load()
    d = PlanDesc()
    L.pam_plan_desc_init(ctypes.byref(d))
    d.n_elem, d.pitch_m, d.fs_hz, d.c_mps = int(n_elem), float(pitch), float(fs), float(c)
    d.n_samples, d.nx, d.nz = int(n_samples), int(nx), int(nz)
    d.z0_m, d.dz_m, d.f_lo_hz, d.f_hi_hz = float(z0), float(dz), float(f_lo), float(f_hi)
    bins_keep = apod_keep = None
    if bins is not None:
        bins_keep = np.ascontiguousarray(np.asarray(bins, dtype=np.int32))
        d.bins = bins_keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        d.n_bins = int(bins_keep.size)
    d.n_apod = int(n_apod)
    if apod is not None:
        apod_keep = np.ascontiguousarray(np.asarray(apod, dtype=np.float32))
        d.apod = apod_keep.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    d.pattern_m, d.eps = int(pattern_m), float(eps)
    if form not in FORMS:
        raise ValueError(f"form must be one of {sorted(FORMS)}")
    d.flags = (PAM_EVANESCENT_ZERO if evanescent_zero else 0) | FORMS[form] | \
        (PAM_LATERAL_UPSAMPLE2X if upsample2x else 0) | (PAM_LATERAL_PAD2X if pad2x else 0)
    d.max_frames = int(max_frames)
    return d, bins_keep, apod_keep


class Plan:
    """An AS / AS-DAX / AS-TAX plan on the current CUDA device.

    Geometry is given in SI units. Either ``bins`` (explicit DFT bin indices)
    or the band ``(f_lo, f_hi)`` selects Omega. ``apod`` is [n_apod][n_elem]
    or None for Pattern-``pattern_m``. ``upsample2x`` and ``pad2x`` are the two
    2x lateral extensions of Sec. II-D: zero-stuffed channels at pitch/2 (the
    image is 2 n_elem wide), or n_elem zero channels appended (transforms over
    2 n_elem points, the image cropped to the n_elem element columns)."""

    def __init__(self, n_elem: int, pitch: float, fs: float, c: float, n_samples: int, nz: int,
                 z0: float, dz: float, bins: Optional[Sequence[int]] = None, f_lo: float = 0.0,
                 f_hi: float = 0.0, n_apod: int = 3, apod=None, pattern_m: int = 16, eps: float = 1e-3,
                 evanescent_zero: bool = False, max_frames: int = 1, nx: int = 0, form: str = "fp32",
                 upsample2x: bool = False, pad2x: bool = False):
        _require_cuda()
        L = load()
        d, self._bins_keep, self._apod_keep = _make_desc(
            n_elem, pitch, fs, c, n_samples, nz, z0, dz, bins, f_lo, f_hi, n_apod, apod, pattern_m, eps,
            evanescent_zero, max_frames, nx, form, upsample2x, pad2x)
        h = _VP()
        _check(L.pam_plan_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.n_elem, self.n_samples, self.nz, self.n_apod = int(n_elem), int(n_samples), int(nz), int(n_apod)
        self.nx = (2 if upsample2x else 1) * self.n_elem if not nx else int(nx)
        self.max_frames = int(max_frames)
        self.form = form
        self.bins = self._query_bins()
        self.apod = self._query_apod()

    @classmethod
    def from_workload(cls, w, n_apod: Optional[int] = None, max_frames: int = 1, **kw) -> "Plan":
        """Plan for a :class:`paper_2412_02413_gb300.synth.Workload`."""
        return cls(n_elem=w.n_elem, pitch=w.pitch, fs=w.fs, c=w.c, n_samples=w.nt, nz=w.nz, z0=w.z0,
                   dz=w.dz, bins=w.bins(), n_apod=w.n_apod if n_apod is None else n_apod,
                   pattern_m=w.pattern_m, max_frames=max_frames, **kw)

    def _query_bins(self) -> np.ndarray:
        L = load()
        n = L.pam_plan_bins(self._h, None)
        out = np.zeros(n, dtype=np.int32)
        L.pam_plan_bins(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return out

    def _query_apod(self) -> np.ndarray:
        L = load()
        out = np.zeros((self.n_apod, self.n_elem), dtype=np.float32)
        L.pam_plan_apod(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        return out

    @property
    def handle(self):
        return self._h

    @property
    def n_bins(self) -> int:
        return int(self.bins.size)

    def close(self):
        if getattr(self, "_h", None):
            load().pam_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------- calls --
    def _check_rf(self, rf):
        torch = _require_cuda()
        if not isinstance(rf, torch.Tensor) or not rf.is_cuda or rf.dtype != torch.float32:
            raise TypeError("rf must be a float32 CUDA tensor")
        if rf.dim() == 2:
            rf = rf.unsqueeze(0)
        if tuple(rf.shape[1:]) != (self.n_elem, self.n_samples):
            raise ValueError(f"rf must be [F][{self.n_elem}][{self.n_samples}], got {tuple(rf.shape)}")
        return rf.contiguous()

    def _empty(self, *shape):
        torch = _require_cuda()
        return torch.empty(shape, dtype=torch.float32, device="cuda")

    def as_backprop(self, rf, apod_index: int = -1, fields: bool = False, out=None, stream=None):
        """Eq. 3 energy map [F][nz][nx] (and the fields [F][n_bins][nz][nx] complex64 if asked)."""
        torch = _require_cuda()
        rf = self._check_rf(rf)
        F = rf.shape[0]
        energy = self._empty(F, self.nz, self.nx) if out is None else out
        fl = self._empty(F, self.n_bins, self.nz, self.nx, 2) if fields else None
        _check(load().pam_as_backprop(self._h, _dptr(rf), F, int(apod_index), _dptr(energy), _dptr(fl),
                                      _stream_ptr(stream)))
        if fields:
            return energy, torch.view_as_complex(fl)
        return energy

    def as_tax(self, rf, rho_n: bool = True, rho_pairs: bool = False, image_as: bool = False,
               outs: Optional[dict] = None, stream=None) -> dict:
        """AS-TAX (Eq. 10-11). Returns a dict of [F][nz][nx] maps (rho_pairs [F][3][nz][nx])."""
        if self.n_apod != 3:
            raise ValueError("as_tax needs a plan with three apodizations")
        return self._xcorr(load().pam_as_tax, 3, rf, rho_n, rho_pairs, image_as, outs, stream)

    def as_dax(self, rf, rho_n: bool = True, rho_pairs: bool = False, image_as: bool = False,
               outs: Optional[dict] = None, stream=None) -> dict:
        """AS-DAX (Eq. 4-5)."""
        if self.n_apod != 2:
            raise ValueError("as_dax needs a plan with two apodizations")
        return self._xcorr(load().pam_as_dax, 1, rf, rho_n, rho_pairs, image_as, outs, stream)

    def _xcorr(self, fn, npairs, rf, rho_n, rho_pairs, image_as, outs, stream):
        rf = self._check_rf(rf)
        F = rf.shape[0]
        o = dict(outs or {})
        if "image" not in o:
            o["image"] = self._empty(F, self.nz, self.nx)
        if rho_n and "rho_n" not in o:
            o["rho_n"] = self._empty(F, self.nz, self.nx)
        if rho_pairs and "rho_pairs" not in o:
            o["rho_pairs"] = self._empty(F, npairs, self.nz, self.nx)
        if image_as and "image_as" not in o:
            o["image_as"] = self._empty(F, self.nz, self.nx)
        _check(fn(self._h, _dptr(rf), F, _dptr(o["image"]), _dptr(o.get("rho_n")), _dptr(o.get("rho_pairs")),
                  _dptr(o.get("image_as")), _stream_ptr(stream)))
        return o

    def as3(self, rf, out=None, stream=None):
        """AS^3 image (Eq. 20) [F][nz][nx]."""
        rf = self._check_rf(rf)
        F = rf.shape[0]
        img = self._empty(F, self.nz, self.nx) if out is None else out
        _check(load().pam_as3(self._h, _dptr(rf), F, _dptr(img), _stream_ptr(stream)))
        return img

    def as_xcorr_host(self, rf_host: np.ndarray, image_out: np.ndarray, rho_n_out: Optional[np.ndarray] = None,
                      stream=None):
        """AS-TAX / AS-DAX from host memory through ``pam_as_xcorr_host``.
        ``rf_host`` [F][n_elem][n_samples] float32, outputs [F][nz][nx] float32
        (pinned buffers make the copies faster). Returns after the results are
        in the host arrays."""
        for a in (rf_host, image_out) + ((rho_n_out,) if rho_n_out is not None else ()):
            if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
                raise TypeError("host buffers must be C-contiguous float32")
        F = rf_host.shape[0] if rf_host.ndim == 3 else 1
        _check(load().pam_as_xcorr_host(self._h, rf_host.ctypes.data, F, image_out.ctypes.data,
                                        None if rho_n_out is None else rho_n_out.ctypes.data,
                                        _stream_ptr(stream)))

    def as_xcorr_host_async(self, rf_host: np.ndarray, image_out: np.ndarray,
                            rho_n_out: Optional[np.ndarray] = None, stream=None):
        """As :meth:`as_xcorr_host` through ``pam_as_xcorr_host_async``: returns
        once the work is queued on ``stream``; the results are in the host arrays
        when the stream gets there (keep the arrays alive until then)."""
        for a in (rf_host, image_out) + ((rho_n_out,) if rho_n_out is not None else ()):
            if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
                raise TypeError("host buffers must be C-contiguous float32")
        F = rf_host.shape[0] if rf_host.ndim == 3 else 1
        _check(load().pam_as_xcorr_host_async(self._h, rf_host.ctypes.data, F, image_out.ctypes.data,
                                              None if rho_n_out is None else rho_n_out.ctypes.data,
                                              _stream_ptr(stream)))

    def set_split(self, n_split: int = 0):
        """Bin chunks per row tile of the fused kernel (0 = automatic)."""
        _check(load().pam_plan_set_split(self._h, int(n_split)))

    def set_grid(self, n_ctas: int = 0):
        """CTAs of the fused kernel's even division (0 = one per SM)."""
        _check(load().pam_plan_set_grid(self._h, int(n_ctas)))

    def set_fft_radix(self, radix: int = 8):
        """Largest radix of the time FFT's stages (4 or 8)."""
        _check(load().pam_plan_set_fft_radix(self._h, int(radix)))

    def set_gemm_frames(self, frames: int = 32):
        """Frames per CTA of the tensor-core form (32 or 16; identical results)."""
        _check(load().pam_plan_set_gemm_frames(self._h, int(frames)))

    def set_lane_rows(self, rows: int = 2):
        """Depth rows per lane of the fused kernel (1 or 2; the maps agree to rounding)."""
        _check(load().pam_plan_set_lane_rows(self._h, int(rows)))

    def set_gemm_tile(self, m: int = 128):
        """M tile of the tensor-core form's MMAs: 128 (one CTA per row) or 256 (CTA pairs on two rows)."""
        _check(load().pam_plan_set_gemm_tile(self._h, int(m)))

    def profile_enable(self, on: bool = True):
        """Record CUDA events around each propagate-and-correlate launch."""
        _check(load().pam_profile_enable(self._h, int(bool(on))))

    def profile_read(self):
        """(summed prop-kernel ms, prop launches, all libpam kernel launches); clears them."""
        ms, n, k = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().pam_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(k)))
        return ms.value, n.value, k.value

    def debug_expire_wait(self, stream=None):
        """Launch the failure-path check kernel (``pam_debug_expire_wait``): the
        next :meth:`sync` raises PAM_ERR_TIMEOUT after about one second."""
        _check(load().pam_debug_expire_wait(self._h, _stream_ptr(stream)))

    def sync(self, stream=None):
        _check(load().pam_sync(self._h, _stream_ptr(stream)))


class Batch:
    """Frames with their own sample counts, depth ranges and bins, run in one
    call (``pam_batch_*``): a time DFT of the selected bins (any nt), the
    lateral FFTs, the persistent propagate-and-correlate kernel and the
    per-frame normalisation, replayed as a CUDA graph.

    ``frames`` is a list of ``(n_samples, nz)`` or ``(n_samples, nz, bins)``.
    Without explicit bins each frame takes ``n_bins`` of its band's bins spread
    evenly. Inputs and outputs are packed 1-D float32 tensors; ``rf_offsets``
    and ``map_offsets`` give each frame's start."""

    def __init__(self, n_elem: int, pitch: float, fs: float, c: float, frames, z0: float, dz: float,
                 n_bins: int, f_lo: float, f_hi: float, n_apod: int = 3, apod=None, pattern_m: int = 16,
                 eps: float = 1e-3, evanescent_zero: bool = False, nx: int = 0):
        _require_cuda()
        L = load()
        d = PlanDesc()
        L.pam_plan_desc_init(ctypes.byref(d))
        d.n_elem, d.pitch_m, d.fs_hz, d.c_mps = int(n_elem), float(pitch), float(fs), float(c)
        d.nx, d.z0_m, d.dz_m = int(nx), float(z0), float(dz)
        d.f_lo_hz, d.f_hi_hz, d.n_bins, d.n_apod = float(f_lo), float(f_hi), int(n_bins), int(n_apod)
        self._apod_keep = None
        if apod is not None:
            self._apod_keep = np.ascontiguousarray(np.asarray(apod, dtype=np.float32))
            d.apod = self._apod_keep.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        d.pattern_m, d.eps = int(pattern_m), float(eps)
        d.flags = PAM_EVANESCENT_ZERO if evanescent_zero else 0
        F = len(frames)
        fd = (FrameDesc * F)()
        self._keep = []
        for i, fr in enumerate(frames):
            fd[i].n_samples, fd[i].nz = int(fr[0]), int(fr[1])
            if len(fr) > 2 and fr[2] is not None:
                b = np.ascontiguousarray(np.asarray(fr[2], dtype=np.int32))
                self._keep.append(b)
                fd[i].bins = b.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        h = _VP()
        _check(L.pam_batch_create(ctypes.byref(d), fd, F, ctypes.byref(h)))
        self._h = h
        self.n_frames, self.n_elem, self.n_apod, self.n_bins = F, int(n_elem), int(n_apod), int(n_bins)
        self.nx = self.n_elem if not nx else int(nx)
        self.n_samples = [int(fr[0]) for fr in frames]
        self.nz = [int(fr[1]) for fr in frames]
        ro = (ctypes.c_size_t * F)()
        mo = (ctypes.c_size_t * F)()
        rt, mt = ctypes.c_size_t(), ctypes.c_size_t()
        _check(L.pam_batch_layout(h, ro, mo, ctypes.byref(rt), ctypes.byref(mt)))
        self.rf_offsets = [int(v) for v in ro]
        self.map_offsets = [int(v) for v in mo]
        self.rf_total, self.map_total = int(rt.value), int(mt.value)
        self.bins = []
        for i in range(F):
            out = np.zeros(self.n_bins, dtype=np.int32)
            n = L.pam_batch_bins(h, i, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
            self.bins.append(out[:n].copy())

    def pack_rf(self, frames_rf) -> "object":
        """Packs per-frame [n_elem][n_samples] arrays into the batch's rf layout (device tensor)."""
        torch = _require_cuda()
        buf = torch.zeros(self.rf_total, dtype=torch.float32)
        for i, a in enumerate(frames_rf):
            t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).reshape(-1)
            buf[self.rf_offsets[i]:self.rf_offsets[i] + t.numel()] = t
        return buf.cuda()

    def unpack(self, maps, i: int):
        """Frame i's [nz][nx] view of a packed map tensor."""
        n = self.nz[i] * self.nx
        return maps[self.map_offsets[i]:self.map_offsets[i] + n].view(self.nz[i], self.nx)

    def as_tax(self, rf, image=None, rho_n=None, want_rho_n: bool = True, stream=None):
        """AS-TAX / AS-DAX of every frame. Returns (image, rho_n) packed tensors."""
        torch = _require_cuda()
        if not isinstance(rf, torch.Tensor) or not rf.is_cuda or rf.dtype != torch.float32:
            raise TypeError("rf must be a float32 CUDA tensor")
        if rf.numel() < self.rf_total:
            raise ValueError(f"rf must hold {self.rf_total} floats")
        if image is None:
            image = torch.empty(self.map_total, dtype=torch.float32, device="cuda")
        if rho_n is None and want_rho_n:
            rho_n = torch.empty(self.map_total, dtype=torch.float32, device="cuda")
        _check(load().pam_batch_as_tax(self._h, _dptr(rf), _dptr(image), _dptr(rho_n), _stream_ptr(stream)))
        return image, rho_n

    def configure(self, use_graph: bool = True, persistent_ctas: int = 0):
        _check(load().pam_batch_configure(self._h, int(bool(use_graph)), int(persistent_ctas)))

    def info(self):
        """(work items, persistent grid, libpam kernel launches so far)."""
        n, g, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        _check(load().pam_batch_info(self._h, ctypes.byref(n), ctypes.byref(g), ctypes.byref(k)))
        return n.value, g.value, k.value

    def sync(self, stream=None):
        _check(load().pam_batch_sync(self._h, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None):
            load().pam_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Learned:
    """Learned AS-TAX (``pam_learn_*``): a 5-layer BF16 network predicts the
    TAX weight from band energies of the full-aperture AS map, with a per-frame
    error gate and the plain method as fallback. Training runs on the GPU in
    the library's kernels. ``max_frames`` is the batch size of every call."""

    def __init__(self, n_elem: int, pitch: float, fs: float, c: float, n_samples: int, nz: int,
                 z0: float, dz: float, bins: Optional[Sequence[int]] = None, f_lo: float = 0.0,
                 f_hi: float = 0.0, pattern_m: int = 16, eps: float = 1e-3, max_frames: int = 1, nx: int = 0,
                 apod=None):
        _require_cuda()
        L = load()
        d, self._bins_keep, self._apod_keep = _make_desc(
            n_elem, pitch, fs, c, n_samples, nz, z0, dz, bins, f_lo, f_hi, 3, apod, pattern_m, eps, False,
            max_frames, nx)
        h = _VP()
        _check(L.pam_learn_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.n_elem, self.n_samples, self.nz = int(n_elem), int(n_samples), int(nz)
        self.nx = self.n_elem if not nx else int(nx)
        self.max_frames = int(max_frames)
        self.n_params = int(L.pam_learn_n_params())
        self.feature_bytes = int(L.pam_learn_feature_bytes(h))

    @classmethod
    def from_workload(cls, w, max_frames: int = 1, **kw) -> "Learned":
        return cls(n_elem=w.n_elem, pitch=w.pitch, fs=w.fs, c=w.c, n_samples=w.nt, nz=w.nz, z0=w.z0, dz=w.dz,
                   bins=w.bins(), pattern_m=w.pattern_m, max_frames=max_frames, **kw)

    def close(self):
        if getattr(self, "_h", None):
            load().pam_learn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # parameters: flat float32, per layer w[out][in][3][3] then b[out]
    def set_params(self, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
        _check(load().pam_learn_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(load().pam_learn_get_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))
        return p

    def get_state(self):
        """(state, adam_steps): parameters, Adam m and v as one float32 array."""
        L = load()
        st = np.zeros(int(L.pam_learn_state_size()), dtype=np.float32)
        t = ctypes.c_longlong()
        _check(L.pam_learn_get_state(self._h, st.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), st.size,
                                     ctypes.byref(t)))
        return st, int(t.value)

    def set_state(self, state, adam_steps: int):
        st = np.ascontiguousarray(np.asarray(state, dtype=np.float32).ravel())
        _check(load().pam_learn_set_state(self._h, st.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), st.size,
                                          int(adam_steps)))

    def configure(self, gate_tol: float = 0.05, tensor_cores: bool = False):
        _check(load().pam_learn_configure(self._h, float(gate_tol), int(bool(tensor_cores))))

    def empty_features(self, n: int):
        """Uninitialised packed-feature tensor of n frames (uint8 view of BF16 [n][nz+2][nx+2][8])."""
        torch = _require_cuda()
        return torch.empty((n, self.feature_bytes), dtype=torch.uint8, device="cuda")

    def _rf(self, rf):
        torch = _require_cuda()
        if not isinstance(rf, torch.Tensor) or not rf.is_cuda or rf.dtype != torch.float32:
            raise TypeError("rf must be a float32 CUDA tensor")
        if rf.dim() == 2:
            rf = rf.unsqueeze(0)
        if tuple(rf.shape[1:]) != (self.n_elem, self.n_samples):
            raise ValueError(f"rf must be [F][{self.n_elem}][{self.n_samples}], got {tuple(rf.shape)}")
        return rf.contiguous()

    def _maps(self, n):
        torch = _require_cuda()
        return torch.empty((n, self.nz, self.nx), dtype=torch.float32, device="cuda")

    def example(self, rf, features=None, target=True, energy=False, stream=None):
        """Packed features and, optionally, the exact rho_TAX and energy E of each frame."""
        rf = self._rf(rf)
        n = rf.shape[0]
        feats = self.empty_features(n) if features is None else features
        tgt = self._maps(n) if target is True else (target if target is not False else None)
        en = self._maps(n) if energy is True else (energy if energy is not False else None)
        _check(load().pam_learn_example(self._h, _dptr(rf), n, _dptr(feats), _dptr(tgt), _dptr(en),
                                        _stream_ptr(stream)))
        return feats, tgt, en

    def forward(self, features, n: Optional[int] = None, out=None, stream=None):
        n = features.shape[0] if n is None else int(n)
        rho = self._maps(n) if out is None else out
        _check(load().pam_learn_forward(self._h, _dptr(features), n, _dptr(rho), _stream_ptr(stream)))
        return rho

    def grads(self, features, target, n: Optional[int] = None, stream=None):
        torch = _require_cuda()
        n = features.shape[0] if n is None else int(n)
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = torch.empty(4, dtype=torch.float32, device="cuda")
        _check(load().pam_learn_grads(self._h, _dptr(features), _dptr(target), n, _dptr(g), _dptr(loss),
                                      _stream_ptr(stream)))
        return g, loss[:1]

    def train_step(self, features, target, lr: float, n: Optional[int] = None, loss=None, stream=None):
        n = features.shape[0] if n is None else int(n)
        _check(load().pam_learn_train_step(self._h, _dptr(features), _dptr(target), n, float(lr), _dptr(loss),
                                           _stream_ptr(stream)))
        return loss

    def as_tax(self, rf, image=None, rho_n=None, want_rho_n: bool = True, stream=None):
        """Learned AS-TAX: dict of image, rho_n, gate_err [F] and gate_pass [F] (int32)."""
        torch = _require_cuda()
        rf = self._rf(rf)
        n = rf.shape[0]
        image = self._maps(n) if image is None else image
        if rho_n is None and want_rho_n:
            rho_n = self._maps(n)
        gerr = torch.empty(max(n, 4), dtype=torch.float32, device="cuda")
        gpass = torch.empty(max(n, 4), dtype=torch.int32, device="cuda")
        _check(load().pam_learn_tax(self._h, _dptr(rf), n, _dptr(image), _dptr(rho_n), _dptr(gerr), _dptr(gpass),
                                    _stream_ptr(stream)))
        return {"image": image, "rho_n": rho_n, "gate_err": gerr[:n], "gate_pass": gpass[:n]}

    def sync(self, stream=None):
        _check(load().pam_learn_sync(self._h, _stream_ptr(stream)))

    def info(self):
        k = ctypes.c_longlong()
        mf = ctypes.c_int()
        t = ctypes.c_longlong()
        _check(load().pam_learn_info(self._h, ctypes.byref(k), ctypes.byref(mf), ctypes.byref(t)))
        return {"kernel_launches": k.value, "max_frames": mf.value, "adam_steps": t.value}


METRIC_FIELDS = ("esa_m2", "isnr_db", "cx_m", "cz_m", "max", "n_inside")


def image_metrics(maps, x0: float, dx: float, z0: float, dz: float, alpha: float = 0.7, stream=None):
    """Eq. 12-13 measures of device maps [F][nz][nx]: a list of dicts (one per frame)."""
    torch = _require_cuda()
    if maps.dim() == 2:
        maps = maps.unsqueeze(0)
    maps = maps.contiguous()
    F, nz, nx = maps.shape
    out = torch.empty((max(F, 1), 6), dtype=torch.float32, device=maps.device)   # 6 x 4-byte fields
    _check(load().pam_image_metrics(_dptr(maps), F, nz, nx, float(x0), float(dx), float(z0), float(dz),
                                    float(alpha), _dptr(out), _stream_ptr(stream)))
    raw = out[:F].cpu().numpy()
    n_in = raw[:, 5].copy().view(np.int32)
    return [dict(zip(METRIC_FIELDS, [float(v) for v in r[:5]] + [int(n)])) for r, n in zip(raw, n_in)]



def unpack_features(features, nz: int, nx: int):
    """Packed features (uint8 tensor or array) -> float32 numpy [n][5][nz][nx]."""
    a = features.detach().cpu().numpy() if hasattr(features, "detach") else np.asarray(features)
    u16 = a.view(np.uint16).reshape(a.shape[0], nz + 2, nx + 2, 8)
    f32 = (u16.astype(np.uint32) << 16).view(np.float32)
    return np.ascontiguousarray(f32[:, 1:nz + 1, 1:nx + 1, :5].transpose(0, 3, 1, 2))


def pack_features(x):
    """float numpy [n][5][nz][nx] -> packed BF16 features as uint8 numpy [n][bytes] (round to nearest even)."""
    x = np.asarray(x, dtype=np.float32)
    n, c, nz, nx = x.shape
    if c != 5:
        raise ValueError("features have 5 channels")
    bits = x.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16).astype(np.uint16)
    out = np.zeros((n, nz + 2, nx + 2, 8), dtype=np.uint16)
    out[:, 1:nz + 1, 1:nx + 1, :5] = rounded.transpose(0, 2, 3, 1)
    return out.reshape(n, -1).view(np.uint8)


def status_string(s: int) -> str:
    return load().pam_status_string(int(s)).decode()
