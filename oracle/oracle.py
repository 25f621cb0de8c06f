"""ctypes front end of the FP64 CPU oracle (``pam_oracle.c``).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module. The GPU library never
does. The oracle computes what the paper (arXiv 2412.02413) defines, in FP64
and by direct sums:

* Eq. 1: time DFT and lateral DFT;
* Eq. 2: spectral propagator;
* Eq. 3: AS energy;
* Eq. 4 with the Appendix A completion: NCC;
* Eq. 5 and Eq. 10-11: AS-DAX and AS-TAX images.

Parity status of each function is in the header of ``pam_oracle.c`` and in
the pins under ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pam_oracle.c")
_LIB = os.path.join(_HERE, "libpam_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc. The flags keep IEEE semantics: no fast-math
    and no FMA contraction, so results match across x86 and Arm hosts."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pam_oracle.h"))
    ):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wextra", "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Geom(ctypes.Structure):
    _fields_ = [
        ("n_elem", ctypes.c_int), ("nt", ctypes.c_int), ("nx", ctypes.c_int),
        ("nz", ctypes.c_int), ("n_bins", ctypes.c_int),
        ("bins", ctypes.POINTER(ctypes.c_int)),
        ("pitch", ctypes.c_double), ("fs", ctypes.c_double), ("c", ctypes.c_double),
        ("z0", ctypes.c_double), ("dz", ctypes.c_double),
        ("evanescent_zero", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.pam_oracle_pattern.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
            L.pam_oracle_band_bins.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, _I, ctypes.c_int]
            L.pam_oracle_time_dft.argtypes = [_F, ctypes.c_int, ctypes.c_int, _I, ctypes.c_int, _D]
            L.pam_oracle_time_dft.restype = None
            L.pam_oracle_lateral_dft.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, _D]
            L.pam_oracle_lateral_dft.restype = None
            L.pam_oracle_kz.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, _D, _D, _D]
            L.pam_oracle_kz.restype = None
            L.pam_oracle_propagate.argtypes = [_D, _D, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_int, _D]
            L.pam_oracle_propagate.restype = None
            L.pam_oracle_lateral_idft.argtypes = [_D, ctypes.c_int, _D]
            L.pam_oracle_lateral_idft.restype = None
            L.pam_oracle_fields.argtypes = [ctypes.POINTER(Geom), _F, _D, _D]
            L.pam_oracle_as_backprop.argtypes = [ctypes.POINTER(Geom), _F, _D, _D, ctypes.c_int]
            L.pam_oracle_as_xcorr.argtypes = [ctypes.POINTER(Geom), _F, ctypes.c_int, _D,
                                              ctypes.c_double, _D, _D, _D, _D, _D, ctypes.c_int]
            L.pam_oracle_set_mutation.argtypes = [ctypes.c_int]
            L.pam_oracle_set_mutation.restype = None
            _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _c128(a):
    """complex128 array -> contiguous float64 view [..., 2]"""
    return np.ascontiguousarray(a, dtype=np.complex128)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class Geometry:
    """Array, sampling, depth grid and bin list of one acquisition."""

    def __init__(self, n_elem, nt, fs, c, pitch, nz, z0, dz, bins, evanescent_zero=False):
        self.n_elem, self.nt, self.fs, self.c, self.pitch = int(n_elem), int(nt), float(fs), float(c), float(pitch)
        self.nx = self.n_elem
        self.nz, self.z0, self.dz = int(nz), float(z0), float(dz)
        self.bins = np.ascontiguousarray(np.asarray(bins, dtype=np.int32))
        self.evanescent_zero = bool(evanescent_zero)

    def c_struct(self) -> Geom:
        g = Geom()
        g.n_elem, g.nt, g.nx, g.nz = self.n_elem, self.nt, self.nx, self.nz
        g.n_bins = int(self.bins.size)
        g.bins = self.bins.ctypes.data_as(_I)
        g.pitch, g.fs, g.c, g.z0, g.dz = self.pitch, self.fs, self.c, self.z0, self.dz
        g.evanescent_zero = int(self.evanescent_zero)
        return g


def pattern(n_elem: int, n_apod: int, m: int) -> np.ndarray:
    out = np.zeros((n_apod, n_elem), dtype=np.float64)
    if lib().pam_oracle_pattern(n_elem, n_apod, m, _dp(out)) != 0:
        raise ValueError("bad pattern arguments")
    return out


def band_bins(nt: int, fs: float, f_lo: float, f_hi: float) -> np.ndarray:
    n = lib().pam_oracle_band_bins(nt, fs, f_lo, f_hi, None, 0)
    out = np.zeros(max(n, 1), dtype=np.int32)
    lib().pam_oracle_band_bins(nt, fs, f_lo, f_hi, out.ctypes.data_as(_I), n)
    return out[:n]


def time_dft(rf: np.ndarray, bins) -> np.ndarray:
    """[n_bins][n_elem] complex128"""
    rf = np.ascontiguousarray(rf, dtype=np.float32)
    ne, nt = rf.shape
    b = np.ascontiguousarray(np.asarray(bins, dtype=np.int32))
    S = np.zeros((b.size, ne), dtype=np.complex128)
    lib().pam_oracle_time_dft(rf.ctypes.data_as(_F), ne, nt, b.ctypes.data_as(_I), b.size, _dp(S))
    return S


def lateral_dft(S_row: np.ndarray, apod=None, nx=None) -> np.ndarray:
    S_row = _c128(S_row)
    ne = S_row.size
    nx = ne if nx is None else nx
    a = None if apod is None else np.ascontiguousarray(apod, dtype=np.float64)
    Q = np.zeros(nx, dtype=np.complex128)
    lib().pam_oracle_lateral_dft(_dp(S_row), _dp(a), ne, nx, _dp(Q))
    return Q


def kz(f_hz: float, c: float, pitch: float, nx: int):
    """(kx[nx], kz[nx] complex) for every lateral bin."""
    kx = np.zeros(nx)
    kzv = np.zeros(nx, dtype=np.complex128)
    for u in range(nx):
        a, r, i = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        lib().pam_oracle_kz(f_hz, c, pitch, nx, u, ctypes.byref(a), ctypes.byref(r), ctypes.byref(i))
        kx[u], kzv[u] = a.value, complex(r.value, i.value)
    return kx, kzv


def propagate(Q: np.ndarray, kzv: np.ndarray, dz: float, evanescent_zero=False) -> np.ndarray:
    Q = _c128(Q)
    k = _c128(kzv)
    P = np.zeros_like(Q)
    lib().pam_oracle_propagate(_dp(Q), _dp(k), Q.size, dz, int(evanescent_zero), _dp(P))
    return P


def lateral_idft(P: np.ndarray) -> np.ndarray:
    P = _c128(P)
    p = np.zeros_like(P)
    lib().pam_oracle_lateral_idft(_dp(P), P.size, _dp(p))
    return p


def fields(geom: Geometry, rf: np.ndarray, apod=None) -> np.ndarray:
    """[n_bins][nz][nx] complex128 monochromatic fields of one apodization."""
    rf = np.ascontiguousarray(rf, dtype=np.float32)
    a = None if apod is None else np.ascontiguousarray(apod, dtype=np.float64)
    out = np.zeros((geom.bins.size, geom.nz, geom.nx), dtype=np.complex128)
    g = geom.c_struct()
    if lib().pam_oracle_fields(ctypes.byref(g), rf.ctypes.data_as(_F), _dp(a), _dp(out)) != 0:
        raise ValueError("oracle rejected the geometry")
    return out


def as_backprop(geom: Geometry, rf: np.ndarray, apod=None, threads=None) -> np.ndarray:
    """[nz][nx] AS energy map (Eq. 3)."""
    rf = np.ascontiguousarray(rf, dtype=np.float32)
    a = None if apod is None else np.ascontiguousarray(apod, dtype=np.float64)
    out = np.zeros((geom.nz, geom.nx))
    g = geom.c_struct()
    rc = lib().pam_oracle_as_backprop(ctypes.byref(g), rf.ctypes.data_as(_F), _dp(a), _dp(out),
                                      threads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle rejected the geometry ({rc})")
    return out


def as_xcorr(geom: Geometry, rf: np.ndarray, apod: np.ndarray, eps: float = 1e-3, threads=None):
    """AS-DAX (2 apodizations) or AS-TAX (3). Returns a dict of FP64 maps:
    image, rho_n, rho_pairs [n_pairs][nz][nx], image_as, acc [7][nz][nx]."""
    rf = np.ascontiguousarray(rf, dtype=np.float32)
    apod = np.ascontiguousarray(apod, dtype=np.float64)
    n_apod = apod.shape[0]
    npairs = 1 if n_apod == 2 else 3
    shp = (geom.nz, geom.nx)
    out = dict(image=np.zeros(shp), rho_n=np.zeros(shp), rho_pairs=np.zeros((npairs,) + shp),
               image_as=np.zeros(shp), acc=np.zeros((7,) + shp))
    g = geom.c_struct()
    rc = lib().pam_oracle_as_xcorr(ctypes.byref(g), rf.ctypes.data_as(_F), n_apod, _dp(apod), eps,
                                   _dp(out["image"]), _dp(out["rho_n"]), _dp(out["rho_pairs"]),
                                   _dp(out["image_as"]), _dp(out["acc"]), threads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle rejected the geometry ({rc})")
    return out


def as_tax(geom: Geometry, rf: np.ndarray, apod: np.ndarray, eps: float = 1e-3, threads=None):
    assert apod.shape[0] == 3
    return as_xcorr(geom, rf, apod, eps, threads)


# ---- 2x lateral padding (Sec. II-D) ----
# Reading: the channel record is extended by n_elem zero channels appended
# after the last element (element e stays on channel e, at the element pitch),
# the lateral transforms of Eq. 1-2 run over 2 n_elem points, and the image is
# cropped back to the n_elem element columns. The TAX weight is normalised to
# its maximum over the cropped image (Eq. 11), and I = rho_n^2 E_full there.
_py_mutation = 0   # deliberate mistakes 11-12 of the mutation tests live in this file


def _padded(geom: Geometry, rf: np.ndarray, apod):
    ne = geom.n_elem
    if _py_mutation == 12:   # planted mistake: no padding at all
        return geom, np.asarray(rf, dtype=np.float32), None if apod is None else np.asarray(apod, np.float64)
    g2 = Geometry(2 * ne, geom.nt, geom.fs, geom.c, geom.pitch, geom.nz, geom.z0, geom.dz, geom.bins,
                  geom.evanescent_zero)
    rf = np.asarray(rf, dtype=np.float32)
    rf2 = np.zeros((2 * ne, rf.shape[-1]), dtype=np.float32)
    rf2[:ne] = rf
    a2 = None
    if apod is not None:
        apod = np.asarray(apod, dtype=np.float64)
        a2 = np.zeros(apod.shape[:-1] + (2 * ne,))
        a2[..., :ne] = apod
    return g2, rf2, a2


def _crop(geom: Geometry) -> slice:
    ne = geom.n_elem
    return slice(ne, 2 * ne) if _py_mutation == 11 else slice(0, ne)   # 11: the padding columns


def as_backprop_pad2x(geom: Geometry, rf: np.ndarray, apod=None, threads=None) -> np.ndarray:
    """[nz][n_elem] AS energy (Eq. 3) with 2x lateral padding."""
    g2, rf2, a2 = _padded(geom, rf, apod)
    return np.ascontiguousarray(as_backprop(g2, rf2, a2, threads)[:, _crop(geom)])


def as_xcorr_pad2x(geom: Geometry, rf: np.ndarray, apod: np.ndarray, eps: float = 1e-3, threads=None):
    """AS-DAX / AS-TAX (Eq. 5, 10-11) with 2x lateral padding: the maps of
    :func:`as_xcorr` on the padded record, cropped to the element columns, with
    rho_n renormalised over the crop and the image rebuilt from it."""
    g2, rf2, a2 = _padded(geom, rf, apod)
    full = as_xcorr(g2, rf2, a2, eps, threads)
    out = {k: np.ascontiguousarray(v[..., _crop(geom)]) for k, v in full.items()}
    rho_n = out["rho_n"] / out["rho_n"].max()
    out["rho_n"] = rho_n
    out["image"] = rho_n * rho_n * out["image_as"]
    return out


def set_mutation(mid: int) -> None:
    """Test hook: switch on deliberate mistake ``mid`` (0 restores the oracle).
    Mistakes 1-10 are in pam_oracle.c, 11-12 in the padding reading above."""
    global _py_mutation
    _py_mutation = int(mid)
    lib().pam_oracle_set_mutation(int(mid))
