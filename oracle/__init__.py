"""FP64 CPU oracle of the beamformer hot path (decode, DAS, DAS gradients).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The library and its CUDA
kernels never import, link or run anything here, and this package imports
nothing from the library.

The arithmetic lives in ``rcbf_oracle.c`` (plain loops, FP64 / int64, OpenMP
over independent outputs); this module compiles it with gcc and marshals
numpy arrays. ``twin.py`` is a second, pure-Python brute-force copy of the
same definitions for tiny inputs.

Passages followed: §THEORY "Synthetic Aperture Imaging" (Eq. (1) DAS,
Eq. (2) constant-F# receive apodization, Eq. (3) Hanning window; decoding as a
product across transmits) and §OPTIMIZATIONS "Decoding".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rcbf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no target-specific flags)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(ctypes.Structure):
    _fields_ = [
        ("n_tx", ctypes.c_int64), ("n_ch", ctypes.c_int64), ("n_samples", ctypes.c_int64),
        ("tx_orientation", ctypes.c_int64), ("rx_orientation", ctypes.c_int64),
        ("dims", ctypes.c_int64 * 3),
        ("has_voxel_transform", ctypes.c_int64), ("has_xdc_transform", ctypes.c_int64),
        ("fs", ctypes.c_double), ("c", ctypes.c_double), ("t0", ctypes.c_double),
        ("tx_pitch", ctypes.c_double), ("rx_pitch", ctypes.c_double),
        ("f_number", ctypes.c_double),
        ("out_min", ctypes.c_double * 3), ("out_max", ctypes.c_double * 3),
        ("voxel_transform", ctypes.c_double * 16), ("xdc_transform", ctypes.c_double * 16),
        ("interp", ctypes.c_int64), ("iq_freq", ctypes.c_double),
        ("tx_wave", ctypes.c_int64), ("tx_focus", ctypes.c_double), ("tx_angles", ctypes.c_void_p),
        ("acq_kind", ctypes.c_int64),
    ]

TX_WAVE = {"line": 0, "plane": 1, "vls": 2, "point": 3}

INTERP = {"linear": 0, "cubic": 1}


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.oracle_hadamard.argtypes = [I64, P]
            lib.oracle_decode.argtypes = [I64, I64, P, P, P]
            lib.oracle_das.argtypes = [P, P, I64, P, ctypes.c_double, I64, P, P]
            lib.oracle_das_grad.argtypes = [P, P, I64, P, ctypes.c_double, P, P, P, P]
            lib.oracle_demodulate.argtypes = [I64, I64, P, P, I64, I64, I64, I64, P]
            lib.oracle_demodulate_complex.argtypes = [I64, I64, P, P, P, I64, I64, I64, I64, P]
            lib.oracle_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def threads() -> int:
    return int(_load().oracle_threads())


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def geom_from(g, c: Optional[float] = None, f_number: Optional[float] = None,
              voxel_transform=None, xdc_transform=None, interp: Optional[str] = None,
              iq_freq: Optional[float] = None) -> _Geom:
    """Oracle geometry from any object with the synth.Geometry attributes
    (interp: 'linear' or 'cubic', default the geometry's own, else linear;
    iq_freq: demodulation frequency of baseband IQ data, default the
    geometry's own, else 0 = RF data)."""
    s = _Geom()
    s.iq_freq = float(iq_freq if iq_freq is not None else getattr(g, "iq_freq", 0.0))
    s.tx_wave = TX_WAVE[getattr(g, "tx_wave", "line")]
    s.tx_focus = float(getattr(g, "tx_focus", 0.0))
    s.acq_kind = int(getattr(g, "acq_kind", 0))
    if s.tx_wave == 1:
        ang = np.ascontiguousarray(getattr(g, "tx_angles"), dtype=np.float64)
        if ang.size != (1 if s.acq_kind == 2 else int(g.n_tx)):
            raise ValueError("one plane-wave angle per transmit (one for a 2D receive aperture)")
        s._angles = ang                      # kept alive with the structure
        s.tx_angles = ang.ctypes.data
    s.interp = INTERP[interp if interp is not None else getattr(g, "interp", "linear")]
    s.n_tx, s.n_ch, s.n_samples = int(g.n_tx), int(g.n_ch), int(g.n_samples)
    s.tx_orientation, s.rx_orientation = int(g.tx_orientation), int(g.rx_orientation)
    for d in range(3):
        s.dims[d] = int(g.out_dims[d])
        s.out_min[d] = float(g.out_min[d])
        s.out_max[d] = float(g.out_max[d])
    s.fs, s.t0 = float(g.fs), float(g.t0)
    s.c = float(c if c is not None else g.c)
    s.tx_pitch, s.rx_pitch = float(g.tx_pitch), float(g.rx_pitch)
    s.f_number = float(f_number if f_number is not None else g.f_number)
    if voxel_transform is not None:
        s.has_voxel_transform = 1
        for k, val in enumerate(np.asarray(voxel_transform, dtype=np.float64).ravel()):
            s.voxel_transform[k] = val
    if xdc_transform is not None:
        s.has_xdc_transform = 1
        for k, val in enumerate(np.asarray(xdc_transform, dtype=np.float64).ravel()):
            s.xdc_transform[k] = val
    return s


# ------------------------------------------------------------------ decode

def hadamard(n: int) -> np.ndarray:
    """Sylvester H[k][i] = (-1)^popcount(k & i), int8."""
    H = np.empty((n, n), dtype=np.int8)
    _load().oracle_hadamard(n, _ptr(H))
    return H


def decode(rf: np.ndarray, H: Optional[np.ndarray] = None) -> np.ndarray:
    """D[i] = sum_k H[k][i] rf[k] over the transmit axis, exact int64."""
    rf = np.ascontiguousarray(rf, dtype=np.int16)
    n = rf.shape[0]
    H = hadamard(n) if H is None else np.ascontiguousarray(H, dtype=np.int8)
    D = np.empty(rf.shape, dtype=np.int64)
    _load().oracle_decode(n, rf.size // n, _ptr(rf), _ptr(H), _ptr(D))
    return D


def decoded_as(D: np.ndarray, n: int, dtype: str) -> np.ndarray:
    """The exact decode D rendered in an output dtype: 'i32' = D; 'f32' /
    'f16' = D / n rounded once to nearest-even (D / n is exact in float64)."""
    if dtype == "i32":
        return D.astype(np.int32)
    exact = D.astype(np.float64) / float(n)
    if dtype == "f32":
        return exact.astype(np.float32)
    if dtype == "f16":
        return exact.astype(np.float16)
    raise ValueError(dtype)


# --------------------------------------------------------------------- DAS

def das(g, rf: np.ndarray, w: Optional[np.ndarray] = None, c: Optional[float] = None,
        voxels: Optional[np.ndarray] = None, **geom_kw) -> np.ndarray:
    """Eq. (1)-(3) in FP64. rf: real [n_tx][n_ch][n_s] or complex (two planes
    are beamformed independently). Returns the image [nz][ny][nx] (or the
    listed voxels), complex when rf is complex."""
    cplx = np.iscomplexobj(rf)
    planes = np.stack([rf.real, rf.imag]) if cplx else rf[None]
    planes = np.ascontiguousarray(planes, dtype=np.float64)
    geom = geom_from(g, c=c, **geom_kw)
    n_all = int(np.prod(g.out_dims))
    vox = None if voxels is None else np.ascontiguousarray(voxels, dtype=np.int64)
    n_vox = n_all if vox is None else vox.size
    out = np.empty((planes.shape[0], n_vox), dtype=np.float64)
    wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    _load().oracle_das(ctypes.byref(geom), _ptr(planes), planes.shape[0], _ptr(wv),
                       float(geom.c), n_vox, _ptr(vox), _ptr(out))
    res = out[0] + 1j * out[1] if cplx else out[0]
    if vox is None:
        res = res.reshape(g.out_dims[2], g.out_dims[1], g.out_dims[0])
    return res


def das_grad(g, rf: np.ndarray, G: np.ndarray, w: Optional[np.ndarray] = None,
             c: Optional[float] = None, want_rf: bool = True, **geom_kw):
    """(grad_rf, grad_c, grad_w) of L given dL/dimage = G (same dtype and
    shape as the image: complex for complex rf, G = dL/dRe + j dL/dIm)."""
    cplx = np.iscomplexobj(rf)
    planes = np.stack([rf.real, rf.imag]) if cplx else rf[None]
    planes = np.ascontiguousarray(planes, dtype=np.float64)
    Gp = np.stack([G.real, G.imag]) if cplx else np.asarray(G)[None]
    Gp = np.ascontiguousarray(Gp.reshape(planes.shape[0], -1), dtype=np.float64)
    geom = geom_from(g, c=c, **geom_kw)
    if geom.interp != 0 or geom.iq_freq > 0 or geom.acq_kind == 2:
        raise NotImplementedError("the DAS gradients are defined for linear interpolation of RF data")
    grad_rf = np.empty_like(planes) if want_rf else None
    gc = np.zeros(1, dtype=np.float64)
    gw = np.zeros(g.n_ch, dtype=np.float64)
    wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    _load().oracle_das_grad(ctypes.byref(geom), _ptr(planes), planes.shape[0], _ptr(wv),
                            float(geom.c), _ptr(Gp), _ptr(grad_rf), _ptr(gc), _ptr(gw))
    if grad_rf is not None:
        grad_rf = grad_rf[0] + 1j * grad_rf[1] if cplx else grad_rf[0]
    return grad_rf, float(gc[0]), gw


# ------------------------------------------------------------ demodulation

def demodulate(rf: np.ndarray, taps: np.ndarray, shift: int, decimation: int,
               taps_imag: Optional[np.ndarray] = None) -> np.ndarray:
    """Eq. (demodulation) at quadrature sampling (f_d = f_s / 4) with int16
    taps (real, or complex with the imaginary parts in taps_imag), a rounding
    right shift and decimation, in exact integers.
    rf: int16 [..., n_in] -> int16 [2, ..., n_in // decimation] (I, Q)."""
    rf = np.ascontiguousarray(rf, dtype=np.int16)
    h = np.ascontiguousarray(taps, dtype=np.int16)
    hi = None if taps_imag is None else np.ascontiguousarray(taps_imag, dtype=np.int16)
    if hi is not None and hi.size != h.size:
        raise ValueError("taps_imag must have the length of taps")
    n_in = rf.shape[-1]
    n_out = n_in // int(decimation)
    n_traces = rf.size // n_in
    out = np.empty((2,) + rf.shape[:-1] + (n_out,), dtype=np.int16)
    _load().oracle_demodulate_complex(n_traces, n_in, _ptr(rf), _ptr(h), _ptr(hi), h.size, int(shift),
                                      int(decimation), n_out, _ptr(out))
    return out
