"""GB300 row-column / TOBE beamformer hot path: Python binding of librcbf.so.

This module only marshals arguments for the C ABI declared in
``include/rcbf.h``: every step of the path (decode, DAS, its adjoint, the
batched persistent launch) runs in the library's CUDA kernels. PyTorch
provides device memory and the current CUDA stream. There is no CPU fallback:
if the compiled library is missing, importing the binding raises.

Names follow the paper (Palamar et al., arXiv 2512.11086): ``decode`` is the
Hadamard aperture decode (§THEORY "Synthetic Aperture Imaging",
§OPTIMIZATIONS "Decoding"), ``das`` the delay-and-sum of Eq. (1) with the
receive apodization of Eq. (2)-(3) (§OPTIMIZATIONS "DAS").
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librcbf.so")

# ---- constants mirrored from rcbf.h
OK, EINVAL, EUNSUPPORTED, ECUDA, ENOMEM, ETIMEOUT = 0, -1, -2, -3, -4, -5
I16, I32, F32, F16, CF32 = 0, 1, 2, 3, 4
FORCES, HERCULES = 0, 1
ROWS, COLUMNS = 0, 1
LINEAR, CUBIC = 0, 1
TX_LINE, TX_PLANE, TX_VLS, TX_POINT = 0, 1, 2, 3
_TX_WAVE_NAMES = {"line": TX_LINE, "plane": TX_PLANE, "vls": TX_VLS, "point": TX_POINT}
HERCULES_2D = 2
_INTERP_NAMES = {"linear": LINEAR, "cubic": CUBIC}
DECODE_MMA_I8, DECODE_PLAIN, DECODE_MMA_F16, DECODE_TC = 0, 1, 2, 3
DAS_TILED, DAS_PLAIN = 0, 1

_DTYPE_NAMES = {"i32": I32, "f32": F32, "f16": F16, "cf32": CF32}


class RcbfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("rcbf error %d: %s" % (code, msg))
        self.code = code


class Params(ctypes.Structure):
    """ctypes mirror of ``rcbf_params`` (field order and types as in rcbf.h)."""
    _fields_ = [
        ("n_tx", ctypes.c_uint32), ("n_ch", ctypes.c_uint32), ("n_samples", ctypes.c_uint32),
        ("hadamard_order", ctypes.c_uint32), ("acq_kind", ctypes.c_uint32),
        ("tx_orientation", ctypes.c_uint32), ("rx_orientation", ctypes.c_uint32),
        ("decoded_dtype", ctypes.c_uint32), ("interp", ctypes.c_uint32),
        ("decode_variant", ctypes.c_uint32), ("das_variant", ctypes.c_uint32),
        ("out_dims", ctypes.c_uint32 * 3), ("tile", ctypes.c_uint32 * 3), ("reserved", ctypes.c_uint32),
        ("fs", ctypes.c_double), ("c", ctypes.c_double), ("t0", ctypes.c_double), ("fc", ctypes.c_double),
        ("tx_pitch", ctypes.c_double), ("rx_pitch", ctypes.c_double),
        ("xdc_transform", ctypes.c_double * 16),
        ("out_min", ctypes.c_double * 3), ("out_max", ctypes.c_double * 3),
        ("voxel_transform", ctypes.c_double * 16),
        ("f_number", ctypes.c_double),
        ("decode_matrix", ctypes.c_void_p),
        ("demod_decimation", ctypes.c_uint32), ("demod_n_taps", ctypes.c_uint32),
        ("demod_shift", ctypes.c_int32), ("reserved2", ctypes.c_uint32),
        ("demod_taps", ctypes.c_void_p),
        ("iq_freq", ctypes.c_double),
        ("tx_wave", ctypes.c_uint32), ("reserved3", ctypes.c_uint32),
        ("tx_focus", ctypes.c_double), ("tx_angles", ctypes.c_void_p),
        ("rx_channel_offset", ctypes.c_uint32), ("rx_channels_total", ctypes.c_uint32),
        ("demod_taps_imag", ctypes.c_void_p),
    ]


class PlanInfo(ctypes.Structure):
    """ctypes mirror of ``rcbf_plan_info``."""
    _fields_ = [
        ("tile", ctypes.c_uint32 * 3), ("tiled", ctypes.c_uint32), ("window", ctypes.c_uint32),
        ("n_split", ctypes.c_uint32), ("das_launches", ctypes.c_uint32),
        ("decode_launches", ctypes.c_uint32), ("workspace_bytes", ctypes.c_uint64),
        ("bwd_tile", ctypes.c_uint32 * 3), ("bwd_mode", ctypes.c_uint32),
    ]


# symbol -> (restype, argtypes); every function rcbf.h declares
_P = ctypes.c_void_p
class Ceilings(ctypes.Structure):
    _fields_ = [("lds64_bytes_per_s", ctypes.c_double), ("ffma_lane_ops_per_s", ctypes.c_double),
                ("ffma2_lane_ops_per_s", ctypes.c_double), ("red_shared_per_s", ctypes.c_double),
                ("sm_clock_hz", ctypes.c_double)]


SIGNATURES = {
    "rcbf_plan": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(_P)]),
    "rcbf_destroy": (None, [_P]),
    "rcbf_plan_query": (ctypes.c_int, [_P, ctypes.POINTER(PlanInfo)]),
    "rcbf_decode": (ctypes.c_int, [_P, _P, _P, _P]),
    "rcbf_demod_decode": (ctypes.c_int, [_P, _P, _P, _P]),
    "rcbf_demodulate": (ctypes.c_int, [_P, _P, _P, _P]),
    "rcbf_das": (ctypes.c_int, [_P, _P, _P, ctypes.c_float, _P, _P]),
    "rcbf_das_backward": (ctypes.c_int, [_P, _P, _P, ctypes.c_float, _P, _P, _P, _P, _P]),
    "rcbf_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_uint32, ctypes.POINTER(_P),
                                         ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "rcbf_batch_run": (ctypes.c_int, [_P, _P]),
    "rcbf_pipeline_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_P)]),
    "rcbf_pipeline_submit": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "rcbf_pipeline_wait": (ctypes.c_int, [_P]),
    "rcbf_pipeline_destroy": (None, [_P]),
    "rcbf_batch_status": (ctypes.c_int, [_P, _P]),
    "rcbf_batch_set_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int32]),
    "rcbf_batch_destroy": (None, [_P]),
    "rcbf_das_noalloc": (ctypes.c_int, [ctypes.POINTER(Params), _P, _P, ctypes.c_float, _P, _P]),
    "rcbf_das_noalloc_status": (ctypes.c_int, [_P]),
    "rcbf_plan_status": (ctypes.c_int, [_P, _P]),
    "rcbf_plan_set_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int32]),
    "rcbf_measure_ceilings": (ctypes.c_int, [ctypes.POINTER(Ceilings), _P]),
    "rcbf_last_error": (ctypes.c_char_p, []),
    "rcbf_version": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load librcbf.so (build it first with ``paper_2512_11086_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("librcbf.so is not built (%s); run __graft_entry__.build() or "
                          "python paper_2512_11086_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code: int):
    if code != OK:
        raise RcbfError(code, load_library().rcbf_last_error().decode())


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def make_params(g, decoded_dtype="f32", decode_variant=DECODE_MMA_I8, das_variant=DAS_TILED,
                tile=None, f_number=None, xdc_transform=None, voxel_transform=None, interp=None,
                demod=None, iq_freq=None) -> Params:
    """Parameter block from any object with the geometry attributes (n_tx,
    n_ch, n_samples, fs, c, t0, fc, pitches, orientations, hadamard_order,
    out_dims, out_min, out_max, f_number, optionally interp: 'linear' or
    'cubic', iq_freq; the arguments override them). demod = (decimation,
    int16 taps, shift[, int16 imaginary taps]) adds the quadrature
    demodulation stage (complex taps when the fourth item is given); the
    geometry then describes the demodulated data (n_samples, fs, t0)."""
    p = Params()
    p.n_tx, p.n_ch, p.n_samples = int(g.n_tx), int(g.n_ch), int(g.n_samples)
    p.hadamard_order = int(getattr(g, "hadamard_order", 0))
    p.acq_kind = int(getattr(g, "acq_kind", FORCES))
    p.tx_orientation, p.rx_orientation = int(g.tx_orientation), int(g.rx_orientation)
    p.decoded_dtype = _DTYPE_NAMES[decoded_dtype] if isinstance(decoded_dtype, str) else int(decoded_dtype)
    it = interp if interp is not None else getattr(g, "interp", "linear")
    p.interp = _INTERP_NAMES[it] if isinstance(it, str) else int(it)
    p.decode_variant, p.das_variant = int(decode_variant), int(das_variant)
    for d in range(3):
        p.out_dims[d] = int(g.out_dims[d])
        p.out_min[d] = float(g.out_min[d])
        p.out_max[d] = float(g.out_max[d])
    if tile is not None:
        for d in range(3):
            p.tile[d] = int(tile[d])
    p.fs, p.c, p.t0, p.fc = float(g.fs), float(g.c), float(g.t0), float(getattr(g, "fc", 0.0))
    p.tx_pitch, p.rx_pitch = float(g.tx_pitch), float(g.rx_pitch)
    p.f_number = float(g.f_number if f_number is None else f_number)
    p.iq_freq = float(iq_freq if iq_freq is not None else getattr(g, "iq_freq", 0.0))
    wave = getattr(g, "tx_wave", "line")
    p.tx_wave = _TX_WAVE_NAMES[wave] if isinstance(wave, str) else int(wave)
    p.tx_focus = float(getattr(g, "tx_focus", 0.0))
    if p.tx_wave == TX_PLANE:
        import numpy as np
        ang = np.ascontiguousarray(getattr(g, "tx_angles"), dtype=np.float64)
        if ang.size < (1 if p.acq_kind == HERCULES_2D else p.n_tx):
            raise ValueError("plane waves need one angle per transmit (one for a 2D receive aperture)")
        p.tx_angles = ang.ctypes.data
        p._angles = ang         # kept alive until rcbf_plan copies it
    if demod is not None:
        import numpy as np
        dec, taps, shift = demod[:3]
        taps = np.ascontiguousarray(taps, dtype=np.int16)
        p.demod_decimation, p.demod_n_taps, p.demod_shift = int(dec), int(taps.size), int(shift)
        p.demod_taps = taps.ctypes.data
        p._taps = taps          # kept alive until rcbf_plan copies it
        if len(demod) > 3 and demod[3] is not None:
            taps_im = np.ascontiguousarray(demod[3], dtype=np.int16)
            if taps_im.size != taps.size:
                raise ValueError("the imaginary taps need the length of the real taps")
            p.demod_taps_imag = taps_im.ctypes.data
            p._taps_im = taps_im
    if xdc_transform is not None:
        for k, v in enumerate([float(x) for row in xdc_transform for x in row]):
            p.xdc_transform[k] = v
    if voxel_transform is not None:
        for k, v in enumerate([float(x) for row in voxel_transform for x in row]):
            p.voxel_transform[k] = v
    return p


class Plan:
    """Owns an ``rcbf_plan_t``. Device buffers are torch CUDA tensors."""

    def __init__(self, params: Params, decode_matrix=None):
        lib = load_library()
        self._keep = None
        if decode_matrix is not None:
            import numpy as np
            m = np.ascontiguousarray(decode_matrix, dtype=np.int8)
            self._keep = m
            params.decode_matrix = m.ctypes.data
        h = ctypes.c_void_p()
        _check(lib.rcbf_plan(ctypes.byref(params), ctypes.byref(h)))
        params.decode_matrix = None
        params.demod_taps = None
        params.demod_taps_imag = None
        params.tx_angles = None
        self.handle = h
        self.params = params

    # sizes
    @property
    def rf_shape(self):
        p = self.params
        return (p.n_tx, p.n_ch, p.n_samples)

    @property
    def image_shape(self):
        p = self.params
        return (p.out_dims[2], p.out_dims[1], p.out_dims[0])

    def close(self):
        if getattr(self, "handle", None):
            load_library().rcbf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        """rcbf_plan_query as a dict."""
        pi = PlanInfo()
        _check(load_library().rcbf_plan_query(self.handle, ctypes.byref(pi)))
        return {"tile": tuple(pi.tile), "tiled": bool(pi.tiled), "window": pi.window,
                "n_split": pi.n_split, "das_launches": pi.das_launches,
                "decode_launches": pi.decode_launches, "workspace_bytes": pi.workspace_bytes,
                "bwd_tile": tuple(pi.bwd_tile), "bwd_mode": pi.bwd_mode}

    def status(self, stream=None) -> int:
        """rcbf_plan_status: synchronise the stream and return OK or ETIMEOUT
        for the last das / das_backward call (no exception)."""
        return int(load_library().rcbf_plan_status(self.handle, _stream(stream)))

    def set_wait(self, wait_ns: int, withhold: int = 0):
        """rcbf_plan_set_wait: bound of the tiled kernels' waits; withhold = 1
        is the test hook that makes every tiled DAS unit's first wait expire."""
        _check(load_library().rcbf_plan_set_wait(self.handle, int(wait_ns), int(withhold)))

    def decoded_torch_dtype(self):
        import torch
        return {I32: torch.int32, F32: torch.float32, F16: torch.float16, CF32: torch.float32}[
            self.params.decoded_dtype]

    def demodulate(self, rf, out=None, stream=None):
        """rcbf_demodulate: raw int16 [n_tx][n_ch][n_s * D] -> int16 IQ planes [2][n_tx][n_ch][n_s]."""
        import torch
        if out is None:
            out = torch.empty((2,) + self.rf_shape, dtype=torch.int16, device=rf.device)
        _check(load_library().rcbf_demodulate(self.handle, _ptr(rf), _ptr(out), _stream(stream)))
        return out

    def demod_decode(self, rf, out=None, stream=None):
        """rcbf_demod_decode: raw int16 [n_tx][n_ch][n_s * D] -> decoded FP32 planes
        [2][n_tx][n_ch][n_s] (demodulation fused into the decode)."""
        import torch
        if out is None:
            out = torch.empty((2,) + self.rf_shape, dtype=torch.float32, device=rf.device)
        _check(load_library().rcbf_demod_decode(self.handle, _ptr(rf), _ptr(out), _stream(stream)))
        return out

    def decode(self, rf, out=None, stream=None):
        """rcbf_decode: int16 [n_tx][n_ch][n_s] CUDA tensor (two planes after
        demodulation) -> decoded tensor (two FP32 planes for RCBF_CF32)."""
        import torch
        if out is None:
            shape = ((2,) if self.params.decoded_dtype == CF32 else ()) + self.rf_shape
            out = torch.empty(shape, dtype=self.decoded_torch_dtype(), device=rf.device)
        _check(load_library().rcbf_decode(self.handle, _ptr(rf), _ptr(out), _stream(stream)))
        return out

    def das(self, decoded, apod=None, c: float = 0.0, out=None, stream=None):
        """rcbf_das: decoded RF -> float32 image [nz][ny][nx] (two planes for complex)."""
        import torch
        if out is None:
            shape = self.image_shape
            if self.params.decoded_dtype == CF32:
                shape = (2,) + shape
            out = torch.empty(shape, dtype=torch.float32, device=decoded.device)
        _check(load_library().rcbf_das(self.handle, _ptr(decoded), _ptr(apod), ctypes.c_float(c),
                                       _ptr(out), _stream(stream)))
        return out

    def das_backward(self, decoded, grad_image, apod=None, c: float = 0.0, want_rf=True,
                     want_c=True, want_apod=True, stream=None, out_rf=None):
        """rcbf_das_backward: (grad_rf, grad_c, grad_apod) for dL/dimage
        (grad_rf written into ``out_rf`` when given: float32, decoded's shape)."""
        import torch
        dev = decoded.device
        if out_rf is not None:
            if out_rf.dtype != torch.float32 or tuple(out_rf.shape) != tuple(decoded.shape) or not out_rf.is_contiguous():
                raise ValueError("out_rf must be a contiguous float32 tensor of decoded's shape")
            grad_rf = out_rf
        else:
            grad_rf = torch.empty_like(decoded, dtype=torch.float32) if want_rf else None
        grad_c = torch.empty((), dtype=torch.float32, device=dev) if want_c else None
        grad_apod = torch.empty(self.params.n_ch, dtype=torch.float32, device=dev) if want_apod else None
        _check(load_library().rcbf_das_backward(self.handle, _ptr(decoded), _ptr(apod), ctypes.c_float(c),
                                                _ptr(grad_image), _ptr(grad_rf), _ptr(grad_c),
                                                _ptr(grad_apod), _stream(stream)))
        return grad_rf, grad_c, grad_apod


class Pipeline:
    """Owns an ``rcbf_pipeline_t``: the upload ring. ``submit`` takes per-frame
    host tensors (inputs: int16 RF for encoded plans, else decoded data;
    outputs: float32 images), enqueues upload, batch and read-back, and returns
    at once; ``wait`` blocks until every submitted step is done."""

    def __init__(self, plans: Sequence["Plan"], n_slots: int = 3):
        lib = load_library()
        n = len(plans)
        self._plans = list(plans)
        self._n = n
        hp = (_P * n)(*[p.handle for p in plans])
        h = _P()
        _check(lib.rcbf_pipeline_create(hp, n, int(n_slots), ctypes.byref(h)))
        self.handle = h
        self._held = []            # host tensors of steps in flight

    def submit(self, host_inputs, host_images):
        if len(host_inputs) != self._n or len(host_images) != self._n:
            raise ValueError("one input and one image per frame")
        for t in list(host_inputs) + list(host_images):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("host buffers must be contiguous CPU tensors")
        ins = (_P * self._n)(*[_P(t.data_ptr()) for t in host_inputs])
        outs = (_P * self._n)(*[_P(t.data_ptr()) for t in host_images])
        self._held.append((list(host_inputs), list(host_images)))
        _check(load_library().rcbf_pipeline_submit(self.handle, ins, outs))

    def wait(self):
        try:
            _check(load_library().rcbf_pipeline_wait(self.handle))
        finally:
            self._held.clear()

    def close(self):
        if getattr(self, "handle", None):
            load_library().rcbf_pipeline_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns an ``rcbf_batch_t``: frames bound to fixed device buffers, run as
    one persistent launch per (window class, tile extent) phase (capturable
    in a CUDA graph)."""

    def __init__(self, plans: Sequence[Plan], rf, decoded, images):
        lib = load_library()
        n = len(plans)
        P = ctypes.c_void_p
        self._plans = list(plans)
        self._bufs = (None if rf is None else list(rf), list(decoded), list(images))
        arr = lambda xs: (P * n)(*[P(0 if x is None else x.data_ptr()) for x in xs])
        hp = (P * n)(*[p.handle for p in plans])
        h = P()
        rf_arr = arr(rf) if rf is not None else None
        _check(lib.rcbf_batch_create(hp, n, rf_arr, arr(decoded), arr(images), ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        _check(load_library().rcbf_batch_run(self.handle, _stream(stream)))

    def status(self, stream=None) -> int:
        """Synchronise the stream and return OK or ETIMEOUT (no exception)."""
        return int(load_library().rcbf_batch_status(self.handle, _stream(stream)))

    def set_wait(self, wait_ns: int, withhold_frame: int = -1):
        """rcbf_batch_set_wait: bound of the per-frame decode wait; the
        withhold_frame test hook makes one frame's wait expire."""
        _check(load_library().rcbf_batch_set_wait(self.handle, int(wait_ns), int(withhold_frame)))

    def close(self):
        if getattr(self, "handle", None):
            load_library().rcbf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> str:
    return load_library().rcbf_version().decode()


def measure_ceilings(stream=None) -> dict:
    """On-chip ceilings of the current device measured by microbenchmark
    kernels at the tiled DAS kernel's occupancy (rcbf_measure_ceilings)."""
    out = Ceilings()
    _check(load_library().rcbf_measure_ceilings(ctypes.byref(out), _stream(stream)))
    return {name: getattr(out, name) for name, _ in Ceilings._fields_}


def _make_das_function():
    import torch

    class DASFunction(torch.autograd.Function):
        """Differentiable DAS: image = rcbf_das(decoded, apod, c). The backward
        pass calls rcbf_das_backward (the hand-written adjoint kernel) for the
        gradients with respect to the decoded RF, the per-channel apodization
        weights and the speed of sound. decoded: float32 [n_tx][n_ch][n_s]
        (or [2][...] planes for a complex plan); apod: float32 [n_ch]; c:
        float32 scalar tensor."""

        @staticmethod
        def forward(ctx, decoded, apod, c, plan):
            ctx.plan = plan
            ctx.save_for_backward(decoded, apod, c)
            return plan.das(decoded.contiguous(), apod=apod.contiguous(), c=float(c.item()))

        @staticmethod
        def backward(ctx, grad_image):
            decoded, apod, c = ctx.saved_tensors
            plan = ctx.plan
            g_rf, g_c, g_w = plan.das_backward(decoded.contiguous(), grad_image.contiguous(),
                                               apod=apod.contiguous(), c=float(c.item()),
                                               want_rf=ctx.needs_input_grad[0],
                                               want_apod=ctx.needs_input_grad[1],
                                               want_c=ctx.needs_input_grad[2])
            return g_rf, g_w, (g_c.reshape(c.shape) if g_c is not None else None), None

    return DASFunction


_DAS_FUNCTION = None


def das_autograd(plan: Plan, decoded, apod, c):
    """image = DAS(decoded; apod, c) with gradients through the adjoint kernel."""
    global _DAS_FUNCTION
    if _DAS_FUNCTION is None:
        _DAS_FUNCTION = _make_das_function()
    return _DAS_FUNCTION.apply(decoded, apod, c, plan)


def envelope_loss(image):
    """Autofocus loss: minus the summed squared envelope, -sum |I|^2 (image as
    two planes [2][...] for a complex plan, or one real plane)."""
    return -(image * image).sum()
