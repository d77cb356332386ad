"""Seeded synthetic acquisitions for the row-column / TOBE beamformer.

This module simulates what an acquisition produces; it holds none of the
beamformer's own arithmetic (no decode, no interpolation, no aperture sums at
image points). Both the CPU oracle (``oracle/``) and the CUDA path read the
arrays it returns, so it is the only code the two share.

Forward model (the physics the beamformer inverts):

* Line elements of a row-column (TOBE) array: transmit element i at lateral
  coordinate e_i = (i - (n_tx-1)/2) * pitch, receive element j at
  e_j = (j - (n_ch-1)/2) * pitch, both at z = 0 (array centred at the origin).
  A row element's lateral coordinate is y, a column element's is x.
* A point scatterer at p echoes the emission of transmit line i into receive
  line j after tau_ij = (|p - line_i| + |p - line_j|) / c, the distance to a
  line element being sqrt((lateral(p) - e)^2 + z^2) (synthetic-aperture model,
  §THEORY "Synthetic Aperture Imaging").
* Echo shape: a Gaussian-windowed two-cycle sinusoid
  e(t) = cos(2 pi fc t) * exp(-t^2 / (2 sigma^2)), FWHM = 2 cycles, truncated at
  |t| <= 4 sigma; the analytic (complex) form replaces cos by exp(+j 2 pi fc t).
* Hadamard aperture encoding across acquisitions: s_k = sum_i H[k, i] r_i
  (§THEORY "Synthetic Aperture Imaging", FORCES / HERCULES), with H the
  Sylvester matrix built here by Kronecker products.
* Noise and quantisation: Gaussian noise of sigma = 1 % of max|s| is added,
  the result scaled so that max|s + n| = 20000 and rounded half-to-even to
  int16 (the receive system's 16-bit samples).

All random draws come from numpy's PCG64 ``default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

MM = 1e-3

ROWS, COLUMNS = 0, 1
FORCES, HERCULES, HERCULES_2D = 0, 1, 2     # HERCULES_2D: decoded rows x columns = a 2D receive aperture


def sylvester_kron(n: int) -> np.ndarray:
    """Sylvester Hadamard matrix of order n (a power of two) by repeated
    Kronecker products with [[1, 1], [1, -1]]; int64."""
    if n < 1 or n & (n - 1):
        raise ValueError("Sylvester order must be a power of two")
    h = np.ones((1, 1), dtype=np.int64)
    base = np.array([[1, 1], [1, -1]], dtype=np.int64)
    while h.shape[0] < n:
        h = np.kron(base, h)
    return h


@dataclasses.dataclass
class Geometry:
    """Acquisition and image description of one frame (SI units)."""
    n_tx: int
    n_ch: int
    n_samples: int
    fs: float = 30e6
    fc: float = 7.5e6
    c: float = 1540.0
    t0: float = 0.0
    tx_pitch: float = 0.1 * MM
    rx_pitch: float = 0.1 * MM
    tx_orientation: int = ROWS
    rx_orientation: int = COLUMNS
    acq_kind: int = FORCES
    hadamard_order: int = 0          # 0: not encoded
    out_dims: Tuple[int, int, int] = (128, 1, 128)   # nx, ny, nz
    out_min: Tuple[float, float, float] = (-2.5 * MM, 0.0, 4 * MM)
    out_max: Tuple[float, float, float] = (2.5 * MM, 0.0, 25 * MM)
    f_number: float = 0.0
    interp: str = "linear"           # sample interpolation of the beamformer: linear or cubic
    iq_freq: float = 0.0             # > 0: the beamformed data is baseband IQ demodulated at this frequency
    tx_wave: str = "line"            # transmit wave of each transmit index: line, plane or vls
    tx_angles: Tuple[float, ...] = ()    # plane-wave angles [rad], one per transmit
    tx_focus: float = 0.0            # virtual line source depth [m]

    @property
    def n_vox(self) -> int:
        return int(self.out_dims[0] * self.out_dims[1] * self.out_dims[2])

    @property
    def sums(self) -> int:
        """voxel x channel x transmit terms of one DAS pass."""
        return self.n_vox * self.n_ch * self.n_tx

    def tx_positions(self) -> np.ndarray:
        return (np.arange(self.n_tx) - (self.n_tx - 1) / 2.0) * self.tx_pitch

    def rx_positions(self) -> np.ndarray:
        return (np.arange(self.n_ch) - (self.n_ch - 1) / 2.0) * self.rx_pitch


def _lateral(p: np.ndarray, orientation: int) -> np.ndarray:
    # a row element spans x, so its lateral coordinate is y; a column's is x
    return p[..., 1] if orientation == ROWS else p[..., 0]


def echo_sigma(fc: float) -> float:
    """Gaussian sigma whose FWHM equals two cycles of fc."""
    return 2.0 / (fc * 2.0 * math.sqrt(2.0 * math.log(2.0)))


def _transmit_path(g: Geometry, e_tx: np.ndarray, lt: float, z: float) -> np.ndarray:
    """Acquisition physics of each transmit wave: a line element radiates a
    cylinder, a steered plane wave crosses the array at t = 0, a virtual line
    source converges at depth f and diverges below it."""
    if g.tx_wave == "plane":
        th = np.asarray(g.tx_angles, dtype=np.float64)
        return z * np.cos(th) + lt * np.sin(th)
    if g.tx_wave == "vls":
        dz = z - g.tx_focus
        return g.tx_focus + (1.0 if dz >= 0 else -1.0) * np.sqrt((lt - e_tx) ** 2 + dz * dz)
    return np.sqrt((lt - e_tx) ** 2 + z * z)


def _accumulate_echoes(g: Geometry, scatterers: np.ndarray, c: float,
                       analytic: bool) -> np.ndarray:
    """Un-encoded traces r[i, j, n] (float64 or complex128) of unit-amplitude
    point scatterers, one Gaussian-windowed echo per (scatterer, i, j)."""
    dtype = np.complex128 if analytic else np.float64
    r = np.zeros((g.n_tx, g.n_ch, g.n_samples), dtype=dtype)
    sig = echo_sigma(g.fc)
    half = int(math.ceil(4.0 * sig * g.fs)) + 1
    k = np.arange(-half, half + 1)
    e_tx = g.tx_positions()
    e_rx = g.rx_positions()
    ii, jj = np.meshgrid(np.arange(g.n_tx), np.arange(g.n_ch), indexing="ij")
    for p in scatterers:
        lt = _lateral(p, g.tx_orientation)
        lr = _lateral(p, g.rx_orientation)
        z = p[2]
        if g.acq_kind == HERCULES_2D:
            # one transmit wave; receive on the 2D aperture (row i, column j)
            if g.tx_wave == "plane":
                a = float(g.tx_angles[0])
                d_wave = z * math.cos(a) + lt * math.sin(a)
            else:
                d_wave = math.sqrt(p[0] ** 2 + p[1] ** 2 + (z - g.tx_focus) ** 2) + g.tx_focus
            rx2 = np.sqrt((lr - e_rx[None, :]) ** 2 + (lt - e_tx[:, None]) ** 2 + z * z)   # [n_tx, n_ch]
            tau = (d_wave + rx2) / c
        else:
            dist_tx = _transmit_path(g, e_tx, lt, z)             # [n_tx]
            dist_rx = np.sqrt((lr - e_rx) ** 2 + z * z)          # [n_ch]
            tau = (dist_tx[:, None] + dist_rx[None, :]) / c      # [n_tx, n_ch]
        centre = np.floor((tau - g.t0) * g.fs).astype(np.int64)
        n = centre[:, :, None] + k[None, None, :]            # [n_tx, n_ch, K]
        t = g.t0 + n / g.fs - tau[:, :, None]
        env = np.exp(-(t * t) / (2.0 * sig * sig))
        env[np.abs(t) > 4.0 * sig] = 0.0
        if analytic:
            val = env * np.exp(1j * 2.0 * math.pi * g.fc * t)
        else:
            val = env * np.cos(2.0 * math.pi * g.fc * t)
        ok = (n >= 0) & (n < g.n_samples)
        I = np.broadcast_to(ii[:, :, None], n.shape)[ok]
        J = np.broadcast_to(jj[:, :, None], n.shape)[ok]
        # one scatterer never hits the same (i, j, n) twice, so plain fancy
        # indexing accumulates correctly
        r[I, J, n[ok]] += val[ok]
    return r


def draw_scatterers(rng: np.random.Generator, count: int,
                    x: Tuple[float, float], y: Tuple[float, float],
                    z: Tuple[float, float]) -> np.ndarray:
    xs = rng.uniform(x[0], x[1], count)
    ys = rng.uniform(y[0], y[1], count) if y[1] > y[0] else np.full(count, y[0])
    zs = rng.uniform(z[0], z[1], count)
    return np.stack([xs, ys, zs], axis=1)


@dataclasses.dataclass
class Frame:
    geometry: Geometry
    rf: Optional[np.ndarray]           # int16 [n_tx][n_ch][n_s] encoded (None if not encoded)
    decoded: Optional[np.ndarray]      # float32 or complex64 un-encoded traces (non-encoded frames)
    scatterers: np.ndarray             # [count, 3] metres
    seed: int


def encode_quantise(g: Geometry, r: np.ndarray, rng: np.random.Generator,
                    noise_frac: float = 0.01, peak: float = 20000.0) -> np.ndarray:
    """s = H r across acquisitions, plus noise, scaled to +-peak, rounded
    half-to-even to int16."""
    h = sylvester_kron(g.n_tx).astype(np.float64)
    flat = r.reshape(g.n_tx, -1)
    s = h @ flat
    amax = float(np.max(np.abs(s)))
    if amax > 0 and noise_frac > 0:
        s += rng.normal(0.0, noise_frac * amax, size=s.shape)
    amax = float(np.max(np.abs(s)))
    if amax > 0:
        s *= peak / amax
    q = np.rint(s)  # numpy rint rounds half to even
    q = np.clip(q, -32768, 32767)
    return q.astype(np.int16).reshape(r.shape)


def make_frame(g: Geometry, seed: int, n_scatterers: int,
               box_x=(-2 * MM, 2 * MM), box_y=(0.0, 0.0), box_z=(5 * MM, 25 * MM),
               c_true: Optional[float] = None, analytic: bool = False,
               noise_frac: float = 0.01) -> Frame:
    rng = np.random.default_rng(seed)
    sc = draw_scatterers(rng, n_scatterers, box_x, box_y, box_z)
    r = _accumulate_echoes(g, sc, c_true if c_true else g.c, analytic)
    if g.hadamard_order:
        rf = encode_quantise(g, r, rng, noise_frac=noise_frac)
        return Frame(g, rf, None, sc, seed)
    dec = r.astype(np.complex64 if analytic else np.float32)
    return Frame(g, None, dec, sc, seed)


def lowpass_taps(n_taps: int, cutoff: float, shift: int = 15) -> np.ndarray:
    """Demodulation filter input: Hann-windowed sinc low-pass with cutoff in
    cycles per raw sample, unit DC gain in Q(shift), rounded to int16."""
    k = np.arange(n_taps) - (n_taps - 1) / 2
    h = np.sinc(2 * cutoff * k) * np.hanning(n_taps + 2)[1:-1]
    h = h / h.sum() * (1 << shift)
    return np.round(h).astype(np.int16)


# ---------------------------------------------------------------------------
# Workloads of the paper's configurations (sizes as the build's configs state;
# grid extents and unstated constants as read in the design notes).
# ---------------------------------------------------------------------------

def tiny_bscan_geometry() -> Geometry:
    """FORCES B-scan, 32 tx x 32 ch x 1024 samples, 128 x 128 image."""
    return Geometry(n_tx=32, n_ch=32, n_samples=1024, hadamard_order=32,
                    out_dims=(128, 1, 128), out_min=(-2.5 * MM, 0.0, 4 * MM),
                    out_max=(2.5 * MM, 0.0, 25 * MM))


def full_bscan_geometry() -> Geometry:
    """FORCES B-scan, 128 tx x 128 ch x 4096 samples, 512 (x) x 1024 (z) image."""
    return Geometry(n_tx=128, n_ch=128, n_samples=4096, hadamard_order=128,
                    out_dims=(512, 1, 1024), out_min=(-6.4 * MM, 0.0, 3 * MM),
                    out_max=(6.4 * MM, 0.0, 27 * MM))


def hercules_volume_geometry() -> Geometry:
    """HERCULES volume, 128 tx x 128 ch x 2048 samples, 128 x 128 x 256 voxels."""
    return Geometry(n_tx=128, n_ch=128, n_samples=2048, hadamard_order=128,
                    acq_kind=HERCULES, out_dims=(128, 128, 256),
                    out_min=(-6.4 * MM, -6.4 * MM, 5 * MM),
                    out_max=(6.4 * MM, 6.4 * MM, 25 * MM))


def autofocus_geometry() -> Geometry:
    """Complex decoded RF 128 x 128 x 2048, 256 x 512 image at c = 1540 m/s."""
    return Geometry(n_tx=128, n_ch=128, n_samples=2048, hadamard_order=0,
                    out_dims=(256, 1, 512), out_min=(-6.4 * MM, 0.0, 3 * MM),
                    out_max=(6.4 * MM, 0.0, 27 * MM))


def tiny_bscan(seed: int = 1) -> Frame:
    return make_frame(tiny_bscan_geometry(), seed, 8)


def full_bscan(seed: int = 2) -> Frame:
    return make_frame(full_bscan_geometry(), seed, 64)


def hercules_volume(seed: int = 3) -> Frame:
    return make_frame(hercules_volume_geometry(), seed, 256,
                      box_x=(-6.4 * MM, 6.4 * MM), box_y=(-6.4 * MM, 6.4 * MM))


def autofocus(seed: int = 5, c_true: float = 1480.0) -> Frame:
    return make_frame(autofocus_geometry(), seed, 32, c_true=c_true,
                      analytic=True, noise_frac=0.0)


def stream_geometries() -> List[Tuple[Geometry, int, dict]]:
    """The 64-frame realtime stream: frames 0-31 FORCES B-scans with n_tx
    cycling {32, 64, 128}, n_s cycling {2048, 3072, 4096} and grids cycling
    {256x512, 512x512, 512x1024}; frames 32-63 are 16 cross-plane pairs
    (128 x 128 x 2048, 256 x 512 each), the second plane with transmit and
    receive orientations swapped and imaged in the y-z plane.
    Returns (geometry, seed, scatterer-box kwargs) per frame."""
    out = []
    ntx = (32, 64, 128)
    ns = (2048, 3072, 4096)
    grids = ((256, 512), (512, 512), (512, 1024))
    for f in range(32):
        nx, nz = grids[f % 3]
        g = Geometry(n_tx=ntx[f % 3], n_ch=128, n_samples=ns[(f // 3) % 3],
                     hadamard_order=ntx[f % 3], out_dims=(nx, 1, nz),
                     out_min=(-6.4 * MM, 0.0, 3 * MM), out_max=(6.4 * MM, 0.0, 27 * MM))
        out.append((g, 1000 + f, dict()))
    for p in range(16):
        for side in range(2):
            f = 32 + 2 * p + side
            if side == 0:
                g = Geometry(n_tx=128, n_ch=128, n_samples=2048, hadamard_order=128,
                             out_dims=(256, 1, 512), out_min=(-6.4 * MM, 0.0, 3 * MM),
                             out_max=(6.4 * MM, 0.0, 27 * MM))
            else:
                g = Geometry(n_tx=128, n_ch=128, n_samples=2048, hadamard_order=128,
                             tx_orientation=COLUMNS, rx_orientation=ROWS,
                             out_dims=(1, 256, 512), out_min=(0.0, -6.4 * MM, 3 * MM),
                             out_max=(0.0, 6.4 * MM, 27 * MM))
            out.append((g, 1000 + f, dict(box_y=(-2 * MM, 2 * MM))))
    return out


def stream_frame(index: int, n_scatterers: int = 16) -> Frame:
    g, seed, box = stream_geometries()[index]
    return make_frame(g, seed, n_scatterers, **box)


def random_int_rf(n_tx: int, n_ch: int, n_s: int, seed: int,
                  lo: int = -32768, hi: int = 32767) -> np.ndarray:
    """Uniform random int16 RF (edge cases: full int16 range)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(n_tx, n_ch, n_s), dtype=np.int64).astype(np.int16)
