"""Pins of the FP64 CPU oracle against facts that do not come from the oracle
itself: textbook Hadamard values and identities, hand-computed times of
flight, closed forms of the DAS sum for constant and ramp data, symmetry,
exact linearity, brute force, and the adjoint identity. CPU only."""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
from oracle import twin
import synth
from synth import Geometry, MM, ROWS, COLUMNS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


# ------------------------------------------------------------- Hadamard

def test_hadamard_h4_golden():
    expect = np.array(_golden_rows("hadamard_sylvester_h4.txt"), dtype=np.int8)
    np.testing.assert_array_equal(oracle.hadamard(4), expect)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256])
def test_hadamard_orthogonal(n):
    H = oracle.hadamard(n).astype(np.int64)
    np.testing.assert_array_equal(H @ H.T, n * np.eye(n, dtype=np.int64))
    np.testing.assert_array_equal(H, H.T)                     # Sylvester H is symmetric
    assert set(np.unique(H)) <= {-1, 1}


@pytest.mark.parametrize("n", [2, 8, 64, 256])
def test_hadamard_matches_kronecker_construction(n):
    # the popcount form and the doubling construction are the same matrix
    np.testing.assert_array_equal(oracle.hadamard(n).astype(np.int64), synth.sylvester_kron(n))


# --------------------------------------------------------------- decode

@pytest.mark.parametrize("n,cols", [(32, 1), (32, 1000), (64, 777), (128, 4096), (256, 96)])
def test_decode_brute_force(n, cols):
    rng = np.random.default_rng(n * 7 + cols)
    S = rng.integers(-32768, 32768, size=(n, cols)).astype(np.int16)
    D = oracle.decode(S)
    H = synth.sylvester_kron(n)
    np.testing.assert_array_equal(D, H.T @ S.astype(np.int64))


def test_decode_twin_tiny():
    rng = np.random.default_rng(3)
    S = rng.integers(-32768, 32768, size=(8, 5)).astype(np.int16)
    np.testing.assert_array_equal(oracle.decode(S), np.array(twin.decode(S.astype(int).tolist())))


@pytest.mark.parametrize("n", [32, 64, 128, 256])
def test_decode_round_trip_recovers_unencoded(n):
    # integer un-encoded data r small enough that the encoded s = H r fits
    # int16; decoding must return n * r bit-exactly (H^T H = n I)
    rng = np.random.default_rng(n)
    lim = 32767 // n
    r = rng.integers(-lim, lim + 1, size=(n, 3, 50)).astype(np.int64)
    H = synth.sylvester_kron(n)
    s = np.einsum("ki,ics->kcs", H, r)
    assert np.abs(s).max() <= 32767
    D = oracle.decode(s.astype(np.int16))
    np.testing.assert_array_equal(D, n * r)


def test_decode_custom_matrix():
    # any +-1 matrix: a column-sign-flipped, row-permuted Sylvester matrix
    rng = np.random.default_rng(11)
    H = synth.sylvester_kron(32)[rng.permutation(32)] * rng.choice([-1, 1], 32)[None, :]
    S = rng.integers(-32768, 32768, size=(32, 100)).astype(np.int16)
    D = oracle.decode(S, H.astype(np.int8))
    np.testing.assert_array_equal(D, H.T @ S.astype(np.int64))


def test_decoded_dtype_rounding():
    n = 128
    D = np.array([2049 * n, 2051 * n, -2049 * n, 3 * n + 64, 2**22, -(2**22)], dtype=np.int64)
    f16 = oracle.decoded_as(D, n, "f16").astype(np.float64)
    # float16 keeps 11 significant bits: 2049 and 2051 are ties -> nearest even
    np.testing.assert_array_equal(f16[:3], [2048.0, 2052.0, -2048.0])
    assert f16[3] == 3.5
    f32 = oracle.decoded_as(D, n, "f32").astype(np.float64)
    np.testing.assert_array_equal(f32 * n, D.astype(np.float64))   # exact
    np.testing.assert_array_equal(oracle.decoded_as(D, n, "i32"), D.astype(np.int32))


# ------------------------------------------------------------------ DAS

def _point_geom(x, y, z, t0=0.0, n_s=1000):
    return Geometry(n_tx=1, n_ch=1, n_samples=n_s, fs=10e6, c=1500.0, t0=t0,
                    tx_orientation=ROWS, rx_orientation=COLUMNS,
                    out_dims=(1, 1, 1), out_min=(x, y, z), out_max=(x, y, z))


def test_hand_computed_time_of_flight():
    for x, y, z, t0_us, expect in _golden_rows("pythagorean_tof.txt"):
        g = _point_geom(x * MM, y * MM, z * MM, t0=t0_us * 1e-6)
        ramp = np.arange(g.n_samples, dtype=np.float64).reshape(1, 1, -1)
        img = oracle.das(g, ramp)
        assert img.ravel()[0] == pytest.approx(expect, rel=0, abs=1e-9)


def test_orientation_swap_uses_the_other_coordinate():
    # transmit on columns (lateral x) and receive on rows (lateral y): the
    # 3-4-5 voxel (x=3, y=0, z=4) now has d_tx = 5, d_rx = 4 -> still s = 60,
    # while (x=3, y=3, z=4) gives 5 + 5 = 10 mm -> s = 66.67
    g = _point_geom(3 * MM, 3 * MM, 4 * MM)
    g.tx_orientation, g.rx_orientation = COLUMNS, ROWS
    ramp = np.arange(g.n_samples, dtype=np.float64).reshape(1, 1, -1)
    assert oracle.das(g, ramp).ravel()[0] == pytest.approx(10e-3 / 1500 * 10e6, abs=1e-9)


def test_fractional_sample_weights():
    # s = 60 + 1/4 -> weights 3/4 on sample 60 and 1/4 on sample 61
    g = _point_geom(3 * MM, 0.0, 4 * MM, t0=-0.025e-6)
    for n, expect in ((60, 0.75), (61, 0.25), (59, 0.0), (62, 0.0)):
        r = np.zeros((1, 1, g.n_samples))
        r[0, 0, n] = 1.0
        assert oracle.das(g, r).ravel()[0] == pytest.approx(expect, abs=1e-12)


def test_zero_outside_record():
    g = _point_geom(3 * MM, 0.0, 4 * MM, n_s=60)   # s = 60 is one past the last sample
    r = np.ones((1, 1, 60))
    assert oracle.das(g, r).ravel()[0] == 0.0
    g = _point_geom(3 * MM, 0.0, 4 * MM, t0=6.05e-6, n_s=10)   # s = -0.5: half of r[0]
    assert oracle.das(g, np.ones((1, 1, 10))).ravel()[0] == pytest.approx(0.5, abs=1e-12)


# ------------------------------------------------------- transmit waves

def test_transmit_waves_hand_computed_delays():
    for x, y, z, wave, ang, focus, expect in _golden_rows("transmit_waves.txt"):
        g = _point_geom(x * MM, y * MM, z * MM)
        if int(wave) == 1:
            g.tx_wave, g.tx_angles = "plane", (np.deg2rad(ang),)
        else:
            g.tx_wave, g.tx_focus = "vls", focus * MM
        ramp = np.arange(g.n_samples, dtype=np.float64).reshape(1, 1, -1)
        assert oracle.das(g, ramp).ravel()[0] == pytest.approx(expect, rel=0, abs=1e-9)


def test_plane_wave_at_zero_angle_and_vls_on_axis_equal_depth():
    # a 0-degree plane wave and a virtual line source directly above the point
    # both travel exactly z on transmit (the line element too, on its axis)
    rng = np.random.default_rng(15)
    r = rng.normal(size=(1, 1, 1000))
    g = _point_geom(2.5 * MM, 0.0, 7.0 * MM)
    want = oracle.das(g, r).ravel()[0]
    g.tx_wave, g.tx_angles = "plane", (0.0,)
    assert oracle.das(g, r).ravel()[0] == pytest.approx(want, abs=1e-12)
    for f in (3 * MM, 7 * MM, 11 * MM):
        g.tx_wave, g.tx_focus = "vls", f
        assert oracle.das(g, r).ravel()[0] == pytest.approx(want, abs=1e-12)


def test_hercules_2d_receive_hand_computed_delays():
    # one row (lateral y = 0) and one column (lateral x = 0); the point
    # (x, y, z) = (3, 4, 12) mm is 13 mm from the 2D element (x_j, y_i) = (0, 0)
    g = _point_geom(3 * MM, 4 * MM, 12 * MM)
    g.acq_kind = synth.HERCULES_2D
    ramp = np.arange(g.n_samples, dtype=np.float64).reshape(1, 1, -1)
    g.tx_wave, g.tx_angles = "plane", (0.0,)        # d_tx = z = 12 -> 25 mm -> s = 166.666...
    assert oracle.das(g, ramp).ravel()[0] == pytest.approx(25e-3 / 1500 * 10e6, abs=1e-9)
    # a diverging wave from a virtual point at depth -5 mm on the axis:
    # d_tx = sqrt(3^2 + 4^2 + 17^2) - 5 = 12.72004514666935 -> 25.72004514666935 mm
    g.tx_wave, g.tx_focus = "point", -5 * MM
    assert oracle.das(g, ramp).ravel()[0] == pytest.approx(171.4669676444623, abs=1e-9)


def test_hercules_2d_with_one_row_on_the_image_plane_equals_the_separable_form():
    # one receive row at lateral 0 and a B-scan in its plane (y = 0): the 2D
    # element distance reduces to the line-element distance, so the image is
    # that of the separable plane-wave form with one transmit
    g = _small_geom(n_tx=1, n_ch=6, dims=(7, 1, 9))
    g.tx_wave, g.tx_angles = "plane", (0.2,)
    r = np.random.default_rng(16).normal(size=(1, 6, g.n_samples))
    sep = oracle.das(g, r, w=np.linspace(0.5, 1.5, 6))
    g.acq_kind = synth.HERCULES_2D
    np.testing.assert_allclose(oracle.das(g, r, w=np.linspace(0.5, 1.5, 6)), sep, rtol=0, atol=1e-12)


# -------------------------------------------- cubic Hermite interpolation

def test_cubic_weights_at_a_quarter_sample():
    # s = 60 + 1/4. The 4-point cubic Hermite spline with central-difference
    # slopes weights samples 59..62 by -(1/2) h10, h00 - (1/2) h11,
    # h01 + (1/2) h10, (1/2) h11 at f = 1/4 (h00 = 27/32, h10 = 9/64,
    # h01 = 5/32, h11 = -3/64): -9/128, 111/128, 29/128, -3/128
    g = _point_geom(3 * MM, 0.0, 4 * MM, t0=-0.025e-6)
    g.interp = "cubic"
    for n, expect in ((59, -9 / 128), (60, 111 / 128), (61, 29 / 128), (62, -3 / 128), (58, 0.0), (63, 0.0)):
        r = np.zeros((1, 1, g.n_samples))
        r[0, 0, n] = 1.0
        assert oracle.das(g, r).ravel()[0] == pytest.approx(expect, abs=1e-12)


def test_cubic_interpolates_the_samples():
    # s = 60 exactly (3-4-5 triangle): the spline passes through r[60]
    g = _point_geom(3 * MM, 0.0, 4 * MM)
    g.interp = "cubic"
    r = np.random.default_rng(11).normal(size=(1, 1, g.n_samples))
    assert oracle.das(g, r).ravel()[0] == pytest.approx(r[0, 0, 60], abs=1e-12)


def test_cubic_reproduces_quadratics_at_hand_computed_delays():
    # central-difference Hermite splines are exact for polynomials of degree
    # <= 2: quadratic data returns the quadratic at the delay s of each
    # hand-computed geometry
    for x, y, z, t0_us, s in _golden_rows("pythagorean_tof.txt"):
        g = _point_geom(x * MM, y * MM, z * MM, t0=t0_us * 1e-6)
        g.interp = "cubic"
        n = np.arange(g.n_samples, dtype=np.float64)
        r = (0.3 * n * n - 2.0 * n + 5.0).reshape(1, 1, -1)
        want = 0.3 * s * s - 2.0 * s + 5.0
        assert oracle.das(g, r).ravel()[0] == pytest.approx(want, rel=1e-12, abs=1e-9)


def test_cubic_matches_scipy_hermite_spline_including_record_ends():
    # one transmit row and one receive column through the origin: a voxel at
    # (0, 0, z) is z from both, so s = 2 z fs / c - t0 fs. The delays sweep
    # the whole record and one sample past each end; the reference is scipy's
    # CubicHermiteSpline through the zero-extended trace with central
    # differences as the knot slopes.
    interp = pytest.importorskip("scipy.interpolate")
    n_s = 64
    fs, c = 10e6, 1500.0
    t0 = 2 * (1.0 * MM) / c + 3.0 / fs               # s = -3 at z = 1 mm
    z1 = 0.5 * c * ((n_s + 2) / fs + t0)               # s = n_s + 2 at the far end
    g = Geometry(n_tx=1, n_ch=1, n_samples=n_s, fs=fs, c=c, t0=t0, out_dims=(1, 1, 997),
                 out_min=(0.0, 0.0, 1.0 * MM), out_max=(0.0, 0.0, z1), interp="cubic")
    r = np.random.default_rng(12).normal(size=n_s)
    img = oracle.das(g, r.reshape(1, 1, -1)).ravel()
    z = np.linspace(1.0 * MM, z1, 997)
    s = 2 * z * fs / c - t0 * fs
    pad = 3
    knots = np.arange(-pad, n_s + pad, dtype=np.float64)
    vals = np.concatenate([np.zeros(pad), r, np.zeros(pad)])
    slopes = np.zeros_like(vals)
    slopes[1:-1] = 0.5 * (vals[2:] - vals[:-2])
    spline = interp.CubicHermiteSpline(knots, vals, slopes)
    want = spline(s)
    assert s.min() < -2.5 and s.max() > n_s + 1.5
    np.testing.assert_allclose(img, want, rtol=0, atol=1e-12)


# ------------------------------------------------- demodulation (Eq. demod)

def test_demod_impulse_response_is_the_mixed_tap_sequence():
    # an FIR's response to an impulse is its tap sequence; the quadrature mixer
    # e^{-j pi n / 2} at n = 13 (13 mod 4 = 1) is -j; decimation by 2 keeps the
    # outputs at n = 2 m, so output m sees tap 2 m - 13
    h = np.array([3, -7, 11, 2, -5, 9, 1, -4, 6], dtype=np.int16)
    s = np.zeros((1, 64), dtype=np.int16)
    s[0, 13] = 8
    iq = oracle.demodulate(s, h, shift=3, decimation=2)
    assert iq.shape == (2, 1, 32)
    for m in range(32):
        k = 2 * m - 13
        want = -int(h[k]) if 0 <= k < h.size else 0
        assert iq[0, 0, m] == 0 and iq[1, 0, m] == want
    s[0, 13], s[0, 12] = 0, 8                       # 12 mod 4 = 0: mixer 1 -> I plane
    iq = oracle.demodulate(s, h, shift=3, decimation=2)
    for m in range(32):
        k = 2 * m - 12
        assert iq[1, 0, m] == 0 and iq[0, 0, m] == (int(h[k]) if 0 <= k < h.size else 0)


def test_demod_tone_at_the_demodulation_frequency_goes_to_baseband():
    # s = A cos(pi n / 2) = A, 0, -A, 0, ...: mixed it is A at even n, 0 at odd
    # n, so (once the filter is full) the output is A * (sum of the even taps)
    # in I and 0 in Q; s = A sin(pi n / 2) mixes to -jA at odd n: -A * (sum of
    # the odd taps) in Q
    h = np.array([1, 2, 3, 4, 5, 4, 3, 2, 1], dtype=np.int16)
    n = np.arange(200)
    A = 100
    cos_t = (A * np.round(np.cos(np.pi * n / 2))).astype(np.int16)[None]
    sin_t = (A * np.round(np.sin(np.pi * n / 2))).astype(np.int16)[None]
    even, odd = int(h[0::2].sum()), int(h[1::2].sum())
    iq = oracle.demodulate(cos_t, h, shift=0, decimation=4)
    assert np.all(iq[0, 0, 3:] == A * even) and np.all(iq[1, 0, :] == 0)
    iq = oracle.demodulate(sin_t, h, shift=0, decimation=4)
    assert np.all(iq[1, 0, 3:] == -A * odd) and np.all(iq[0, 0, :] == 0)


def test_demod_rounding_ties_to_even_and_saturation():
    # one tap of 1, shift 1: v / 2 rounded half to even (by hand)
    vals = [3, 5, -3, -5, 7, 1, -1, 4]
    want = [2, 2, -2, -2, 4, 0, 0, 2]
    s = np.zeros((1, 4 * len(vals)), dtype=np.int16)
    s[0, 0::4] = vals                               # n mod 4 = 0: mixer 1
    iq = oracle.demodulate(s, np.array([1], dtype=np.int16), shift=1, decimation=4)
    assert list(iq[0, 0]) == want
    # a tap of 32767 with no shift saturates both ways
    s[0, 0::4] = [2, -2, 1, -1, 0, 0, 0, 0]
    iq = oracle.demodulate(s, np.array([32767], dtype=np.int16), shift=0, decimation=4)
    assert list(iq[0, 0, :4]) == [32767, -32768, 32767, -32767]


def test_iq_beamforming_restores_the_carrier_at_integer_delays():
    # at an integer delay s the interpolants return the samples, and IQ
    # beamforming multiplies (I + jQ)[s] by e^{j 2 pi (f_d / f_s) s}
    rng = np.random.default_rng(14)
    for x, y, z, t0_us, s_exact in _golden_rows("pythagorean_tof.txt"):
        if abs(s_exact - round(s_exact)) > 1e-9:
            continue
        g = _point_geom(x * MM, y * MM, z * MM, t0=t0_us * 1e-6)
        g.iq_freq = 2.5e6                             # f_d / f_s = 1/4
        iq = rng.normal(size=(1, 1, g.n_samples)) + 1j * rng.normal(size=(1, 1, g.n_samples))
        sn = int(round(s_exact))
        want = iq[0, 0, sn] * np.exp(2j * np.pi * 0.25 * sn)
        for interp in ("linear", "cubic"):
            got = oracle.das(g, iq, interp=interp).ravel()[0]
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


def _small_geom(n_tx=4, n_ch=4, n_s=256, dims=(5, 1, 6), fnum=0.0):
    return Geometry(n_tx=n_tx, n_ch=n_ch, n_samples=n_s, fs=30e6, c=1540.0,
                    out_dims=dims, out_min=(-1 * MM, 0.0, 2 * MM), out_max=(1 * MM, 0.0, 4 * MM),
                    f_number=fnum)


def test_constant_rf_closed_form():
    g = _small_geom()
    img = oracle.das(g, np.ones((g.n_tx, g.n_ch, g.n_samples)))
    np.testing.assert_allclose(img, g.n_tx * g.n_ch, rtol=0, atol=1e-12)


def test_constant_rf_hanning_closed_form():
    # receive columns at x = -0.5 mm and +0.5 mm (pitch 1 mm, 2 channels),
    # voxel at x = 0, z = 1 mm, F# = 0.5: u = 0.5 * 0.5 / 1 = 0.25 ->
    # W = cos^2(pi/4) = 1/2 per channel; two channels, one transmit -> 1.0
    g = Geometry(n_tx=1, n_ch=2, n_samples=400, fs=30e6, c=1540.0,
                 rx_pitch=1 * MM, out_dims=(1, 1, 1), out_min=(0.0, 0.0, 1 * MM),
                 out_max=(0.0, 0.0, 1 * MM), f_number=0.5)
    assert oracle.das(g, np.ones((1, 2, 400))).ravel()[0] == pytest.approx(1.0, abs=1e-12)
    g.f_number = 1.0      # u = 0.5: outside the window
    assert oracle.das(g, np.ones((1, 2, 400))).ravel()[0] == 0.0
    # per-channel weights multiply the window
    g.f_number = 0.5
    assert oracle.das(g, np.ones((1, 2, 400)), w=np.array([3.0, -1.0])).ravel()[0] == \
        pytest.approx(1.0, abs=1e-12)


def test_twin_matches_oracle_on_tiny_grid():
    g = _small_geom(fnum=0.7)
    rng = np.random.default_rng(5)
    rf = rng.normal(size=(g.n_tx, g.n_ch, g.n_samples))
    w = rng.uniform(0.5, 1.5, g.n_ch)
    a = oracle.das(g, rf, w=w, c=1500.0).ravel()
    b = np.array(twin.das(g, rf, w=w, c=1500.0))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(b).max())


def test_listed_voxels_match_full_image():
    g = _small_geom(dims=(7, 3, 5))
    rng = np.random.default_rng(6)
    rf = rng.normal(size=(g.n_tx, g.n_ch, g.n_samples))
    full = oracle.das(g, rf).ravel()
    vox = np.array([0, 3, 17, 50, 104])
    np.testing.assert_array_equal(oracle.das(g, rf, voxels=vox), full[vox])


def test_linearity_and_complex_planes():
    g = _small_geom()
    rng = np.random.default_rng(7)
    r1 = rng.normal(size=(g.n_tx, g.n_ch, g.n_samples))
    r2 = rng.normal(size=(g.n_tx, g.n_ch, g.n_samples))
    lhs = oracle.das(g, 2.0 * r1 - 3.0 * r2)
    rhs = 2.0 * oracle.das(g, r1) - 3.0 * oracle.das(g, r2)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    cimg = oracle.das(g, r1 + 1j * r2)
    np.testing.assert_allclose(cimg.real, oracle.das(g, r1), rtol=1e-15)
    np.testing.assert_allclose(cimg.imag, oracle.das(g, r2), rtol=1e-15)


def _scatterer_on_node(orientation_swap=False):
    g = Geometry(n_tx=32, n_ch=32, n_samples=1024, hadamard_order=32,
                 out_dims=(41, 1, 41), out_min=(-2 * MM, 0.0, 8 * MM),
                 out_max=(2 * MM, 0.0, 12 * MM))
    node = (27, 0, 13)         # x = 0.7 mm, z = 9.3 mm
    p = [g.out_min[d] + node[d] * (g.out_max[d] - g.out_min[d]) / max(g.out_dims[d] - 1, 1)
         for d in range(3)]
    frame = synth.make_frame(g, seed=0, n_scatterers=1, box_x=(p[0], p[0]),
                             box_z=(p[2], p[2]), noise_frac=0.0)
    return g, node, frame


def test_point_scatterer_peaks_at_its_voxel():
    g, node, frame = _scatterer_on_node()
    D = oracle.decode(frame.rf)
    r = oracle.decoded_as(D, g.n_tx, "f32").astype(np.float64)
    env = np.abs(oracle.das(g, r))
    iz, iy, ix = np.unravel_index(np.argmax(env), env.shape)
    assert (ix, iy, iz) == node


def test_mirror_symmetry_about_x0():
    # a scatterer on the axis gives receive data symmetric under j -> n-1-j;
    # on a grid symmetric about x = 0 the image is then mirror symmetric
    g = Geometry(n_tx=8, n_ch=8, n_samples=512, out_dims=(9, 1, 7),
                 out_min=(-1 * MM, 0.0, 4 * MM), out_max=(1 * MM, 0.0, 6 * MM))
    frame = synth.make_frame(g, seed=0, n_scatterers=1, box_x=(0.0, 0.0),
                             box_z=(5 * MM, 5 * MM), noise_frac=0.0)
    r = frame.decoded.astype(np.float64)
    np.testing.assert_allclose(r, r[:, ::-1, :], atol=1e-6)
    img = oracle.das(g, r)
    np.testing.assert_allclose(img, img[:, :, ::-1], rtol=1e-9, atol=1e-9 * np.abs(img).max())


# ------------------------------------------------------------- gradients

def test_adjoint_dot_product_identity():
    # <DAS(r), G> == <r, DAS^T(G)>: the RF gradient is the exact adjoint
    g = _small_geom(fnum=0.8)
    rng = np.random.default_rng(8)
    r = rng.normal(size=(g.n_tx, g.n_ch, g.n_samples))
    G = rng.normal(size=(g.out_dims[2], g.out_dims[1], g.out_dims[0]))
    w = rng.uniform(0.5, 1.5, g.n_ch)
    lhs = float(np.sum(oracle.das(g, r, w=w) * G))
    grad_rf, _, _ = oracle.das_grad(g, r, G, w=w)
    rhs = float(np.sum(r * grad_rf))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_apodization_gradient_is_exact_for_linear_loss():
    # L = <DAS(r; w), G> is linear in w, so dL/dw_j = <DAS(r; e_j), G>
    g = _small_geom(fnum=0.6)
    rng = np.random.default_rng(9)
    r = rng.normal(size=(g.n_tx, g.n_ch, g.n_samples))
    G = rng.normal(size=(g.out_dims[2], 1, g.out_dims[0]))
    _, _, gw = oracle.das_grad(g, r, G, w=rng.uniform(0.5, 1.5, g.n_ch))
    for j in range(g.n_ch):
        e = np.zeros(g.n_ch)
        e[j] = 1.0
        assert gw[j] == pytest.approx(float(np.sum(oracle.das(g, r, w=e) * G)), rel=1e-12, abs=1e-12)


def test_speed_of_sound_gradient_matches_small_step_difference():
    # a step of 1e-9 relative moves no sample across an integer here, so the
    # central difference of the piecewise-linear interpolant is exact up to
    # rounding
    g = _small_geom()
    rng = np.random.default_rng(10)
    r = rng.normal(size=(g.n_tx, g.n_ch, g.n_samples))
    G = rng.normal(size=(g.out_dims[2], 1, g.out_dims[0]))
    c = 1530.0
    _, gc, _ = oracle.das_grad(g, r, G, c=c, want_rf=False)
    h = c * 1e-9
    fd = (np.sum(oracle.das(g, r, c=c + h) * G) - np.sum(oracle.das(g, r, c=c - h) * G)) / (2 * h)
    assert gc == pytest.approx(fd, rel=1e-5)


def test_complex_gradient_planes():
    g = _small_geom()
    rng = np.random.default_rng(12)
    r = rng.normal(size=(g.n_tx, g.n_ch, g.n_samples)) + 1j * rng.normal(size=(g.n_tx, g.n_ch, g.n_samples))
    G = rng.normal(size=(g.out_dims[2], 1, g.out_dims[0])) + 1j * rng.normal(size=(g.out_dims[2], 1, g.out_dims[0]))
    grc, gcc, gwc = oracle.das_grad(g, r, G)
    gr_re, gc_re, gw_re = oracle.das_grad(g, r.real, G.real)
    gr_im, gc_im, gw_im = oracle.das_grad(g, r.imag, G.imag)
    np.testing.assert_allclose(grc.real, gr_re, atol=1e-12)
    np.testing.assert_allclose(grc.imag, gr_im, atol=1e-12)
    assert gcc == pytest.approx(gc_re + gc_im, rel=1e-12)
    np.testing.assert_allclose(gwc, gw_re + gw_im, rtol=1e-12)


# ------------------------------------- world -> array and voxel affines

CORNER = [[1.0, 0.0, 0.0, -1.0 * MM], [0.0, 1.0, 0.0, -1.0 * MM], [0.0, 0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]]


def test_corner_element_origin_hand_computed_delays():
    # §METHODS "Data Processing": the world frame has its origin at the centre
    # of the corner element; for 3 x 3 elements of 1 mm pitch the world ->
    # array affine is a translation by (-1, -1, 0) mm. The ramp sits in one
    # trace (i, j), so the image is that trace's delay; the inverse
    # translation, or a transform applied array -> world, gives other values.
    for i, j, x, y, z, expect in _golden_rows("corner_origin_tof.txt"):
        g = Geometry(n_tx=3, n_ch=3, n_samples=1000, fs=10e6, c=1500.0, t0=0.0,
                     tx_pitch=1 * MM, rx_pitch=1 * MM, tx_orientation=ROWS, rx_orientation=COLUMNS,
                     out_dims=(1, 1, 1), out_min=(x * MM, y * MM, z * MM), out_max=(x * MM, y * MM, z * MM))
        r = np.zeros((3, 3, g.n_samples))
        r[int(i), int(j)] = np.arange(g.n_samples)
        got = oracle.das(g, r, xdc_transform=CORNER).ravel()[0]
        assert got == pytest.approx(expect, rel=0, abs=1e-9)
        # without the transform the same world point is read in the centred
        # frame: a different delay
        assert abs(oracle.das(g, r).ravel()[0] - expect) > 1.0


def _ray_affine(axis):
    # index axis `axis` onto (3, 0, 4) mm * (k + 1): row-major, index -> world
    M = np.zeros((4, 4))
    M[0, axis], M[0, 3] = 3 * MM, 3 * MM
    M[2, axis], M[2, 3] = 4 * MM, 4 * MM
    M[3, 3] = 1.0
    return M


def test_voxel_affine_hand_computed_delays():
    # Fig. "das_dispatch": a 4x4 voxel-index affine. Each index axis in turn
    # walks the ray (3, 0, 4) mm (k + 1), where the delay is 60 (k + 1)
    # samples; reading the matrix column-major (its transpose) or mapping the
    # wrong index axis moves every voxel off the ray.
    rows = _golden_rows("voxel_affine_tof.txt")
    for axis in (0, 2):
        dims = [1, 1, 1]
        dims[axis] = 3
        g = Geometry(n_tx=1, n_ch=1, n_samples=1000, fs=10e6, c=1500.0, t0=0.0,
                     tx_orientation=ROWS, rx_orientation=COLUMNS, out_dims=tuple(dims),
                     out_min=(0.0, 0.0, 0.0), out_max=(0.0, 0.0, 0.0))
        ramp = np.arange(g.n_samples, dtype=np.float64).reshape(1, 1, -1)
        got = oracle.das(g, ramp, voxel_transform=_ray_affine(axis)).ravel()
        want = [e for a, k, e in rows if int(a) == axis]
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)
        got_t = oracle.das(g, ramp, voxel_transform=_ray_affine(axis).T).ravel()
        assert np.abs(got_t - want).max() > 1.0


def test_voxel_affine_permuting_index_axes_matches_the_linspace_grid():
    # an affine that sends index axis 0 to world z and index axis 2 to world
    # x, on a grid whose x and z extents are swapped, reads the same world
    # points as the inclusive linspace grid, transposed (voxel (ix, 0, iz) of
    # the affine grid is voxel (iz, 0, ix) of the linspace grid)
    rng = np.random.default_rng(21)
    lin = Geometry(n_tx=4, n_ch=4, n_samples=256, fs=30e6, c=1540.0, out_dims=(5, 1, 7),
                   out_min=(-1 * MM, 0.0, 2 * MM), out_max=(1 * MM, 0.0, 4 * MM), f_number=0.8)
    r = rng.normal(size=(4, 4, 256))
    want = oracle.das(lin, r)                      # [nz=7][1][nx=5]
    M = np.zeros((4, 4))
    M[2, 0] = (4 - 2) * MM / 6                     # index axis 0 (7 points) -> z
    M[2, 3] = 2 * MM
    M[0, 2] = (1 - -1) * MM / 4                    # index axis 2 (5 points) -> x
    M[0, 3] = -1 * MM
    M[3, 3] = 1.0
    perm = dataclasses.replace(lin, out_dims=(7, 1, 5))
    got = oracle.das(perm, r, voxel_transform=M)   # [nz=5][1][nx=7]
    np.testing.assert_allclose(got[:, 0, :], want[:, 0, :].T, rtol=1e-12, atol=1e-12)


# ---------------------------------- radial F# window of the 2D aperture

def test_hercules_2d_window_is_radial():
    # Eq. (2)-(3) on the 2D receive aperture: the voxel (3, 4, 12) mm lies at
    # radial lateral distance 5 mm from the element (row y = 0, column x = 0).
    # F# = 0.6: u = 0.6 * 5 / 12 = 1/4, W = cos^2(pi / 4) = 1/2 exactly
    # (a window on the x offset alone gives cos^2(0.15 pi) = 0.794, on y
    # alone cos^2(0.2 pi) = 0.655). F# = 1.2: u = 1/2, the support edge, W = 0.
    g = _point_geom(3 * MM, 4 * MM, 12 * MM)
    g.acq_kind = synth.HERCULES_2D
    g.tx_wave, g.tx_angles = "plane", (0.0,)
    one = np.ones((1, 1, g.n_samples))
    g.f_number = 0.6
    assert oracle.das(g, one).ravel()[0] == pytest.approx(0.5, abs=1e-12)
    g.f_number = 1.2
    assert oracle.das(g, one).ravel()[0] == 0.0
    g.f_number = 1.19                              # just inside the support
    u = 1.19 * 5 / 12
    assert oracle.das(g, one).ravel()[0] == pytest.approx(math.cos(math.pi * u) ** 2, abs=1e-12)


# ------------------------------------- IQ at a fractional delay

def test_iq_beamforming_at_a_quarter_sample_delay():
    # s = 60 + 1/4 (the 3-4-5 geometry with t0 = -0.025 us), f_d / f_s = 1/4,
    # baseband samples b[n] = j^n (a linear phase of pi/2 per sample).
    # Linear: (3/4) b[60] + (1/4) b[61] = 3/4 + j/4. Cubic (weights -9, 111,
    # 29, -3 over 128 on samples 59..62): (9j + 111 + 29j + 3)/128 =
    # (114 + 38j)/128. Both are then rotated by e^{j 2 pi s / 4} =
    # e^{j 30.125 pi} = e^{j pi / 8}; a phase taken at floor(s) would rotate
    # by e^{j 30 pi} = 1 instead.
    g = _point_geom(3 * MM, 0.0, 4 * MM, t0=-0.025e-6)
    g.iq_freq = 2.5e6
    n = np.arange(g.n_samples)
    b = (1j ** (n % 4)).reshape(1, 1, -1)
    rot = complex(math.cos(math.pi / 8), math.sin(math.pi / 8))
    got = oracle.das(g, b, interp="linear").ravel()[0]
    assert abs(got - (0.75 + 0.25j) * rot) <= 1e-12
    got = oracle.das(g, b, interp="cubic").ravel()[0]
    assert abs(got - (114 + 38j) / 128 * rot) <= 1e-12


# ------------------------------------- complex matched-filter taps (Eq. demod)

def test_demod_complex_impulse_response_by_hand():
    # impulse A at raw index n0; the mixer e^{-j pi n0 / 2} gives A, -jA, -A, jA
    # for n0 mod 4 = 0..3; the complex product with h = hr + j hi then gives
    # (I, Q) = (hr A, hi A), (hi A, -hr A), (-hr A, -hi A), (-hi A, hr A)
    hr = np.array([3, -7, 11, 2, -5, 9], dtype=np.int16)
    hi = np.array([-4, 6, 1, -8, 10, -2], dtype=np.int16)
    A = 5
    want = {0: lambda r, i: (r * A, i * A), 1: lambda r, i: (i * A, -r * A),
            2: lambda r, i: (-r * A, -i * A), 3: lambda r, i: (-i * A, r * A)}
    for n0 in (12, 13, 14, 15):
        s = np.zeros((1, 48), dtype=np.int16)
        s[0, n0] = A
        iq = oracle.demodulate(s, hr, shift=0, decimation=1, taps_imag=hi)
        for m in range(48):
            k = m - n0
            wi, wq = want[n0 % 4](int(hr[k]), int(hi[k])) if 0 <= k < hr.size else (0, 0)
            assert (iq[0, 0, m], iq[1, 0, m]) == (wi, wq), (n0, m)


def test_demod_taps_times_j_rotate_the_output_by_a_quarter_turn():
    # taps j h (hr = 0, hi = h) give j times the output of the real taps h:
    # (I, Q) -> (-Q, I), exactly when nothing is rounded or saturated
    # (|h| <= 10 over 31 taps and |s| <= 50 keep every sum below 2^15: no saturation)
    rng = np.random.default_rng(23)
    h = rng.integers(-10, 11, size=31).astype(np.int16)
    s = rng.integers(-50, 51, size=(3, 400)).astype(np.int16)
    real = oracle.demodulate(s, h, shift=0, decimation=4)
    rot = oracle.demodulate(s, np.zeros_like(h), shift=0, decimation=4, taps_imag=h)
    np.testing.assert_array_equal(rot[0], -real[1])
    np.testing.assert_array_equal(rot[1], real[0])
    # and a general complex tap set is the sum of its real and imaginary parts' outputs
    h2 = rng.integers(-10, 11, size=31).astype(np.int16)
    both = oracle.demodulate(s, h2, shift=0, decimation=4, taps_imag=h)
    part = oracle.demodulate(s, h2, shift=0, decimation=4)
    np.testing.assert_array_equal(both[0].astype(int), part[0].astype(int) - real[1].astype(int))
    np.testing.assert_array_equal(both[1].astype(int), part[1].astype(int) + real[0].astype(int))
