"""Quadrature demodulation, complex decode and IQ beamforming on the GPU
(through the C ABI) against the FP64 / integer oracle: rcbf_demodulate bit
for bit (decimations, filter lengths, saturation, ragged segments), the
demodulated planes decoded bit for bit, IQ DAS (tiled linear and cubic, plain)
within 1e-4, the whole chain on an encoded point-scatterer frame (small and at
the full B-scan size), and the entry points built for RF data only."""
import numpy as np
import pytest

import oracle
import synth
from synth import MM
from tests._frames import rel_l2, sample_voxels

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2512_11086_gb300 as rc  # noqa: E402

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11086_gb300 import build
    build.build()
    torch.cuda.set_device(0)


_lowpass_taps = synth.lowpass_taps


def _geom(n_tx, n_ch, n_s, **kw):
    return synth.Geometry(n_tx=n_tx, n_ch=n_ch, n_samples=n_s, **kw)


@pytest.mark.parametrize("D,n_taps,shift", [(1, 1, 0), (2, 33, 12), (3, 64, 13), (4, 166, 15),
                                            (8, 255, 15), (16, 1024, 15)])
def test_demodulate_bit_exact(D, n_taps, shift):
    rng = np.random.default_rng(100 + D)
    n_out = 1000 if D < 8 else 520              # several CTA segments plus a ragged one (1024 outputs each)
    n_out = (n_out + 7) // 8 * 8
    taps = rng.integers(-60, 61, size=n_taps).astype(np.int16)
    if n_taps == 1:
        taps[:] = 12345
    g = _geom(8, 16, n_out)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32", demod=(D, taps, shift)))
    rf = rng.integers(-32768, 32768, size=(8, 16, n_out * D), dtype=np.int16)
    got = plan.demodulate(torch.from_numpy(rf).cuda()).cpu().numpy()
    want = oracle.demodulate(rf, taps, shift, D)
    assert got.shape == want.shape == (2, 8, 16, n_out)
    np.testing.assert_array_equal(got, want)


def test_demodulate_saturates_like_the_oracle():
    rng = np.random.default_rng(7)
    taps = np.full(2, 30000, dtype=np.int16)     # sum |h| = 60000: exact 32-bit sums that overflow int16
    g = _geom(4, 8, 256)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32", demod=(2, taps, 1)))
    rf = rng.integers(-32768, 32768, size=(4, 8, 512), dtype=np.int16)
    got = plan.demodulate(torch.from_numpy(rf).cuda()).cpu().numpy()
    want = oracle.demodulate(rf, taps, 1, 2)
    assert np.mean(np.abs(want.astype(np.int32)) == 32767) > 0.05 or np.any(want == -32768)
    np.testing.assert_array_equal(got, want)


def test_demodulate_then_decode_bit_exact():
    # encoded acquisitions: demodulation and decode commute only up to the
    # int16 rounding, so the chain is compared with the oracle's own chain
    g = _geom(32, 32, 512, hadamard_order=32)
    rng = np.random.default_rng(9)
    r = rng.integers(-900, 900, size=(32, 32, 2048))
    rf = (oracle.hadamard(32).astype(np.int64).T @ r.reshape(32, -1)).reshape(r.shape).astype(np.int16)
    taps = _lowpass_taps(41, 0.1)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32", demod=(4, taps, 15)))
    iq = plan.demodulate(torch.from_numpy(rf).cuda())
    dec = plan.decode(iq).cpu().numpy()
    iq_want = oracle.demodulate(rf, taps, 15, 4)
    np.testing.assert_array_equal(iq.cpu().numpy(), iq_want)
    for p in range(2):
        want = oracle.decoded_as(oracle.decode(iq_want[p]), 32, "f32")
        np.testing.assert_array_equal(dec[p].view(np.uint32), want.view(np.uint32))


def _iq_case():
    g = _geom(32, 32, 1024, fs=7.5e6, iq_freq=7.5e6, out_dims=(128, 1, 640),
              out_min=(-3 * MM, 0.0, 4 * MM), out_max=(3 * MM, 0.0, 40 * MM))
    rng = np.random.default_rng(21)
    # smooth baseband data: low-pass filtered complex noise
    x = rng.normal(size=(32, 32, 1024)) + 1j * rng.normal(size=(32, 32, 1024))
    k = np.hanning(9)
    x = np.apply_along_axis(lambda v: np.convolve(v, k, mode="same"), -1, x)
    return g, x


@pytest.mark.parametrize("interp,variant", [("linear", rc.DAS_TILED), ("cubic", rc.DAS_TILED),
                                            ("linear", rc.DAS_PLAIN), ("cubic", rc.DAS_PLAIN)])
def test_iq_beamforming_matches_oracle(interp, variant):
    g, x = _iq_case()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32", das_variant=variant, interp=interp))
    info = plan.info()
    dec = torch.from_numpy(np.stack([x.real, x.imag]).astype(np.float32)).cuda()
    img = plan.das(dec).cpu().numpy().astype(np.float64)
    got = img[0] + 1j * img[1]
    want = oracle.das(g, x.astype(np.complex64).astype(np.complex128), interp=interp)
    err = rel_l2(got, want)
    print("IQ %s v%d (tiled %s, window %d): rel-L2 %.3e" % (interp, variant, info["tiled"], info["window"], err))
    assert info["tiled"] == (variant == rc.DAS_TILED)
    assert err <= TOL
    # the carrier matters: without the re-modulation the image is different
    assert rel_l2(oracle.das(g, x, iq_freq=0.0, interp=interp), want) > 0.1


@pytest.mark.parametrize("interp", ["linear", "cubic"])
@pytest.mark.parametrize("tile", [(32, 1, 32), (64, 1, 16), (128, 1, 8)])
def test_iq_general_ratio_weights_and_tiles(interp, tile):
    # a demodulation frequency that is not the sampling rate (the carrier
    # phase of every window start matters: r = f_d / f_s = 0.3), the F#
    # window with per-channel weights, and every voxels-per-thread class of
    # the tiled IQ form
    g = _geom(32, 32, 1024, fs=7.5e6, iq_freq=0.3 * 7.5e6, out_dims=(128, 1, 320),
              out_min=(-3 * MM, 0.0, 4 * MM), out_max=(3 * MM, 0.0, 22 * MM), f_number=1.0)
    _, x = _iq_case()
    w = np.random.default_rng(5).uniform(0.5, 1.5, size=g.n_ch)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32", das_variant=rc.DAS_TILED, interp=interp, tile=tile))
    dec = torch.from_numpy(np.stack([x.real, x.imag]).astype(np.float32)).cuda()
    img = plan.das(dec, apod=torch.from_numpy(w.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    got = img[0] + 1j * img[1]
    want = oracle.das(g, x.astype(np.complex64).astype(np.complex128), w=w, interp=interp)
    err = rel_l2(got, want)
    print("IQ r=0.3 %s tile %s: rel-L2 %.3e" % (interp, tile, err))
    assert plan.info()["tiled"]
    assert err <= TOL


def _chain(g_raw, D, taps, frame_seed, n_scatterers, point=None):
    """Encoded RF at 4 f_d -> (plan of the demodulated data, raw int16 RF)."""
    kw = {} if point is None else dict(box_x=(point[0], point[0]), box_z=(point[2], point[2]))
    fr = synth.make_frame(g_raw, seed=frame_seed, n_scatterers=n_scatterers, noise_frac=0.0, **kw)
    gd = (taps.size - 1) / 2
    g = synth.Geometry(n_tx=g_raw.n_tx, n_ch=g_raw.n_ch, n_samples=g_raw.n_samples // D, fs=g_raw.fs / D,
                       t0=g_raw.t0 - gd / g_raw.fs, iq_freq=g_raw.fs / 4, hadamard_order=g_raw.hadamard_order,
                       out_dims=g_raw.out_dims, out_min=g_raw.out_min, out_max=g_raw.out_max)
    return fr, g


def _oracle_chain(fr, g, D, taps, shift, voxels=None, interp="linear"):
    iq = oracle.demodulate(fr.rf, taps, shift, D)
    planes = [oracle.decode(iq[p]).astype(np.float64) / g.n_tx for p in range(2)]
    return iq, oracle.das(g, planes[0] + 1j * planes[1], voxels=voxels, interp=interp)


@pytest.mark.parametrize("interp", ["linear", "cubic"])
def test_chain_point_scatterer(interp):
    # raw 32 x 32 x 2048 at 30 MHz (= 4 x 7.5 MHz), 33-tap low-pass, D = 4
    p = (0.0, 0.0, 12 * MM)
    g_raw = synth.Geometry(n_tx=32, n_ch=32, n_samples=2048, hadamard_order=32, out_dims=(81, 1, 161),
                           out_min=(-2 * MM, 0.0, 10 * MM), out_max=(2 * MM, 0.0, 14 * MM))
    taps = _lowpass_taps(33, 0.12)
    fr, g = _chain(g_raw, 4, taps, 3, 1, point=p)
    g.interp = interp
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32", demod=(4, taps, 15)))
    rf = torch.from_numpy(fr.rf).cuda()
    iq = plan.demodulate(rf)
    img = plan.das(plan.decode(iq)).cpu().numpy().astype(np.float64)
    got = img[0] + 1j * img[1]
    iq_w, want = _oracle_chain(fr, g, 4, taps, 15, interp=interp)
    np.testing.assert_array_equal(iq.cpu().numpy(), iq_w)
    err = rel_l2(got, want)
    print("chain %s: rel-L2 %.3e" % (interp, err))
    assert err <= TOL
    # the envelope peaks at the scatterer, like the RF image of the same frame
    peak = np.unravel_index(np.argmax(np.abs(got)), got.shape)
    assert peak == (80, 0, 40)


def test_chain_full_bscan_sampled():
    # the benchmark's IQ form: the B-scan acquisition (128 x 128 x 4096 at
    # 30 MHz), 166-tap filter, D = 4, cubic IQ DAS to 512 x 1024
    g_raw = synth.full_bscan_geometry()
    taps = _lowpass_taps(166, 0.12, shift=14)      # Q14: the long filter's sum |h| stays <= 65535
    assert int(np.abs(taps.astype(np.int64)).sum()) <= 65535
    fr, g = _chain(g_raw, 4, taps, 2, 64)
    g.interp = "cubic"
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32", demod=(4, taps, 14)))
    img = plan.das(plan.decode(plan.demodulate(torch.from_numpy(fr.rf).cuda()))).cpu().numpy()
    vox = sample_voxels(g.out_dims, 800, seed=4)
    _, want = _oracle_chain(fr, g, 4, taps, 14, voxels=vox, interp="cubic")
    got = img[0].ravel()[vox] + 1j * img[1].ravel()[vox]
    err = rel_l2(got, want)
    print("full B-scan IQ chain: rel-L2 %.3e, tiled %s" % (err, plan.info()["tiled"]))
    assert err <= TOL


def test_rf_only_entry_points_reject_iq():
    g, x = _iq_case()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32"))
    dec = torch.zeros(2, g.n_tx, g.n_ch, g.n_samples, device="cuda")
    gi = torch.zeros(2, g.out_dims[2], g.out_dims[1], g.out_dims[0], device="cuda")
    with pytest.raises(rc.RcbfError) as e:
        plan.das_backward(dec, gi)
    assert e.value.code == rc.EUNSUPPORTED
    with pytest.raises(rc.RcbfError) as e:
        rc.Plan(rc.make_params(g, decoded_dtype="f32"))          # IQ needs complex data
    assert e.value.code == rc.EINVAL
    with pytest.raises(rc.RcbfError) as e:                        # sum |taps| too large
        rc.Plan(rc.make_params(g, decoded_dtype="cf32", demod=(2, np.full(3, 30000), 0)))
    assert e.value.code == rc.EINVAL
