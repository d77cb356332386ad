"""Demodulation fused into the decode (rcbf_demod_decode) and complex
(matched-filter) taps on the GPU, through the C ABI, against the oracle's own
chain: oracle.demodulate (integer FIR with the quadrature mixer, rounding
shift, int16 saturation) then oracle.decode of both planes, compared bit for
bit with the decoded FP32 planes. Covers real and complex taps, D = 4 and 8,
every supported order, ragged sample blocks, full-range int16 with saturation,
the unfused rcbf_demodulate with complex taps, and the full B-scan
acquisition (128 x 128 x 4096 at 4 f_d, 166 taps)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2512_11086_gb300 as rc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11086_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _encoded(n, n_ch, n_raw, seed, lim=900):
    rng = np.random.default_rng(seed)
    r = rng.integers(-lim, lim + 1, size=(n, n_ch, n_raw))
    return (oracle.hadamard(n).astype(np.int64).T @ r.reshape(n, -1)).reshape(r.shape).astype(np.int16)


def _want(rf, taps, shift, D, taps_im=None):
    iq = oracle.demodulate(rf, taps, shift, D, taps_imag=taps_im)
    n = rf.shape[0]
    return np.stack([oracle.decoded_as(oracle.decode(iq[p]), n, "f32") for p in range(2)])


def _complex_taps(n_taps, seed, scale=0.45):
    # a complex baseband filter: the low-pass with a linear phase ramp (a
    # matched filter that also corrects a phase), rounded to int16 with
    # sum |re| + sum |im| within the exact-accumulation bound
    h = synth.lowpass_taps(n_taps, 0.12, shift=14).astype(np.float64)
    k = np.arange(n_taps)
    z = h * np.exp(1j * (0.3 + 0.05 * k)) * scale
    re, im = np.round(z.real).astype(np.int16), np.round(z.imag).astype(np.int16)
    assert np.abs(re.astype(int)).sum() + np.abs(im.astype(int)).sum() <= 65535
    return re, im


def _plan(n, n_ch, n_s, D, taps, shift, taps_im=None):
    g = synth.Geometry(n_tx=n, n_ch=n_ch, n_samples=n_s, hadamard_order=n)
    return rc.Plan(rc.make_params(g, decoded_dtype="cf32", demod=(D, taps, shift, taps_im)))


@pytest.mark.parametrize("n,n_ch,n_s,D,n_taps,cplx", [
    (32, 8, 256, 4, 41, False), (32, 8, 256, 4, 41, True), (64, 5, 200, 4, 166, False),
    (128, 3, 136, 4, 166, True), (32, 6, 128, 8, 63, False), (64, 4, 96, 8, 31, True),
    (128, 2, 64, 4, 1, False), (32, 3, 8, 4, 7, True)])
def test_fused_equals_demodulate_then_decode(n, n_ch, n_s, D, n_taps, cplx):
    rf = _encoded(n, n_ch, n_s * D, seed=n + n_ch + n_s + D + n_taps)
    if cplx:
        taps, taps_im = _complex_taps(n_taps, seed=n_taps)
    else:
        taps, taps_im = synth.lowpass_taps(n_taps, 0.1), None
    shift = 15
    plan = _plan(n, n_ch, n_s, D, taps, shift, taps_im)
    got = plan.demod_decode(torch.from_numpy(rf).cuda()).cpu().numpy()
    want = _want(rf, taps, shift, D, taps_im)
    np.testing.assert_array_equal(got, want)
    # the unfused chain (rcbf_demodulate, then rcbf_decode of the two planes) agrees too
    unfused = plan.decode(plan.demodulate(torch.from_numpy(rf).cuda())).cpu().numpy()
    np.testing.assert_array_equal(unfused, want)


def test_fused_saturation_and_full_int16_range():
    # full-range int16 encoded data and a filter whose sums overflow int16:
    # the demodulated samples saturate exactly as the oracle's
    rng = np.random.default_rng(31)
    n, n_ch, n_s, D = 64, 4, 128, 4
    rf = rng.integers(-32768, 32768, size=(n, n_ch, n_s * D), dtype=np.int64).astype(np.int16)
    taps = np.array([30000, -20000, 10000, 4000, -500], dtype=np.int16)   # sum |h| = 64500 + 410
    taps_im = np.array([-100, 200, 0, 77, -33], dtype=np.int16)
    plan = _plan(n, n_ch, n_s, D, taps, 3, taps_im)
    got = plan.demod_decode(torch.from_numpy(rf).cuda()).cpu().numpy()
    iq = oracle.demodulate(rf, taps, 3, D, taps_imag=taps_im)
    assert np.mean(np.abs(iq.astype(np.int32)) >= 32767) > 0.05
    np.testing.assert_array_equal(got, _want(rf, taps, 3, D, taps_im))


def test_unfused_demodulate_complex_taps_bit_exact():
    rng = np.random.default_rng(33)
    taps, taps_im = _complex_taps(166, seed=5)
    g = synth.Geometry(n_tx=8, n_ch=16, n_samples=1000)
    for D in (1, 3, 4):
        plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32", demod=(D, taps, 14, taps_im)))
        rf = rng.integers(-32768, 32768, size=(8, 16, 1000 * D), dtype=np.int64).astype(np.int16)
        got = plan.demodulate(torch.from_numpy(rf).cuda()).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.demodulate(rf, taps, 14, D, taps_imag=taps_im))


def test_fused_rejects_unsupported_decimation():
    taps = synth.lowpass_taps(31, 0.1)
    plan = _plan(32, 4, 64, 2, taps, 15)
    rf = torch.zeros(32, 4, 128, dtype=torch.int16, device="cuda")
    with pytest.raises(rc.RcbfError) as e:
        plan.demod_decode(rf)
    assert e.value.code == rc.EUNSUPPORTED


@pytest.mark.parametrize("cplx", [False, True])
def test_fused_full_bscan_acquisition(cplx):
    # the FORCES B-scan acquisition at 4 f_d: 128 tx x 128 ch x 4096 raw samples,
    # 166-tap filter, D = 4 -> both decoded planes of 128 x 128 x 1024
    fr = synth.full_bscan(2)
    taps = synth.lowpass_taps(166, 0.12, shift=14)
    taps_im = None
    if cplx:
        taps, taps_im = _complex_taps(166, seed=7, scale=1.0)
    plan = _plan(128, 128, 1024, 4, taps, 14, taps_im)
    got = plan.demod_decode(torch.from_numpy(fr.rf).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, _want(fr.rf, taps, 14, 4, taps_im))
