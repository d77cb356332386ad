"""Edge cases of the DAS path on the GPU against the FP64 oracle: the maximum
Hadamard order and channel count (256 x 256), a one-voxel image, the minimum
record length, a record that no delay reaches (all zero), transmit counts the
tiled form cannot take (an explicit error, or the plain form), and misaligned
buffers rejected before any launch."""
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


def test_maximum_order_and_channels():
    # 256 encoded transmits x 256 channels: exact decode, then tiled DAS
    g = synth.Geometry(n_tx=256, n_ch=256, n_samples=1024, hadamard_order=256, out_dims=(128, 1, 96),
                       tx_pitch=0.05 * MM, rx_pitch=0.05 * MM,
                       out_min=(-3 * MM, 0.0, 5 * MM), out_max=(3 * MM, 0.0, 15 * MM))
    fr = synth.make_frame(g, seed=61, n_scatterers=4, box_x=(-2 * MM, 2 * MM), box_z=(6 * MM, 14 * MM))
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    dec = plan.decode(torch.from_numpy(fr.rf).cuda())
    D = oracle.decode(fr.rf)
    want_dec = oracle.decoded_as(D, 256, "f32")
    np.testing.assert_array_equal(dec.cpu().numpy().view(np.uint32), want_dec.view(np.uint32))
    img = plan.das(dec).cpu().numpy()
    vox = sample_voxels(g.out_dims, 1500, seed=61)
    want = oracle.das(g, D.astype(np.float64) / 256, voxels=vox)
    assert plan.info()["tiled"]
    assert rel_l2(img.ravel()[vox], want) <= TOL


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
def test_one_voxel_image(variant):
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=512, out_dims=(1, 1, 1),
                       out_min=(0.3 * MM, 0.0, 6 * MM), out_max=(0.3 * MM, 0.0, 6 * MM))
    r = np.random.default_rng(62).normal(size=(16, 16, 512))
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32", das_variant=variant))
    img = plan.das(torch.from_numpy(r.astype(np.float32)).cuda()).cpu().numpy()
    assert img.shape == (1, 1, 1)
    assert rel_l2(img, oracle.das(g, r)) <= TOL


def test_minimum_record_and_unreached_record():
    # 8 samples (the minimum) reached by every delay at t0 = ToF - 3 samples:
    # compare with the oracle; then a record that ends before the shallowest
    # echo: every term is outside the record and the image is exactly zero
    g = synth.Geometry(n_tx=8, n_ch=8, n_samples=8, out_dims=(4, 1, 4),
                       out_min=(-0.02 * MM, 0.0, 6 * MM), out_max=(0.02 * MM, 0.0, 6.02 * MM))
    g.t0 = 2 * 6e-3 / g.c - 3.0 / g.fs
    r = np.random.default_rng(63).normal(size=(8, 8, 8))
    for variant in (rc.DAS_TILED, rc.DAS_PLAIN):
        plan = rc.Plan(rc.make_params(g, decoded_dtype="f32", das_variant=variant))
        img = plan.das(torch.from_numpy(r.astype(np.float32)).cuda()).cpu().numpy()
        assert rel_l2(img, oracle.das(g, r)) <= TOL
    g.t0 = 0.0                                         # samples 0..7 end long before 7.8 us
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    img = plan.das(torch.from_numpy(r.astype(np.float32)).cuda()).cpu().numpy()
    assert np.all(img == 0.0)


def test_transmit_counts_the_tiled_form_cannot_take():
    g = synth.Geometry(n_tx=12, n_ch=16, n_samples=512, out_dims=(64, 1, 64),
                       out_min=(-1 * MM, 0.0, 5 * MM), out_max=(1 * MM, 0.0, 9 * MM))
    r = np.random.default_rng(64).normal(size=(12, 16, 512)).astype(np.float32)
    tiled = rc.Plan(rc.make_params(g, decoded_dtype="f32", das_variant=rc.DAS_TILED))
    with pytest.raises(rc.RcbfError) as e:
        tiled.das(torch.from_numpy(r).cuda())
    assert e.value.code == rc.EUNSUPPORTED
    plain = rc.Plan(rc.make_params(g, decoded_dtype="f32", das_variant=rc.DAS_PLAIN))
    img = plain.das(torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel_l2(img, oracle.das(g, r.astype(np.float64))) <= TOL


def test_misaligned_buffers_are_rejected():
    g = synth.tiny_bscan_geometry()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    buf = torch.zeros(g.n_tx * g.n_ch * g.n_samples + 1, device="cuda")
    dec = buf[1:].view(g.n_tx, g.n_ch, g.n_samples)            # 4-byte, not 16-byte aligned
    with pytest.raises(rc.RcbfError) as e:
        plan.das(dec)
    assert e.value.code == rc.EINVAL
    rf = torch.zeros(g.n_tx * g.n_ch * g.n_samples + 1, dtype=torch.int16, device="cuda")[1:]
    with pytest.raises(rc.RcbfError) as e:
        plan.decode(rf.view(g.n_tx, g.n_ch, g.n_samples))
    assert e.value.code == rc.EINVAL


def test_channel_shards_sum_to_the_frame():
    # the per-GPU plans of a channel-sharded frame, run one after the other
    # on one GPU: each sees only its slice of the decoded data, with the
    # element positions of that slice in the whole array
    from paper_2512_11086_gb300 import shard
    g = synth.Geometry(n_tx=32, n_ch=48, n_samples=1024, out_dims=(96, 1, 160),
                       out_min=(-2 * MM, 0.0, 4 * MM), out_max=(2 * MM, 0.0, 14 * MM))
    fr = synth.make_frame(g, seed=65, n_scatterers=5, box_x=(-1.5 * MM, 1.5 * MM), box_z=(5 * MM, 13 * MM))
    dec = torch.from_numpy(fr.decoded).cuda()
    total = None
    for rank in range(3):
        off, cnt = shard.channel_slices(g.n_ch, 3)[rank]
        plan = rc.Plan(shard.shard_params(g, rank, 3, decoded_dtype="f32"))
        part = plan.das(dec[:, off:off + cnt].contiguous())
        total = part if total is None else total + part
    full = rc.Plan(rc.make_params(g, decoded_dtype="f32")).das(dec).cpu().numpy()
    assert rel_l2(total.cpu().numpy(), full) <= 1e-5
    assert rel_l2(total.cpu().numpy(), oracle.das(g, fr.decoded.astype(np.float64))) <= TOL


def test_measured_ceilings_are_consistent_with_the_clock():
    # the microbenchmarks behind the DAS roofline: per SM and clock, 8-byte
    # shared loads deliver at most 128 B (one wavefront), FP32 FMA at most
    # 128 lane operations, shared reductions at most one warp instruction
    c = rc.measure_ceilings()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per_clk = sms * c["sm_clock_hz"]
    assert 1e8 < c["sm_clock_hz"] < 4e9
    assert 0.5 * 128 <= c["lds64_bytes_per_s"] / per_clk <= 1.05 * 128
    assert 0.5 * 128 <= c["ffma_lane_ops_per_s"] / per_clk <= 1.05 * 128
    assert 0.5 * 128 <= c["ffma2_lane_ops_per_s"] / per_clk <= 1.05 * 128
    assert 0.25 <= c["red_shared_per_s"] / per_clk <= 1.05
