"""Batched stream on the GPU: frames of uneven size (transmit counts, sample
counts, grids, orientations) decoded and beamformed by one persistent launch
through rcbf_batch_*; checked against the single-frame entry points and the
FP64 oracle, replayed from a captured CUDA graph, and with the bounded
per-frame wait driven to expiry through the test hook."""
import numpy as np
import pytest

import oracle
import synth
from synth import MM
from tests._frames import rel_l2, sample_voxels

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


def _stream_frames():
    """Eight frames: three transmit counts, three sample counts, three grids,
    a cross-plane pair and one frame handed over already decoded."""
    frames = []
    geos = synth.stream_geometries()
    for idx in (0, 1, 2, 4, 32, 33):
        g, seed, box = geos[idx]
        frames.append(synth.make_frame(g, seed, 6, **box))
    g = synth.Geometry(n_tx=64, n_ch=128, n_samples=2048, out_dims=(256, 1, 512),
                       out_min=(-6.4 * MM, 0.0, 3 * MM), out_max=(6.4 * MM, 0.0, 27 * MM))
    frames.append(synth.make_frame(g, 77, 6))                 # not encoded
    return frames


@pytest.fixture(scope="module")
def stream():
    frames = _stream_frames()
    plans, rf, dec, img = [], [], [], []
    for k, fr in enumerate(frames):
        g = fr.geometry
        variant = rc.DECODE_MMA_F16 if k % 2 else rc.DECODE_MMA_I8
        plans.append(rc.Plan(rc.make_params(g, decoded_dtype="f16", decode_variant=variant, tile=(64, 1, 16))))
        if fr.rf is not None:
            rf.append(torch.from_numpy(fr.rf).cuda())
            dec.append(torch.empty(g.n_tx, g.n_ch, g.n_samples, dtype=torch.float16, device="cuda"))
        else:
            rf.append(None)
            dec.append(torch.from_numpy(fr.decoded).to(torch.float16).cuda())
        img.append(torch.empty(g.out_dims[2], g.out_dims[1], g.out_dims[0], dtype=torch.float32, device="cuda"))
    batch = rc.Batch(plans, rf, dec, img)
    return frames, plans, rf, dec, img, batch


def test_batch_matches_single_frames_and_oracle(stream):
    frames, plans, rf, dec, img, batch = stream
    batch.run()
    assert batch.status() == rc.OK
    for k, fr in enumerate(frames):
        g = fr.geometry
        if fr.rf is not None:
            D = oracle.decode(fr.rf)
            want16 = oracle.decoded_as(D, g.n_tx, "f16")
            np.testing.assert_array_equal(dec[k].cpu().numpy().view(np.uint16), want16.view(np.uint16))
            exact16 = want16.astype(np.float64)
        else:
            exact16 = dec[k].cpu().numpy().astype(np.float64)
        single = plans[k].das(dec[k]).cpu().numpy()
        got = img[k].cpu().numpy()
        e_single = rel_l2(got, single)
        vox = sample_voxels(g.out_dims, 600, seed=k)
        e_oracle = rel_l2(got.ravel()[vox], oracle.das(g, exact16, voxels=vox))
        print("frame %d (%d tx, %d s, %s): vs single-frame %.2e, vs oracle %.2e"
              % (k, g.n_tx, g.n_samples, g.out_dims, e_single, e_oracle))
        assert e_single <= 1e-5 and e_oracle <= 1e-4


def test_batch_graph_capture_and_replay(stream):
    frames, plans, rf, dec, img, batch = stream
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.run(stream=s)                   # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.run()
    # new inputs in the bound buffers, then replay
    for k, fr in enumerate(frames):
        if rf[k] is not None:
            rf[k].copy_(torch.from_numpy(np.ascontiguousarray(-fr.rf)))
    graph.replay()
    torch.cuda.synchronize()
    assert batch.status() == rc.OK
    for k, fr in enumerate(frames):
        if fr.rf is None:
            continue
        g = fr.geometry
        want = oracle.decoded_as(oracle.decode(-fr.rf), g.n_tx, "f16")
        np.testing.assert_array_equal(dec[k].cpu().numpy().view(np.uint16), want.view(np.uint16))
        assert rel_l2(img[k].cpu().numpy(), plans[k].das(dec[k]).cpu().numpy()) <= 1e-5
    graph.replay()
    torch.cuda.synchronize()
    assert batch.status() == rc.OK


def test_batch_bounded_wait_expires_and_context_survives(stream):
    frames, plans, rf, dec, img, batch = stream
    batch.set_wait(2_000_000, withhold_frame=1)       # 2 ms bound; frame 1 never completes its decode
    batch.run()
    assert batch.status() == rc.ETIMEOUT
    batch.set_wait(1_000_000_000, withhold_frame=-1)
    for k, fr in enumerate(frames):
        if rf[k] is not None:
            rf[k].copy_(torch.from_numpy(fr.rf))
    batch.run()
    assert batch.status() == rc.OK
    k = 1
    assert rel_l2(img[k].cpu().numpy(), plans[k].das(dec[k]).cpu().numpy()) <= 1e-5


def test_batch_phases_of_mixed_tiles_and_window_classes():
    # frames with different tile extents along u and different window classes
    # run as several persistent launches (phases), the later ones launched as
    # programmatic dependents; interleaved in the frame list, captured in a
    # graph and replayed: every frame equals its single-frame DAS
    geos = synth.stream_geometries()
    specs = [(0, (64, 1, 16)), (2, (32, 1, 32)), (1, (64, 1, 16)), (2, (128, 1, 8)), (0, (32, 1, 32)),
             (33, (64, 1, 16))]
    frames, plans, rf, dec, img = [], [], [], [], []
    for idx, tile in specs:
        g, seed, box = geos[idx]
        fr = synth.make_frame(g, seed, 4, **box)
        frames.append(fr)
        variant = rc.DECODE_TC if len(plans) % 2 else rc.DECODE_MMA_I8
        plans.append(rc.Plan(rc.make_params(g, decoded_dtype="f16", decode_variant=variant, tile=tile)))
        rf.append(torch.from_numpy(fr.rf).cuda())
        dec.append(torch.empty(g.n_tx, g.n_ch, g.n_samples, dtype=torch.float16, device="cuda"))
        img.append(torch.empty(g.out_dims[2], g.out_dims[1], g.out_dims[0], device="cuda"))
    cls = lambda w: 48 if w <= 48 else 64 if w <= 64 else 96 if w <= 96 else 128
    phases = {(cls(p.info()["window"]), p.info()["tile"][0]) for p in plans}
    assert len(phases) >= 3, phases
    batch = rc.Batch(plans, rf, dec, img)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.run()
    for k in range(len(frames)):
        img[k].zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert batch.status() == rc.OK
    for k, fr in enumerate(frames):
        g = fr.geometry
        want16 = oracle.decoded_as(oracle.decode(fr.rf), g.n_tx, "f16")
        np.testing.assert_array_equal(dec[k].cpu().numpy().view(np.uint16), want16.view(np.uint16))
        single = plans[k].das(dec[k]).cpu().numpy()
        assert rel_l2(img[k].cpu().numpy(), single) <= 1e-5, k
        vox = sample_voxels(g.out_dims, 300, seed=k)
        assert rel_l2(img[k].cpu().numpy().ravel()[vox], oracle.das(g, want16.astype(np.float64), voxels=vox)) <= 1e-4
    # a withheld frame in a later phase times out; the other phases finish
    batch.set_wait(2_000_000, withhold_frame=1)
    batch.run()
    assert batch.status() == rc.ETIMEOUT
    batch.set_wait(1_000_000_000, withhold_frame=-1)
    batch.run()
    assert batch.status() == rc.OK


def test_batch_at_the_benchmark_configuration():
    # the launch the benchmark times: four full B-scans (128 tx x 128 ch x
    # 4096 samples -> 512 x 1024) in one persistent launch replayed from a
    # CUDA graph, split-byte int8 decode to FP16, tiled DAS with the tuned
    # tile. Frames alternate in sign so that each slot has its own data.
    from paper_2512_11086_gb300 import tune
    from tests._frames import frame
    fr = frame("bscan")
    g = fr.geometry
    tile = tune.tune_tile(g, "f16")
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f16", decode_variant=rc.DECODE_MMA_I8,
                                  das_variant=rc.DAS_TILED, tile=tile))
    B = 4
    signs = [1 if k % 2 == 0 else -1 for k in range(B)]
    rf = [torch.from_numpy(np.ascontiguousarray(s * fr.rf)).cuda() for s in signs]
    dec = [torch.empty(g.n_tx, g.n_ch, g.n_samples, dtype=torch.float16, device="cuda") for _ in range(B)]
    img = [torch.empty(g.out_dims[2], g.out_dims[1], g.out_dims[0], device="cuda") for _ in range(B)]
    batch = rc.Batch([plan] * B, rf, dec, img)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.run()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert batch.status() == rc.OK
    D = oracle.decode(fr.rf)
    want16 = oracle.decoded_as(D, g.n_tx, "f16")
    vox = sample_voxels(g.out_dims, 1500, seed=9)
    want = oracle.das(g, want16.astype(np.float64), voxels=vox)
    want16_neg = oracle.decoded_as(-D, g.n_tx, "f16")     # D = 0 stays +0 in either sign
    for k, sg in enumerate(signs):
        np.testing.assert_array_equal(dec[k].cpu().numpy().view(np.uint16),
                                      (want16 if sg > 0 else want16_neg).view(np.uint16))
        got = img[k].cpu().numpy().ravel()[vox]
        err = rel_l2(got, sg * want)
        print("benchmark batch slot %d (tile %s): rel-L2 %.2e" % (k, tile, err))
        assert err <= 1e-4


def test_batch_with_tcgen05_decode_frames():
    # frames whose plans use the tcgen05 decode are decoded by their own
    # launches ahead of the persistent kernel; mixed with an in-kernel
    # (split-byte int8) frame, an unencoded frame, and replayed from a graph
    frames = _stream_frames()
    plans, rf, dec, img = [], [], [], []
    for k, fr in enumerate(frames):
        g = fr.geometry
        variant = rc.DECODE_MMA_I8 if k == 1 else rc.DECODE_TC
        plans.append(rc.Plan(rc.make_params(g, decoded_dtype="f16", decode_variant=variant, tile=(64, 1, 16))))
        if fr.rf is not None:
            rf.append(torch.from_numpy(fr.rf).cuda())
            dec.append(torch.empty(g.n_tx, g.n_ch, g.n_samples, dtype=torch.float16, device="cuda"))
        else:
            rf.append(None)
            dec.append(torch.from_numpy(fr.decoded).to(torch.float16).cuda())
        img.append(torch.empty(g.out_dims[2], g.out_dims[1], g.out_dims[0], dtype=torch.float32, device="cuda"))
    batch = rc.Batch(plans, rf, dec, img)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.run()
    for k, fr in enumerate(frames):                       # new data in the bound buffers
        if rf[k] is not None:
            rf[k].copy_(torch.from_numpy(np.ascontiguousarray(-fr.rf)))
    graph.replay()
    torch.cuda.synchronize()
    assert batch.status() == rc.OK
    for k, fr in enumerate(frames):
        g = fr.geometry
        if fr.rf is not None:
            want16 = oracle.decoded_as(oracle.decode(-fr.rf), g.n_tx, "f16")
            np.testing.assert_array_equal(dec[k].cpu().numpy().view(np.uint16), want16.view(np.uint16))
            data = want16.astype(np.float64)
        else:
            data = dec[k].cpu().numpy().astype(np.float64)
        vox = sample_voxels(g.out_dims, 400, seed=20 + k)
        err = rel_l2(img[k].cpu().numpy().ravel()[vox], oracle.das(g, data, voxels=vox))
        print("tcgen05-decoded batch frame %d (%d tx): rel-L2 %.2e" % (k, g.n_tx, err))
        assert err <= 1e-4
    # the bounded per-frame wait still guards a tcgen05-decoded frame
    batch.set_wait(2_000_000, withhold_frame=0)
    batch.run()
    assert batch.status() == rc.ETIMEOUT
    batch.set_wait(1_000_000_000, withhold_frame=-1)
    batch.run()
    assert batch.status() == rc.OK
