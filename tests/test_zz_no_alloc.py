"""rcbf_das_noalloc: the delay-and-sum entry point for callers that must not
allocate device memory (allocation owned by a host framework's pool, real-time
loops). It takes the parameter block
instead of a plan and keeps its scratch (the channel-split partial images) in
a fixed 16 MiB device array of the library. Its images must equal those of the
planned rcbf_das on the same inputs, call after call."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests._frames import frame, rel_l2

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


def _noalloc(params, decoded, out, c=0.0):
    lib = rc.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.rcbf_das_noalloc(ctypes.byref(params), ctypes.c_void_p(decoded.data_ptr()), None,
                                ctypes.c_float(c), ctypes.c_void_p(out.data_ptr()), stream)
    assert code == rc.OK, lib.rcbf_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("name", ["tiny", "bscan"])
def test_noalloc_matches_planned_das_on_two_calls(name):
    fr = frame(name)
    g = fr.geometry
    params = rc.make_params(g, decoded_dtype="f32")
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    assert plan.info()["n_split"] > 1        # the partial-image scratch is in use
    D = oracle.decode(fr.rf)
    dec = torch.from_numpy((D.astype(np.float64) / g.n_tx).astype(np.float32)).cuda()
    out = torch.empty(plan.image_shape, dtype=torch.float32, device="cuda")
    # first call, then a second one on other inputs (speed of sound, scaled data)
    for c, scale in ((0.0, 1.0), (1500.0, -0.5)):
        d = dec * scale
        want = plan.das(d, c=c).cpu().numpy()
        got = _noalloc(params, d, out, c=c)
        err = rel_l2(got, want)
        print("%s c=%g: rel-L2 vs rcbf_das %.2e" % (name, c, err))
        assert err <= 1e-4
        assert rc.load_library().rcbf_das_noalloc_status(
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == rc.OK


def test_noalloc_call_allocates_no_device_memory():
    # after one call (which looks up the device address of the static scratch),
    # a further call changes neither torch's allocator nor the device's free
    # memory: the entry point itself allocates nothing
    fr = frame("bscan")
    g = fr.geometry
    params = rc.make_params(g, decoded_dtype="f16")
    dec = torch.from_numpy((oracle.decode(fr.rf).astype(np.float64) / g.n_tx).astype(np.float16)).cuda()
    out = torch.empty(g.out_dims[2], g.out_dims[1], g.out_dims[0], dtype=torch.float32, device="cuda")
    first = _noalloc(params, dec, out).copy()
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    second = _noalloc(params, dec, out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    np.testing.assert_array_equal(second, first)


def test_noalloc_2d_aperture_diverging_wave():
    # HERCULES read as a 2D receive aperture with a diverging wave (a plane
    # wave needs the plan's device direction table): the tiled 2D form from
    # the parameter block alone, equal to the planned call and to the oracle
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=1024, acq_kind=synth.HERCULES_2D, out_dims=(48, 40, 80),
                       out_min=(-1.5e-3, -1.2e-3, 4e-3), out_max=(1.5e-3, 1.2e-3, 14e-3))
    g.tx_wave, g.tx_focus = "point", -6e-3
    fr = synth.make_frame(g, seed=57, n_scatterers=4, box_x=(-1e-3, 1e-3), box_y=(-1e-3, 1e-3),
                          box_z=(5e-3, 13e-3), noise_frac=0.0)
    params = rc.make_params(g, decoded_dtype="f32")
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    assert plan.info()["tiled"]
    d = torch.from_numpy(fr.decoded.astype(np.float32)).cuda()
    out = torch.empty(plan.image_shape, dtype=torch.float32, device="cuda")
    got = _noalloc(params, d, out)
    want = plan.das(d).cpu().numpy()
    np.testing.assert_array_equal(got, want)
    assert rel_l2(got, oracle.das(g, fr.decoded.astype(np.float64))) <= 1e-4


def test_noalloc_vls_focal_plane_inside_the_image():
    # the split form (tiled tiles plus the plain pass over the tiles across
    # the focal depth) from the parameter block alone, equal to the plan's
    g = synth.Geometry(n_tx=32, n_ch=64, n_samples=1024, out_dims=(128, 1, 320),
                       out_min=(-3e-3, 0.0, 3e-3), out_max=(3e-3, 0.0, 18e-3))
    g.tx_wave, g.tx_focus = "vls", 9e-3
    fr = synth.make_frame(g, seed=59, n_scatterers=5, box_x=(-2.5e-3, 2.5e-3), box_z=(4e-3, 17e-3),
                          noise_frac=0.0)
    params = rc.make_params(g, decoded_dtype="f32")
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    assert plan.info()["tiled"]
    d = torch.from_numpy(fr.decoded.astype(np.float32)).cuda()
    out = torch.empty(plan.image_shape, dtype=torch.float32, device="cuda")
    got = _noalloc(params, d, out)
    np.testing.assert_array_equal(got, plan.das(d).cpu().numpy())
    assert rel_l2(got, oracle.das(g, fr.decoded.astype(np.float64))) <= 1e-4


def test_noalloc_keeps_the_channel_parts_of_the_grid_tail():
    # a frame whose tail parts' partial images fit the static scratch (512 x
    # 256 image in 128 tiles: 8 channel splits, the last 3/4 wave of units in
    # halves, 16 partial images of 0.5 MB): the same units and partial images
    # as the planned call, so the two images are equal bit for bit
    g = synth.Geometry(n_tx=128, n_ch=128, n_samples=2048, out_dims=(512, 1, 256),
                       out_min=(-6.4e-3, 0.0, 3e-3), out_max=(6.4e-3, 0.0, 15e-3))
    params = rc.make_params(g, decoded_dtype="f32", tile=(64, 1, 16))
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32", tile=(64, 1, 16)))
    info = plan.info()
    assert info["tiled"] and info["n_split"] == 8 and info["das_launches"] == 2
    gen = torch.Generator(device="cuda").manual_seed(61)
    d = torch.randn(g.n_tx, g.n_ch, g.n_samples, device="cuda", generator=gen)
    out = torch.empty(plan.image_shape, dtype=torch.float32, device="cuda")
    got = _noalloc(params, d, out)
    np.testing.assert_array_equal(got, plan.das(d).cpu().numpy())
