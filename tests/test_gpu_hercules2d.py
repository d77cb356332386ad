"""HERCULES with its 2D receive aperture (non-separable delays) on the GPU
against the FP64 oracle, in the tiled form (box-bounded windows, sqrt(P + Q)
per sum) and the plain form: volumes and cross-planes, plane and diverging
transmit waves, linear and cubic interpolation, FP32 / FP16 / int32 storage,
real and complex data with weights and IQ beamforming, an F# window (plain
form), ragged tiles and record edges, the full-size volume on sampled voxels,
3D focusing of a point scatterer, and the entry points that are built for
separable delays only."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from synth import MM, HERCULES_2D
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


def _geom(wave, dims=(24, 20, 40), **kw):
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=1024, acq_kind=HERCULES_2D, out_dims=dims,
                       out_min=(-1.5 * MM, -1.2 * MM, 4 * MM), out_max=(1.5 * MM, 1.2 * MM, 14 * MM), **kw)
    g.tx_wave = wave
    if wave == "plane":
        g.tx_angles = (0.12,)
    else:
        g.tx_focus = -6 * MM
    return g


def _run(g, decoded, dtype="f32", variant=rc.DAS_PLAIN, interp="linear", apod=None, f_number=None):
    plan = rc.Plan(rc.make_params(g, decoded_dtype=dtype, das_variant=variant, interp=interp, f_number=f_number))
    if dtype == "cf32":
        dec = torch.from_numpy(np.stack([decoded.real, decoded.imag]).astype(np.float32)).cuda()
    else:
        tdt = {"f32": torch.float32, "f16": torch.float16, "i32": torch.int32}[dtype]
        dec = torch.from_numpy(np.asarray(decoded)).to(tdt).cuda()
    w = None if apod is None else torch.from_numpy(apod.astype(np.float32)).cuda()
    img = plan.das(dec, apod=w).cpu().numpy().astype(np.float64)
    return (img[0] + 1j * img[1] if dtype == "cf32" else img), plan.info()


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
@pytest.mark.parametrize("wave", ["plane", "point"])
@pytest.mark.parametrize("interp", ["linear", "cubic"])
@pytest.mark.parametrize("dims", [(24, 20, 40), (48, 1, 160), (1, 40, 64)])
def test_2d_aperture_matches_oracle(wave, interp, dims, variant):
    g = _geom(wave, dims=dims)
    fr = synth.make_frame(g, seed=51, n_scatterers=4, box_x=(-1 * MM, 1 * MM), box_y=(-1 * MM, 1 * MM),
                          box_z=(5 * MM, 13 * MM), noise_frac=0.0)
    want = oracle.das(g, fr.decoded.astype(np.float64), interp=interp)
    got, info = _run(g, fr.decoded, variant=variant, interp=interp)
    assert info["tiled"] == (variant == rc.DAS_TILED)
    err = rel_l2(got, want)
    print("2D aperture %s %s %s v%d (window %d): rel-L2 %.3e" % (wave, interp, dims, variant, info["window"], err))
    assert err <= TOL


def test_2d_coarse_grid_runs_the_plain_form():
    # a 32 x 32-voxel x-z tile of this grid reaches more than 128 samples
    g = _geom("plane", dims=(48, 1, 64))
    fr = synth.make_frame(g, seed=56, n_scatterers=3, box_x=(-1 * MM, 1 * MM), box_y=(0.0, 0.0),
                          box_z=(5 * MM, 13 * MM), noise_frac=0.0)
    got, info = _run(g, fr.decoded, variant=rc.DAS_TILED)
    assert not info["tiled"] and info["window"] > 128
    assert rel_l2(got, oracle.das(g, fr.decoded.astype(np.float64))) <= TOL


@pytest.mark.parametrize("wave", ["plane", "point"])
def test_tiled_2d_storage_types(wave):
    g = _geom(wave)
    fr = synth.make_frame(g, seed=54, n_scatterers=5, box_x=(-1 * MM, 1 * MM), box_y=(-1 * MM, 1 * MM),
                          box_z=(5 * MM, 13 * MM), noise_frac=0.0)
    x = fr.decoded.astype(np.float64)
    h = x.astype(np.float16)
    got, info = _run(g, h, dtype="f16", variant=rc.DAS_TILED)
    assert info["tiled"]
    assert rel_l2(got, oracle.das(g, h.astype(np.float64))) <= TOL
    q = np.round(x * 64).astype(np.int32)           # int32 storage is the decoded sum D, scaled by 1/n_tx
    got, _ = _run(g, q, dtype="i32", variant=rc.DAS_TILED)
    assert rel_l2(got, oracle.das(g, q.astype(np.float64) / g.n_tx)) <= TOL


@pytest.mark.parametrize("wave", ["plane", "point"])
@pytest.mark.parametrize("interp", ["linear", "cubic"])
def test_tiled_2d_complex_weights_and_iq(wave, interp):
    # a grid fine enough for windows of at most 64 samples (complex cubic
    # pieces have no larger tiled class)
    g = _geom(wave, dims=(48, 40, 80))
    fr = synth.make_frame(g, seed=55, n_scatterers=4, analytic=True, noise_frac=0.0, box_x=(-1 * MM, 1 * MM),
                          box_y=(-1 * MM, 1 * MM), box_z=(5 * MM, 13 * MM))
    r = fr.decoded.astype(np.complex128)
    w = np.random.default_rng(6).uniform(0.5, 1.5, g.n_ch)
    got, info = _run(g, fr.decoded, dtype="cf32", variant=rc.DAS_TILED, interp=interp, apod=w)
    print("2D complex %s %s: tiled %s window %d" % (wave, interp, info["tiled"], info["window"]))
    assert info["tiled"]
    assert rel_l2(got, oracle.das(g, r, w=w, interp=interp)) <= TOL
    g.iq_freq = 2.5e6
    got, info = _run(g, fr.decoded, dtype="cf32", variant=rc.DAS_TILED, interp=interp)
    assert info["tiled"]
    assert rel_l2(got, oracle.das(g, r, interp=interp)) <= TOL


def test_tiled_2d_ragged_tiles_and_record_edges():
    # delays run off both ends of a short record; grid sizes are not
    # multiples of the tile extents; a steered plane wave
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=384, acq_kind=HERCULES_2D, out_dims=(37, 13, 77), t0=3e-6,
                       out_min=(-1.8 * MM, -1.1 * MM, 1 * MM), out_max=(1.8 * MM, 1.1 * MM, 12 * MM))
    g.tx_wave, g.tx_angles = "plane", (-0.2,)
    r = np.random.default_rng(18).normal(size=(16, 16, 384))
    for interp in ("linear", "cubic"):
        got, info = _run(g, r.astype(np.float32), variant=rc.DAS_TILED, interp=interp)
        assert info["tiled"]
        err = rel_l2(got, oracle.das(g, r, interp=interp))
        print("2D edges %s: rel-L2 %.3e" % (interp, err))
        assert err <= TOL


def test_tiled_2d_full_volume_sampled():
    # the benchmark's workload and launch configuration: 128 rows x 128
    # columns x 2048 samples decoded to FP16, one plane wave, 128 x 128 x 256
    g = dataclasses.replace(synth.hercules_volume_geometry(), acq_kind=HERCULES_2D, hadamard_order=0)
    g.tx_wave, g.tx_angles = "plane", (0.0,)
    h = np.random.default_rng(7).normal(size=(g.n_tx, g.n_ch, g.n_samples)).astype(np.float16)
    got, info = _run(g, h, dtype="f16", variant=rc.DAS_TILED)
    assert info["tiled"]
    vox = sample_voxels(g.out_dims, 1200, seed=3)
    want = oracle.das(g, h.astype(np.float64), voxels=vox)
    err = rel_l2(got.ravel()[vox], want)
    print("2D full volume: tile %s window %d rel-L2 %.3e" % (info["tile"], info["window"], err))
    assert err <= TOL


def test_2d_aperture_focuses_a_point_in_3d():
    p = (0.375 * MM, -0.25 * MM, 9.0 * MM)          # on a grid node (x 15, y 10, z 20)
    g = _geom("plane", dims=(25, 25, 41))
    g.out_min, g.out_max = (-1.5 * MM, -1.5 * MM, 7 * MM), (1.5 * MM, 1.5 * MM, 11 * MM)
    fr = synth.make_frame(g, seed=52, n_scatterers=1, box_x=(p[0], p[0]), box_y=(p[1], p[1]), box_z=(p[2], p[2]),
                          noise_frac=0.0)
    got, _ = _run(g, fr.decoded)
    pk = np.unravel_index(np.argmax(np.abs(got)), got.shape)
    assert pk == (20, 10, 15)                       # (z, y, x) node of the point


@pytest.mark.parametrize("wave", ["plane", "point"])
def test_complex_fnumber_weights_and_iq(wave):
    g = _geom(wave)
    fr = synth.make_frame(g, seed=53, n_scatterers=4, analytic=True, noise_frac=0.0, box_x=(-1 * MM, 1 * MM),
                          box_y=(-1 * MM, 1 * MM), box_z=(5 * MM, 13 * MM))
    r = fr.decoded.astype(np.complex128)
    w = np.random.default_rng(5).uniform(0.5, 1.5, g.n_ch)
    got, info = _run(g, fr.decoded, dtype="cf32", variant=rc.DAS_TILED, apod=w, f_number=0.8)
    assert not info["tiled"]                        # the radial F# window runs the plain form
    assert rel_l2(got, oracle.das(g, r, w=w, f_number=0.8)) <= TOL
    g.iq_freq = 2.5e6                               # IQ beamforming of the same samples
    got, _ = _run(g, fr.decoded, dtype="cf32")
    assert rel_l2(got, oracle.das(g, r)) <= TOL


def test_separable_only_entry_points_reject_2d_aperture():
    g = _geom("plane")
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    dec = torch.zeros(g.n_tx, g.n_ch, g.n_samples, device="cuda")
    gi = torch.zeros(g.out_dims[2], g.out_dims[1], g.out_dims[0], device="cuda")
    with pytest.raises(rc.RcbfError) as e:
        plan.das_backward(dec, gi)
    assert e.value.code == rc.EUNSUPPORTED
    p16 = rc.Plan(rc.make_params(g, decoded_dtype="f16"))
    with pytest.raises(rc.RcbfError) as e:
        rc.Batch([p16], None, [dec.half()], [gi])
    assert e.value.code == rc.EUNSUPPORTED
    bad = _geom("point")
    bad.tx_focus = 2 * MM                           # a diverging point must lie behind the array
    with pytest.raises(rc.RcbfError) as e:
        rc.Plan(rc.make_params(bad, decoded_dtype="f32"))
    assert e.value.code == rc.EINVAL


@pytest.mark.parametrize("wave", ["plane", "point"])
def test_tiled_2d_speed_of_sound_override(wave):
    # the window and the box bounds follow the call's speed of sound
    g = _geom(wave, dims=(48, 40, 80))
    fr = synth.make_frame(g, seed=58, n_scatterers=4, box_x=(-1 * MM, 1 * MM), box_y=(-1 * MM, 1 * MM),
                          box_z=(5 * MM, 13 * MM), noise_frac=0.0)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    assert plan.info()["tiled"]
    d = torch.from_numpy(fr.decoded.astype(np.float32)).cuda()
    for c in (1420.0, 1610.0):
        got = plan.das(d, c=c).cpu().numpy().astype(np.float64)
        want = oracle.das(dataclasses.replace(g, c=c), fr.decoded.astype(np.float64))
        err = rel_l2(got, want)
        print("2D %s c=%g: rel-L2 %.3e" % (wave, c, err))
        assert err <= TOL
