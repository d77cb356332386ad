"""DAS parity on the GPU: the library's delay-and-sum (through the C ABI)
against the FP64 oracle of Eq. (1)-(3), within relative L2 1e-4 (the bound
the method is graded at), with the max-abs error printed. Full images where
the oracle is fast, sampled voxels (plus the grid corners) at full size."""
import numpy as np
import pytest

import oracle
import synth
from synth import MM
from tests._frames import frame, rel_l2, sample_voxels

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


def _decoded_exact(fr):
    D = oracle.decode(fr.rf)
    return D, D.astype(np.float64) / fr.geometry.n_tx


def _gpu_image(g, decoded_np, dtype="f32", variant=rc.DAS_TILED, tile=None, apod=None, c=0.0, **kw):
    plan = rc.Plan(rc.make_params(g, decoded_dtype=dtype, das_variant=variant, tile=tile, **kw))
    if np.iscomplexobj(decoded_np):
        dec = torch.from_numpy(np.stack([decoded_np.real, decoded_np.imag]).astype(np.float32)).cuda()
    else:
        tdt = {"f32": torch.float32, "f16": torch.float16, "i32": torch.int32}[dtype]
        dec = torch.from_numpy(np.asarray(decoded_np)).to(tdt).cuda()
    w = None if apod is None else torch.from_numpy(np.asarray(apod, dtype=np.float32)).cuda()
    img = plan.das(dec, apod=w, c=c)
    torch.cuda.synchronize()
    out = img.cpu().numpy().astype(np.float64)
    if np.iscomplexobj(decoded_np):
        out = out[0] + 1j * out[1]
    return out


def _report(tag, got, want):
    err = rel_l2(got, want)
    mx = float(np.max(np.abs(np.asarray(got) - np.asarray(want))))
    print("%s: rel-L2 %.3e  max-abs %.3e (peak %.3e)" % (tag, err, mx, float(np.max(np.abs(want)))))
    return err


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
def test_tiny_bscan_full_image(variant):
    fr = frame("tiny")
    g = fr.geometry
    _, exact = _decoded_exact(fr)
    want = oracle.das(g, exact)
    got = _gpu_image(g, exact.astype(np.float32), variant=variant)
    assert _report("tiny v%d" % variant, got, want) <= TOL


def _dense_tiny():
    # the tiny acquisition on a grid fine enough for every tile shape to stay
    # within the tiled kernel's 128-sample window
    fr = frame("tiny")
    g = synth.tiny_bscan_geometry()
    g.out_dims = (128, 1, 512)
    return fr, g


@pytest.mark.parametrize("tile", [(32, 1, 32), (64, 1, 16), (128, 1, 8)])
def test_tiny_bscan_every_tile_shape(tile):
    fr, g = _dense_tiny()
    _, exact = _decoded_exact(fr)
    vox = sample_voxels(g.out_dims, 6000, seed=5)
    want = oracle.das(g, exact, voxels=vox)
    got = _gpu_image(g, exact.astype(np.float32), tile=tile).ravel()[vox]
    assert _report("tiny tile %s" % (tile,), got, want) <= TOL


def test_coarse_grid_runs_plain_form():
    # 1024-voxel tiles of this grid reach more than 128 samples: the library
    # runs the plain GPU form, still within the bound
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=512, out_dims=(40, 12, 20),
                       out_min=(-1.5 * MM, -1 * MM, 3 * MM), out_max=(1.5 * MM, 1 * MM, 9 * MM))
    r = np.random.default_rng(31).normal(size=(16, 16, 512))
    got = _gpu_image(g, r.astype(np.float32))
    assert _report("coarse volume", got, oracle.das(g, r)) <= TOL


def test_full_bscan_sampled_voxels_f32():
    fr = frame("bscan")
    g = fr.geometry
    _, exact = _decoded_exact(fr)
    vox = sample_voxels(g.out_dims, 3000, seed=1)
    want = oracle.das(g, exact, voxels=vox)
    got = _gpu_image(g, exact.astype(np.float32)).ravel()[vox]
    assert _report("bscan f32", got, want) <= TOL


def test_full_bscan_sampled_voxels_f16_storage():
    # FP16-stored decoded RF: the DAS arithmetic is held to the bound against
    # the oracle run on the same FP16-rounded samples; the storage rounding
    # itself is reported against the exact decode.
    fr = frame("bscan")
    g = fr.geometry
    D, exact = _decoded_exact(fr)
    r16 = oracle.decoded_as(D, g.n_tx, "f16")
    vox = sample_voxels(g.out_dims, 3000, seed=2)
    got = _gpu_image(g, r16, dtype="f16").ravel()[vox]
    assert _report("bscan f16 vs oracle(f16 data)", got, oracle.das(g, r16.astype(np.float64), voxels=vox)) <= TOL
    _report("bscan f16 vs exact decode (storage error, stated)", got, oracle.das(g, exact, voxels=vox))


def test_full_bscan_f_number_and_weights_sampled():
    # the full frame runs its channel split with a tail of channel parts in
    # partial images of their own (512 tiles: 2 splits, the last 3/4 wave in
    # quarters); with the F# window and channel weights the units also skip
    # the chunks outside their aperture
    fr = frame("bscan")
    g = fr.geometry
    _, exact = _decoded_exact(fr)
    w = np.random.default_rng(8).uniform(0.5, 1.5, g.n_ch)
    vox = sample_voxels(g.out_dims, 2000, seed=5)
    want = oracle.das(g, exact, w=w, f_number=1.0, voxels=vox)
    got = _gpu_image(g, exact.astype(np.float32), apod=w, f_number=1.0).ravel()[vox]
    assert _report("bscan F#1 + w", got, want) <= TOL


def test_full_bscan_plain_form_sampled():
    fr = frame("bscan")
    g = fr.geometry
    _, exact = _decoded_exact(fr)
    vox = sample_voxels(g.out_dims, 1500, seed=3)
    want = oracle.das(g, exact, voxels=vox)
    got = _gpu_image(g, exact.astype(np.float32), variant=rc.DAS_PLAIN).ravel()[vox]
    # the plain FP32 form is the baseline the tuned form is measured against:
    # it is held to the same bound
    assert _report("bscan plain FP32", got, want) <= TOL


def test_volume_sampled_voxels():
    fr = frame("volume")
    g = fr.geometry
    _, exact = _decoded_exact(fr)
    vox = sample_voxels(g.out_dims, 1500, seed=4)
    want = oracle.das(g, exact, voxels=vox)
    got = _gpu_image(g, exact.astype(np.float32)).ravel()[vox]
    assert _report("volume f32", got, want) <= TOL


def test_int32_decoded_input_is_scaled():
    fr = frame("tiny")
    g = fr.geometry
    D, exact = _decoded_exact(fr)
    got = _gpu_image(g, D.astype(np.int32), dtype="i32")
    assert _report("tiny i32", got, oracle.das(g, exact)) <= TOL


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
def test_f_number_and_channel_weights(variant):
    fr = frame("tiny")
    g = fr.geometry
    _, exact = _decoded_exact(fr)
    w = np.random.default_rng(3).uniform(0.5, 1.5, g.n_ch)
    want = oracle.das(g, exact, w=w, f_number=1.2)
    got = _gpu_image(g, exact.astype(np.float32), variant=variant, apod=w, f_number=1.2)
    assert _report("tiny F#1.2 + w", got, want) <= TOL


def test_speed_of_sound_override():
    fr = frame("tiny")
    g = fr.geometry
    _, exact = _decoded_exact(fr)
    got = _gpu_image(g, exact.astype(np.float32), c=1480.0)
    assert _report("tiny c=1480", got, oracle.das(g, exact, c=1480.0)) <= TOL


def test_complex_input():
    g = synth.Geometry(n_tx=32, n_ch=32, n_samples=1024, out_dims=(128, 1, 256),
                       out_min=(-3 * MM, 0.0, 4 * MM), out_max=(3 * MM, 0.0, 14 * MM))
    fr = synth.make_frame(g, seed=9, n_scatterers=6, analytic=True, noise_frac=0.0)
    r = fr.decoded.astype(np.complex128)
    want = oracle.das(g, r)
    for variant in (rc.DAS_TILED, rc.DAS_PLAIN):
        got = _gpu_image(g, fr.decoded, dtype="cf32", variant=variant)
        assert _report("complex v%d" % variant, got, want) <= TOL


def test_ragged_tiles_and_record_edges():
    # image sizes that are not tile multiples, and a time origin that puts
    # part of every window before sample 0 or past the end of the record
    for k, t0 in enumerate((-8e-6, 0.0, 30e-6)):
        g = synth.Geometry(n_tx=32, n_ch=16, n_samples=1024, t0=t0, out_dims=(70, 1, 450),
                           out_min=(-2 * MM, 0.0, 2 * MM), out_max=(2 * MM, 0.0, 28 * MM))
        rng = np.random.default_rng(50 + k)
        r = rng.normal(size=(g.n_tx, g.n_ch, g.n_samples))
        want = oracle.das(g, r)
        got = _gpu_image(g, r.astype(np.float32))
        assert _report("ragged t0=%g" % t0, got, want) <= TOL


def test_cross_plane_orientation_swap():
    # second plane of a cross-plane pair: columns transmit, rows receive,
    # image in the y-z plane (nx = 1)
    g = synth.Geometry(n_tx=32, n_ch=32, n_samples=1024, tx_orientation=synth.COLUMNS,
                       rx_orientation=synth.ROWS, hadamard_order=32, out_dims=(1, 128, 256),
                       out_min=(0.0, -3 * MM, 4 * MM), out_max=(0.0, 3 * MM, 16 * MM))
    fr = synth.make_frame(g, seed=21, n_scatterers=5, box_y=(-2 * MM, 2 * MM))
    D = oracle.decode(fr.rf)
    exact = D.astype(np.float64) / g.n_tx
    want = oracle.das(g, exact)
    got = _gpu_image(g, exact.astype(np.float32))
    assert _report("cross-plane y-z", got, want) <= TOL


def test_small_volume_every_row_split():
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=512, out_dims=(70, 16, 48),
                       out_min=(-1.5 * MM, -0.5 * MM, 3 * MM), out_max=(1.5 * MM, 0.5 * MM, 4.5 * MM))
    r = np.random.default_rng(31).normal(size=(16, 16, 512))
    want = oracle.das(g, r)
    for tile in [(32, 4, 8), (32, 1, 32), (64, 2, 8), (64, 16, 1), (128, 1, 8)]:
        got = _gpu_image(g, r.astype(np.float32), tile=tile)
        assert _report("volume tile %s" % (tile,), got, want) <= TOL


def test_point_scatterer_peak_matches_oracle():
    g = synth.Geometry(n_tx=32, n_ch=32, n_samples=1024, hadamard_order=32, out_dims=(81, 1, 81),
                       out_min=(-2 * MM, 0.0, 8 * MM), out_max=(2 * MM, 0.0, 12 * MM))
    node = (54, 0, 26)
    p = [g.out_min[d] + node[d] * (g.out_max[d] - g.out_min[d]) / max(g.out_dims[d] - 1, 1) for d in range(3)]
    fr = synth.make_frame(g, seed=0, n_scatterers=1, box_x=(p[0], p[0]), box_z=(p[2], p[2]), noise_frac=0.0)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    img = plan.das(plan.decode(torch.from_numpy(fr.rf).cuda())).cpu().numpy()
    iz, iy, ix = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    assert (ix, iy, iz) == node


@pytest.mark.parametrize("dtype,cubic", [("f32", False), ("f16", False), ("f32", True)])
def test_f_number_chunk_skip_and_tiles_outside_every_aperture(dtype, cubic):
    # lateral extent ±8 mm against a 3.2 mm array and F# = 3: tiles beyond
    # about 3 mm from the array have no channel chunk inside their window
    # (the unit sums nothing) and shallow tiles keep only a few chunks; the
    # image must equal the oracle's, with exact zeros where every weight is 0
    g = synth.Geometry(n_tx=32, n_ch=32, n_samples=1024, hadamard_order=0, out_dims=(256, 1, 160),
                       out_min=(-8 * MM, 0.0, 2 * MM), out_max=(8 * MM, 0.0, 10 * MM))
    if cubic:
        g.interp = "cubic"
    r = np.random.default_rng(19).normal(size=(32, 32, 1024))
    w = np.random.default_rng(20).uniform(0.5, 1.5, 32)
    data = r.astype(np.float16).astype(np.float64) if dtype == "f16" else r
    want = oracle.das(g, data, w=w, f_number=3.0, interp="cubic" if cubic else "linear")
    got = _gpu_image(g, data if dtype == "f32" else data.astype(np.float16), dtype=dtype, apod=w, f_number=3.0)
    assert _report("F#3 wide grid %s cubic=%s" % (dtype, cubic), got, want) <= TOL
    dead = want == 0.0
    assert dead.sum() > 0.2 * dead.size                 # many voxels lie outside every aperture
    assert np.all(got[dead] == 0.0)
