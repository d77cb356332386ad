"""Cubic Hermite DAS on the GPU (through the C ABI) against the FP64 oracle
with the same interpolation: every tile shape and window class, FP32 / FP16 /
int32 storage, complex data (tiled, and the plain form where a complex cubic
window exceeds 64 samples), F# window with channel weights, record edges, the
full-size B-scan, and the entry points that are built for linear
interpolation only."""
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


def _exact(fr):
    D = oracle.decode(fr.rf)
    return D, D.astype(np.float64) / fr.geometry.n_tx


def _run(g, decoded, dtype="f32", variant=rc.DAS_TILED, tile=None, apod=None, c=0.0, f_number=None):
    plan = rc.Plan(rc.make_params(g, decoded_dtype=dtype, das_variant=variant, tile=tile,
                                  f_number=f_number, interp="cubic"))
    if dtype == "cf32":
        dec = torch.from_numpy(np.stack([decoded.real, decoded.imag]).astype(np.float32)).cuda()
    else:
        tdt = {"f32": torch.float32, "f16": torch.float16, "i32": torch.int32}[dtype]
        dec = torch.from_numpy(np.asarray(decoded)).to(tdt).cuda()
    w = None if apod is None else torch.from_numpy(np.asarray(apod, dtype=np.float32)).cuda()
    img = plan.das(dec, apod=w, c=c).cpu().numpy().astype(np.float64)
    if dtype == "cf32":
        img = img[0] + 1j * img[1]
    return img, plan.info()


def _check(tag, got, want, tol=TOL):
    err = rel_l2(got, want)
    mx = float(np.max(np.abs(np.asarray(got) - np.asarray(want))))
    print("%s: rel-L2 %.3e  max-abs %.3e (peak %.3e)" % (tag, err, mx, float(np.max(np.abs(want)))))
    assert err <= tol


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
def test_tiny_bscan_full_image(variant):
    fr = frame("tiny")
    g = fr.geometry
    _, exact = _exact(fr)
    want = oracle.das(g, exact, interp="cubic")
    got, info = _run(g, exact.astype(np.float32), variant=variant)
    assert info["tiled"] == (variant == rc.DAS_TILED)
    _check("cubic tiny v%d" % variant, got, want)
    # the cubic image differs from the linear one by far more than the bound
    assert rel_l2(want, oracle.das(g, exact)) > 10 * TOL


@pytest.mark.parametrize("tile", [(32, 1, 32), (64, 1, 16), (128, 1, 8)])
@pytest.mark.parametrize("nz", [512, 1024, 2048])
def test_every_tile_shape_and_window_class(tile, nz):
    fr = frame("tiny")
    g = synth.tiny_bscan_geometry()
    g.out_dims = (128, 1, nz)
    _, exact = _exact(fr)
    vox = sample_voxels(g.out_dims, 4000, seed=nz)
    want = oracle.das(g, exact, voxels=vox, interp="cubic")
    got, info = _run(g, exact.astype(np.float32), tile=tile)
    print("tile %s nz %d: window %d tiled %s" % (tile, nz, info["window"], info["tiled"]))
    _check("cubic tile %s nz %d" % (tile, nz), got.ravel()[vox], want)


def test_f16_and_int32_storage():
    fr = frame("tiny")
    g = fr.geometry
    D, exact = _exact(fr)
    h = oracle.decoded_as(D, g.n_tx, "f16")
    got, _ = _run(g, h, dtype="f16")
    _check("cubic f16", got, oracle.das(g, h.astype(np.float64), interp="cubic"))
    got, _ = _run(g, D.astype(np.int32), dtype="i32")
    _check("cubic i32", got, oracle.das(g, exact, interp="cubic"))


@pytest.mark.parametrize("nz,expect_tiled", [(1024, True), (256, False)])
def test_complex_input(nz, expect_tiled):
    # complex cubic pieces have no 128-interval class: the coarser grid's
    # windows exceed 64 samples and run the plain form
    g = synth.Geometry(n_tx=32, n_ch=32, n_samples=1024, out_dims=(128, 1, nz),
                       out_min=(-3 * MM, 0.0, 4 * MM), out_max=(3 * MM, 0.0, 14 * MM))
    fr = synth.make_frame(g, seed=9, n_scatterers=6, analytic=True, noise_frac=0.0)
    r = fr.decoded.astype(np.complex128)
    got, info = _run(g, fr.decoded, dtype="cf32")
    print("complex cubic nz %d: window %d tiled %s" % (nz, info["window"], info["tiled"]))
    assert info["tiled"] == expect_tiled
    _check("cubic complex nz %d" % nz, got, oracle.das(g, r, interp="cubic"))


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
def test_f_number_and_channel_weights(variant):
    fr = frame("tiny")
    g = fr.geometry
    _, exact = _exact(fr)
    w = np.random.default_rng(3).uniform(0.5, 1.5, g.n_ch)
    want = oracle.das(g, exact, w=w, f_number=1.2, interp="cubic")
    got, _ = _run(g, exact.astype(np.float32), variant=variant, apod=w, f_number=1.2)
    _check("cubic F#1.2 + w v%d" % variant, got, want)


def test_ragged_tiles_and_record_edges():
    # delays run off both ends of a short record (t0 after the shallowest
    # echoes, record shorter than the deepest); grid sizes are not multiples
    # of the tile extents
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=256, out_dims=(77, 1, 301), t0=2e-6,
                       out_min=(-2 * MM, 0.0, 1 * MM), out_max=(2 * MM, 0.0, 9 * MM))
    rng = np.random.default_rng(17)
    r = rng.normal(size=(16, 16, 256))
    want = oracle.das(g, r, interp="cubic")
    for variant in (rc.DAS_TILED, rc.DAS_PLAIN):
        got, _ = _run(g, r.astype(np.float32), variant=variant)
        _check("cubic edges v%d" % variant, got, want)


def test_full_bscan_sampled_voxels_f16():
    # the benchmark's workload and launch configuration, 128 x 128 x 4096
    # decoded to FP16, 512 x 1024 image
    fr = frame("bscan")
    g = fr.geometry
    D = oracle.decode(fr.rf)
    h = oracle.decoded_as(D, g.n_tx, "f16")
    vox = sample_voxels(g.out_dims, 1500, seed=2)
    want = oracle.das(g, h.astype(np.float64), voxels=vox, interp="cubic")
    got, info = _run(g, h, dtype="f16")
    assert info["tiled"]
    _check("cubic full B-scan f16", got.ravel()[vox], want)


def test_linear_only_entry_points_reject_cubic():
    g = synth.tiny_bscan_geometry()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32", interp="cubic"))
    dec = torch.zeros(g.n_tx, g.n_ch, g.n_samples, device="cuda")
    gi = torch.zeros(g.out_dims[2], g.out_dims[1], g.out_dims[0], device="cuda")
    with pytest.raises(rc.RcbfError) as e:
        plan.das_backward(dec, gi)
    assert e.value.code == rc.EUNSUPPORTED
    p16 = rc.Plan(rc.make_params(g, decoded_dtype="f16", interp="cubic", tile=(64, 1, 16)))
    d16 = torch.zeros(g.n_tx, g.n_ch, g.n_samples, dtype=torch.float16, device="cuda")
    with pytest.raises(rc.RcbfError) as e:
        rc.Batch([p16], None, [d16], [gi])
    assert e.value.code == rc.EUNSUPPORTED
