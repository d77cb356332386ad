"""Plane-wave (TPW) and virtual-line-source (VLS) transmits on the GPU
against the FP64 oracle: tiled and plain DAS (linear and cubic, real and
complex with an F# window), the adjoint, and a batch of plane-wave frames; the
VLS focus inside the image (tiles across the focal depth run the plain form,
the others the tiled one, with and without a channel split), above it, and
behind the array (a diverging wave)."""
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


def _geom(wave, n_tx=16, **kw):
    g = synth.Geometry(n_tx=n_tx, n_ch=32, n_samples=1024, out_dims=(128, 1, 320),
                       out_min=(-3 * MM, 0.0, 3 * MM), out_max=(3 * MM, 0.0, 18 * MM), **kw)
    g.tx_wave = wave
    if wave == "plane":
        g.tx_angles = tuple(np.deg2rad(np.linspace(-15, 15, n_tx)))
    return g


def _image(g, decoded, dtype="f32", variant=rc.DAS_TILED, interp="linear", apod=None, f_number=None):
    plan = rc.Plan(rc.make_params(g, decoded_dtype=dtype, das_variant=variant, interp=interp, f_number=f_number))
    if dtype == "cf32":
        dec = torch.from_numpy(np.stack([decoded.real, decoded.imag]).astype(np.float32)).cuda()
    else:
        dec = torch.from_numpy(decoded.astype(np.float32)).cuda()
    w = None if apod is None else torch.from_numpy(apod.astype(np.float32)).cuda()
    img = plan.das(dec, apod=w).cpu().numpy().astype(np.float64)
    return (img[0] + 1j * img[1] if dtype == "cf32" else img), plan.info()


CASES = [("plane", {}), ("vls", {"tx_focus": 8 * MM}), ("vls", {"tx_focus": 25 * MM}),
         ("vls", {"tx_focus": -4 * MM})]


@pytest.mark.parametrize("wave,kw", CASES)
@pytest.mark.parametrize("variant,interp", [(rc.DAS_TILED, "linear"), (rc.DAS_TILED, "cubic"),
                                            (rc.DAS_PLAIN, "linear")])
def test_transmit_wave_das_matches_oracle(wave, kw, variant, interp):
    g = _geom(wave, **kw)
    fr = synth.make_frame(g, seed=41, n_scatterers=6, box_x=(-2.5 * MM, 2.5 * MM), box_z=(4 * MM, 17 * MM),
                          noise_frac=0.0)
    want = oracle.das(g, fr.decoded.astype(np.float64), interp=interp)
    got, info = _image(g, fr.decoded, variant=variant, interp=interp)
    err = rel_l2(got, want)
    print("%s %s v%d %s: tiled %s window %d rel-L2 %.3e" % (wave, kw, variant, interp, info["tiled"],
                                                             info["window"], err))
    # a virtual-line-source focus inside the image (8 mm) makes the transmit
    # delay jump at the focal depth off axis: the tiles across it run the
    # plain form, every other tile the tiled form
    assert info["tiled"] == (variant == rc.DAS_TILED)
    assert err <= TOL
    # the image of the wave's own data focuses: its peak is within a few voxels of a scatterer
    pk = np.unravel_index(np.argmax(np.abs(got)), got.shape)
    pos = np.array([g.out_min[0] + pk[2] * (g.out_max[0] - g.out_min[0]) / (g.out_dims[0] - 1),
                    g.out_min[2] + pk[0] * (g.out_max[2] - g.out_min[2]) / (g.out_dims[2] - 1)])
    d = np.min(np.hypot(fr.scatterers[:, 0] - pos[0], fr.scatterers[:, 2] - pos[1]))
    assert d < 0.3 * MM


@pytest.mark.parametrize("wave,kw", CASES[:2])
def test_complex_with_fnumber_and_weights(wave, kw):
    g = _geom(wave, **kw)
    fr = synth.make_frame(g, seed=43, n_scatterers=6, analytic=True, noise_frac=0.0,
                          box_x=(-2.5 * MM, 2.5 * MM), box_z=(4 * MM, 17 * MM))
    w = np.random.default_rng(4).uniform(0.5, 1.5, g.n_ch)
    r = fr.decoded.astype(np.complex128)
    want = oracle.das(g, r, w=w, f_number=1.0)
    for variant in (rc.DAS_TILED, rc.DAS_PLAIN):
        got, _ = _image(g, fr.decoded, dtype="cf32", variant=variant, apod=w, f_number=1.0)
        assert rel_l2(got, want) <= TOL


@pytest.mark.parametrize("wave,kw", CASES[:2])
def test_adjoint_with_transmit_waves(wave, kw):
    g = _geom(wave, **kw)
    rng = np.random.default_rng(44)
    r = rng.normal(size=(g.n_tx, g.n_ch, g.n_samples))
    G = rng.normal(size=(g.out_dims[2], g.out_dims[1], g.out_dims[0]))
    w = rng.uniform(0.5, 1.5, g.n_ch)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    grf, _, gw = plan.das_backward(torch.from_numpy(r.astype(np.float32)).cuda(),
                                   torch.from_numpy(G.astype(np.float32)).cuda(),
                                   apod=torch.from_numpy(w.astype(np.float32)).cuda(), c=1500.0)
    want_rf, _, want_w = oracle.das_grad(g, r, G, w=w, c=1500.0)
    assert rel_l2(grf.cpu().numpy(), want_rf) <= TOL
    assert rel_l2(gw.cpu().numpy(), want_w) <= TOL


def test_batch_of_plane_wave_frames():
    g = _geom("plane", n_tx=32, hadamard_order=32)
    fr = synth.make_frame(g, seed=45, n_scatterers=6, box_x=(-2.5 * MM, 2.5 * MM), box_z=(4 * MM, 17 * MM))
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f16", tile=(64, 1, 16)))
    rf = [torch.from_numpy(fr.rf).cuda() for _ in range(2)]
    dec = [torch.empty(32, 32, 1024, dtype=torch.float16, device="cuda") for _ in range(2)]
    img = [torch.empty(plan.image_shape, device="cuda") for _ in range(2)]
    batch = rc.Batch([plan, plan], rf, dec, img)
    batch.run()
    assert batch.status() == rc.OK
    h = oracle.decoded_as(oracle.decode(fr.rf), 32, "f16").astype(np.float64)
    vox = sample_voxels(g.out_dims, 800, seed=6)
    want = oracle.das(g, h, voxels=vox)
    for k in range(2):
        assert rel_l2(img[k].cpu().numpy().ravel()[vox], want) <= TOL


@pytest.mark.parametrize("focus_mm,dtype", [(8.0, "f32"), (11.0, "f16"), (3.0, "f32"), (18.0, "f32")])
def test_vls_focal_plane_split_full_image(focus_mm, dtype):
    # the focal depth inside the image, on a tile row boundary or at the
    # image's top and bottom rows; FP16 storage; the split works for any
    # channel split of the plan
    g = _geom("vls", n_tx=32, tx_focus=focus_mm * MM)
    g.n_ch = 64
    fr = synth.make_frame(g, seed=46, n_scatterers=6, box_x=(-2.5 * MM, 2.5 * MM), box_z=(4 * MM, 17 * MM),
                          noise_frac=0.0)
    data = fr.decoded.astype(np.float16).astype(np.float64) if dtype == "f16" else fr.decoded.astype(np.float64)
    want = oracle.das(g, data)
    plan = rc.Plan(rc.make_params(g, decoded_dtype=dtype))
    assert plan.info()["tiled"]
    dec = torch.from_numpy(data.astype(np.float16 if dtype == "f16" else np.float32)).cuda()
    got = plan.das(dec).cpu().numpy().astype(np.float64)
    err = rel_l2(got, want)
    print("VLS focus %.1f mm %s: split %d, rel-L2 %.3e" % (focus_mm, dtype, plan.info()["n_split"], err))
    assert err <= TOL


def test_batch_rejects_a_vls_focal_plane_inside_the_image():
    g = _geom("vls", n_tx=32, hadamard_order=32, tx_focus=8 * MM)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f16"))
    rf = [torch.zeros(32, 32, 1024, dtype=torch.int16, device="cuda")]
    dec = [torch.empty(32, 32, 1024, dtype=torch.float16, device="cuda")]
    img = [torch.empty(plan.image_shape, device="cuda")]
    with pytest.raises(rc.RcbfError) as e:
        rc.Batch([plan], rf, dec, img)
    assert e.value.code == rc.EUNSUPPORTED


@pytest.mark.parametrize("variant", ["das", "adjoint"])
def test_vls_focus_inside_a_ragged_last_tile(variant):
    # 291 depth rows with 16-row tiles: the last tile holds 3 real rows (17.4 to
    # 17.5 mm) and its reference sits at its centre (17.775 mm). A focal depth
    # of 17.6 mm lies below every real voxel but inside that tile's box, so the
    # real voxels and the tile's reference are on opposite sides of the focus:
    # that tile must run the plain form (its tiled windows would take the
    # transmit delay with the reference's sign)
    g = synth.Geometry(n_tx=16, n_ch=32, n_samples=1024, out_dims=(128, 1, 291),
                       out_min=(-3 * MM, 0.0, 3 * MM), out_max=(3 * MM, 0.0, 17.5 * MM))
    g.tx_wave, g.tx_focus = "vls", 17.6 * MM
    fr = synth.make_frame(g, seed=48, n_scatterers=6, box_x=(-2.5 * MM, 2.5 * MM), box_z=(15 * MM, 17.5 * MM),
                          noise_frac=0.0)
    data = fr.decoded.astype(np.float64)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32", tile=(64, 1, 16)))
    assert plan.info()["tiled"]
    dec = torch.from_numpy(data.astype(np.float32)).cuda()
    if variant == "das":
        want = oracle.das(g, data)
        got = plan.das(dec).cpu().numpy().astype(np.float64)
        tail = rel_l2(got[-3:], want[-3:])
        err = rel_l2(got, want)
        print("VLS focus in the ragged last tile: rel-L2 %.3e (last 3 rows %.3e)" % (err, tail))
        assert err <= TOL and tail <= TOL
    else:
        # the autofocus loss gradient G = dL/dI = -2 I; every adjoint tile that
        # reaches the focal depth keeps the adjoint off its tiled forms
        G = -2.0 * oracle.das(g, data)
        gr, gc, gw = plan.das_backward(dec, torch.from_numpy(G.astype(np.float32)).cuda())
        wr, wc, ww = oracle.das_grad(g, data, G)
        err = rel_l2(gr.cpu().numpy(), wr)
        print("VLS focus in the ragged last tile, adjoint: dR rel-L2 %.3e, dc %.6e vs %.6e" % (err, gc.item(), wc))
        assert err <= 1e-4
        assert abs(gc.item() - wc) <= 1e-2 * abs(wc)     # FP32 delays of the plain form
        assert rel_l2(gw.cpu().numpy(), ww) <= 1e-4
