"""Transmit and channel counts that are not powers of two on the GPU: the
tiled DAS walks its (transmit group, channel chunk) stages with a division of
the stage index by the number of transmit groups (3, 5 or 6 here), the
adjoint likewise (its own group sizes), and the batched stream splits the
tiles of a phase's tail into ordered channel halves only when the channel
chunks divide evenly. Each
result is checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from synth import MM
from tests._frames import rel_l2

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


def _geom(n_tx, n_ch, **kw):
    return synth.Geometry(n_tx=n_tx, n_ch=n_ch, n_samples=512, out_dims=(96, 1, 160),
                          out_min=(-2 * MM, 0.0, 3 * MM), out_max=(2 * MM, 0.0, 8 * MM), **kw)


@pytest.mark.parametrize("n_tx,n_ch,interp", [(24, 40, "linear"), (40, 24, "linear"), (24, 40, "cubic"),
                                              (48, 56, "linear")])
def test_tiled_das_odd_counts(n_tx, n_ch, interp):
    g = _geom(n_tx, n_ch, interp=interp)
    r = np.random.default_rng(n_tx + n_ch).normal(size=(n_tx, n_ch, 512))
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32", das_variant=rc.DAS_TILED, interp=interp))
    assert plan.info()["tiled"]
    got = plan.das(torch.from_numpy(r.astype(np.float32)).cuda()).cpu().numpy()
    err = rel_l2(got, oracle.das(g, r, interp=interp))
    print("n_tx %d n_ch %d %s: rel-L2 %.2e" % (n_tx, n_ch, interp, err))
    assert err <= TOL


@pytest.mark.parametrize("cplx", [False, True])
def test_adjoint_odd_counts(cplx):
    # 24 transmits (six groups of four), 24 channels (six chunks of four)
    g = _geom(24, 24, f_number=0.8)
    rng = np.random.default_rng(7 + cplx)
    r = rng.normal(size=(24, 24, 512))
    G = rng.normal(size=(160, 1, 96))
    if cplx:
        r = r + 1j * rng.normal(size=r.shape)
        G = G + 1j * rng.normal(size=G.shape)
    w = rng.uniform(0.5, 1.5, 24)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32" if cplx else "f32", das_variant=rc.DAS_TILED))
    assert plan.info()["bwd_mode"] == 2          # the adjoint's own tiled form
    to_dev = (lambda x: torch.from_numpy(np.stack([x.real, x.imag]).astype(np.float32)).cuda()) if cplx else \
        (lambda x: torch.from_numpy(np.asarray(x, dtype=np.float32)).cuda())
    grf, gc, gw = plan.das_backward(to_dev(r), to_dev(G), apod=torch.from_numpy(w.astype(np.float32)).cuda())
    want_rf, want_c, want_w = oracle.das_grad(g, r, G, w=w)
    got_rf = grf.cpu().numpy().astype(np.float64)
    if cplx:
        got_rf = got_rf[0] + 1j * got_rf[1]
    assert rel_l2(got_rf, want_rf) <= 1e-3
    assert abs(float(gc.cpu()) - want_c) <= 1e-3 * abs(want_c)
    assert rel_l2(gw.cpu().numpy().astype(np.float64), want_w) <= 1e-3


def test_batch_odd_channel_chunks_and_halves():
    # frames whose channel chunks cannot be halved (5 chunks) beside frames
    # whose chunks can (6 chunks): each phase picks its own split
    frames, plans, dec, img = [], [], [], []
    for k, (n_tx, n_ch) in enumerate([(24, 40), (24, 48), (40, 40)]):
        g = _geom(n_tx, n_ch)
        r = np.random.default_rng(50 + k).normal(size=(n_tx, n_ch, 512)).astype(np.float16)
        frames.append((g, r))
        plans.append(rc.Plan(rc.make_params(g, decoded_dtype="f16", das_variant=rc.DAS_TILED, tile=(32, 1, 32))))
        dec.append(torch.from_numpy(r).cuda())
        img.append(torch.empty(160, 1, 96, device="cuda"))
    batch = rc.Batch(plans, None, dec, img)
    batch.run()
    assert batch.status() == rc.OK
    for k, (g, r) in enumerate(frames):
        got = img[k].cpu().numpy()
        assert rel_l2(got, plans[k].das(dec[k]).cpu().numpy()) <= 1e-5
        assert rel_l2(got, oracle.das(g, r.astype(np.float64))) <= TOL
