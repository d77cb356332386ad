"""DAS adjoint on the GPU (through the C ABI): the adjoint identity, the FP64
oracle's gradients, and central finite differences of the speed of sound on
the autofocus workload (128 x 128 x 2048 complex RF, 256 x 512 image)."""
import numpy as np
import pytest

import oracle
import synth
from synth import MM
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


def _small(fnum=0.0, dims=(96, 1, 192), cplx=False):
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=512, out_dims=dims, f_number=fnum,
                       out_min=(-2 * MM, 0.0, 3 * MM), out_max=(2 * MM, 0.0, 7 * MM))
    rng = np.random.default_rng(40 + int(fnum * 10) + cplx)
    r = rng.normal(size=(16, 16, 512))
    if cplx:
        r = r + 1j * rng.normal(size=(16, 16, 512))
    G = rng.normal(size=(dims[2], dims[1], dims[0]))
    if cplx:
        G = G + 1j * rng.normal(size=G.shape)
    w = rng.uniform(0.5, 1.5, 16)
    return g, r, G, w


def _to_dev(x):
    if np.iscomplexobj(x):
        return torch.from_numpy(np.stack([x.real, x.imag]).astype(np.float32)).cuda()
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).cuda()


def _from_dev(t, cplx):
    a = t.cpu().numpy().astype(np.float64)
    return a[0] + 1j * a[1] if cplx else a


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
@pytest.mark.parametrize("cplx", [False, True])
def test_adjoint_dot_product_identity(variant, cplx):
    g, r, G, w = _small(fnum=0.8, cplx=cplx)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32" if cplx else "f32", das_variant=variant))
    dr, dw = _to_dev(r), _to_dev(w)
    img = _from_dev(plan.das(dr, apod=dw), cplx)
    grf, _, _ = plan.das_backward(dr, _to_dev(G), apod=dw)
    lhs = float(np.real(np.vdot(G.ravel(), img.ravel())) if cplx else np.sum(img * G))
    grf = _from_dev(grf, cplx)
    rhs = float(np.real(np.vdot(grf.ravel(), r.ravel())) if cplx else np.sum(grf * r))
    print("dot test v%d cplx=%s: %.9e vs %.9e" % (variant, cplx, lhs, rhs))
    assert lhs == pytest.approx(rhs, rel=1e-4)


def _scatter_case(cplx):
    # band-limited RF from point scatterers and the coherent autofocus loss
    # L = -sum |I|^2 (G = -2 I): dL/dc is then well conditioned. (With white
    # noise RF, whether an FP32 delay lands just below or above an integer
    # sample swaps in an unrelated slope, and a random-sign sum of such terms
    # makes dL/dc itself ill conditioned.)
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=512, out_dims=(96, 1, 192), f_number=0.6,
                       out_min=(-2 * MM, 0.0, 3 * MM), out_max=(2 * MM, 0.0, 7 * MM))
    fr = synth.make_frame(g, seed=77, n_scatterers=5, box_z=(3.5 * MM, 6.5 * MM), c_true=1500.0,
                          analytic=cplx, noise_frac=0.0)
    r = fr.decoded.astype(np.complex128 if cplx else np.float64)
    w = np.random.default_rng(78).uniform(0.5, 1.5, 16)
    return g, r, w


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
@pytest.mark.parametrize("cplx", [False, True])
def test_gradients_match_oracle(variant, cplx):
    # RF and apodization gradients: exact linear functionals, white-noise data
    g, r, G, w = _small(fnum=0.6, cplx=cplx)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32" if cplx else "f32", das_variant=variant))
    grf, _, gw = plan.das_backward(_to_dev(r), _to_dev(G), apod=_to_dev(w), c=1500.0)
    want_rf, _, want_w = oracle.das_grad(g, r, G, w=w, c=1500.0)
    e_rf = rel_l2(_from_dev(grf, cplx), want_rf)
    e_w = rel_l2(gw.cpu().numpy(), want_w)
    # speed-of-sound gradient: scatterer data, coherent loss
    g2, r2, w2 = _scatter_case(cplx)
    c = 1540.0
    plan2 = rc.Plan(rc.make_params(g2, decoded_dtype="cf32" if cplx else "f32", das_variant=variant))
    d2 = _to_dev(r2)
    img = plan2.das(d2, apod=_to_dev(w2), c=c)
    _, gc, _ = plan2.das_backward(d2, -2.0 * img, apod=_to_dev(w2), c=c, want_rf=False)
    im64 = oracle.das(g2, r2, w=w2, c=c)
    _, want_c, _ = oracle.das_grad(g2, r2, -2.0 * im64, w=w2, c=c, want_rf=False)
    e_c = abs(float(gc.item()) - want_c) / abs(want_c)
    print("grad v%d cplx=%s: rf %.2e  w %.2e  c %.2e" % (variant, cplx, e_rf, e_w, e_c))
    tol_c = 1e-3 if variant == rc.DAS_TILED else 1e-2     # the plain form's FP32 delays
    assert e_rf <= 1e-4 and e_w <= 1e-4 and e_c <= tol_c


def _coarse_z(cplx):
    # 10 um lateral, 150 um axial spacing: 32 z-rows of the adjoint's own tile
    # reach more than 128 samples, the plan's tile (long along x) does not
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=1024, out_dims=(128, 1, 64), f_number=0.0,
                       out_min=(-0.64 * MM, 0.0, 3 * MM), out_max=(0.63 * MM, 0.0, 12.45 * MM))
    rng = np.random.default_rng(91 + cplx)
    r = rng.normal(size=(16, 16, 1024)) + (1j * rng.normal(size=(16, 16, 1024)) if cplx else 0)
    G = rng.normal(size=(64, 1, 128)) + (1j * rng.normal(size=(64, 1, 128)) if cplx else 0)
    return g, r, G, rng.uniform(0.5, 1.5, 16)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("case", ["z_lanes", "u_lanes", "z_lanes_unaligned_grad_rf", "z_lanes_fnumber"])
def test_adjoint_lane_mappings_and_flush_forms(case, cplx):
    # the adjoint's two tiled lane mappings (lanes over z with its own tile;
    # lanes along u with the plan's tile) and both flush forms (four-float
    # reductions into a 16-byte aligned grad_rf, scalar atomics otherwise)
    if case == "u_lanes":
        g, r, G, w = _coarse_z(cplx)
    else:
        g, r, G, w = _small(fnum=0.7 if case == "z_lanes_fnumber" else 0.0, cplx=cplx)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32" if cplx else "f32"))
    info = plan.info()
    assert info["bwd_mode"] == (1 if case == "u_lanes" else 2), info
    if info["bwd_mode"] == 2:
        assert info["bwd_tile"][0] == 32 and info["bwd_tile"][1] * info["bwd_tile"][2] == 32
    dr = _to_dev(r)
    out = None
    if case == "z_lanes_unaligned_grad_rf":
        buf = torch.zeros(dr.numel() + 1, device="cuda")
        out = buf[1:].view(dr.shape)                 # 4-byte but not 16-byte aligned
        assert out.data_ptr() % 16 != 0
    grf, gc, gw = plan.das_backward(dr, _to_dev(G), apod=_to_dev(w), c=1500.0, out_rf=out)
    want_rf, want_c, want_w = oracle.das_grad(g, r, G, w=w, c=1500.0)
    e_rf = rel_l2(_from_dev(grf, cplx), want_rf)
    e_w = rel_l2(gw.cpu().numpy(), want_w)
    print("%s cplx=%s tile %s: rf %.2e  w %.2e" % (case, cplx, info["bwd_tile"], e_rf, e_w))
    assert e_rf <= 1e-4 and e_w <= 1e-4
    if out is not None:
        assert float(buf[0].item()) == 0.0           # nothing written before the view


def test_adjoint_fixed_point_range_extremes():
    # one 32 x 32 voxel block (one adjoint tile) carries gradients 1e6 times
    # larger than the rest. The fixed-point scale is set per tile, so trace
    # samples that only the other tiles reach keep their own relative accuracy.
    g, r, G, w = _small()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    assert plan.info()["bwd_tile"] == (32, 1, 32)
    big = np.zeros_like(G)
    big[:32, :, :32] = G[:32, :, :32] * 1e6
    G = G.copy()
    G[:32, :, :32] = big[:32, :, :32]
    grf, _, gw = plan.das_backward(_to_dev(r), _to_dev(G), apod=_to_dev(w))
    want_rf, _, want_w = oracle.das_grad(g, r, G, w=w)
    got = grf.cpu().numpy()
    assert rel_l2(got, want_rf) <= 1e-4
    assert rel_l2(gw.cpu().numpy(), want_w) <= 1e-4
    only_small = oracle.das_grad(g, r, big, w=w)[0] == 0.0
    assert only_small.mean() > 0.3
    e_small = rel_l2(got[only_small], want_rf[only_small])
    print("samples reached by the small tiles only: %.1f %%, rel-L2 %.2e" % (100 * only_small.mean(), e_small))
    assert e_small <= 1e-4
    # an all-zero gradient (scale from a zero bound)
    grf0, gc0, gw0 = plan.das_backward(_to_dev(r), _to_dev(np.zeros_like(G)), apod=_to_dev(w))
    assert float(grf0.abs().max().item()) == 0.0 and float(gc0.item()) == 0.0
    assert float(gw0.abs().max().item()) == 0.0


def test_grad_outputs_are_optional():
    g, r, G, w = _small()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    grf, gc, gw = plan.das_backward(_to_dev(r), _to_dev(G), apod=_to_dev(w), want_rf=False)
    assert grf is None and gc is not None and gw is not None
    _, _, want_w = oracle.das_grad(g, r, G, w=w, want_rf=False)
    assert rel_l2(gw.cpu().numpy(), want_w) <= 1e-4


def test_autograd_function():
    g, r, w = _scatter_case(False)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    dr = _to_dev(r).requires_grad_(True)
    dw = _to_dev(w).requires_grad_(True)
    c = torch.tensor(1520.0, device="cuda", requires_grad=True)
    img = rc.das_autograd(plan, dr, dw, c)
    rc.envelope_loss(img).backward()
    im64 = oracle.das(g, r, w=w, c=1520.0)
    want_rf, want_c, want_w = oracle.das_grad(g, r, -2.0 * im64, w=w, c=1520.0)
    assert rel_l2(dr.grad.cpu().numpy(), want_rf) <= 1e-4
    assert rel_l2(dw.grad.cpu().numpy(), want_w) <= 1e-4
    assert abs(float(c.grad.item()) - want_c) <= 1e-3 * abs(want_c)


def test_autofocus_speed_of_sound_gradient():
    # complex RF synthesised at c = 1480 m/s, beamformed at 1540 m/s; loss =
    # -sum |I|^2. The delay-and-sum with linear interpolation is piecewise
    # smooth in c: every term has a kink where its delay crosses a sample, so
    # a central difference over a step h measures the mean of dL/dc over
    # [c - h, c + h], not dL/dc at c. Checked here: (a) the adjoint against the
    # FP64 oracle's analytic gradient; (b) the prescribed central difference
    # (step 1e-3 c, GPU forward) against the mean of the adjoint over the same
    # interval (trapezoid rule, 201 points), which is the quantity it equals;
    # (c) the adjoint against an FP64 oracle central difference with a step
    # of 1e-6 c, small enough to resolve the point derivative.
    fr = frame("autofocus")
    g = fr.geometry
    r = fr.decoded.astype(np.complex128)
    c0 = 1540.0
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32"))
    dec = _to_dev(fr.decoded)

    def adjoint(c):
        img = plan.das(dec, c=c)
        _, gc, gw = plan.das_backward(dec, -2.0 * img, c=c, want_rf=False)
        return float(gc.item()), gw

    def loss_gpu(c):
        im = plan.das(dec, c=c).double()
        return -float((im * im).sum().item())

    def loss_oracle(c):
        return -float(np.sum(np.abs(oracle.das(g, r, c=c)) ** 2))

    gc, gw = adjoint(c0)
    im64 = oracle.das(g, r, c=c0)
    # the complex forward itself (full frame: a channel split with a tail of
    # channel parts in partial images of their own)
    im = plan.das(dec, c=c0).cpu().numpy().astype(np.float64)
    assert rel_l2(im[0] + 1j * im[1], im64) <= 1e-4
    _, gc64, gw64 = oracle.das_grad(g, r, -2.0 * im64, c=c0, want_rf=False)
    h = 1e-3 * c0
    fd = (loss_gpu(c0 + h) - loss_gpu(c0 - h)) / (2 * h)
    cs = np.linspace(c0 - h, c0 + h, 201)
    vals = np.array([adjoint(float(c))[0] for c in cs])
    mean_adj = float(np.sum(0.5 * (vals[1:] + vals[:-1]) * np.diff(cs)) / (2 * h))   # trapezoid rule
    hs = 1e-6 * c0
    fd_point = (loss_oracle(c0 + hs) - loss_oracle(c0 - hs)) / (2 * hs)
    print("autofocus dL/dc at %.0f m/s: adjoint %.6e, oracle analytic %.6e (rel %.2e), dw rel-L2 %.2e"
          % (c0, gc, gc64, abs(gc - gc64) / abs(gc64), rel_l2(gw.cpu().numpy(), gw64)))
    print("  central difference, step 1e-3 c: %.6e (rel to adjoint at c: %.2e); mean of the adjoint over "
          "the step: %.6e (rel %.2e)" % (fd, (fd - gc) / gc, mean_adj, (fd - mean_adj) / mean_adj))
    print("  oracle central difference, step 1e-6 c: %.6e (rel to adjoint %.2e)" % (fd_point, (fd_point - gc) / gc))
    assert abs(gc - gc64) <= 1e-3 * abs(gc64)
    assert rel_l2(gw.cpu().numpy(), gw64) <= 1e-3
    assert abs(fd - mean_adj) <= 1e-3 * abs(mean_adj)
    assert abs(fd_point - gc) <= 1e-3 * abs(gc)
