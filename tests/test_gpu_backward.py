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


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
@pytest.mark.parametrize("cplx", [False, True])
def test_gradients_match_oracle(variant, cplx):
    g, r, G, w = _small(fnum=0.6, cplx=cplx)
    c = 1500.0
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32" if cplx else "f32", das_variant=variant))
    grf, gc, gw = plan.das_backward(_to_dev(r), _to_dev(G), apod=_to_dev(w), c=c)
    want_rf, want_c, want_w = oracle.das_grad(g, r, G, w=w, c=c)
    e_rf = rel_l2(_from_dev(grf, cplx), want_rf)
    e_c = abs(float(gc.item()) - want_c) / abs(want_c)
    e_w = rel_l2(gw.cpu().numpy(), want_w)
    print("grad v%d cplx=%s: rf %.2e  c %.2e  w %.2e" % (variant, cplx, e_rf, e_c, e_w))
    assert e_rf <= 1e-4 and e_c <= 1e-3 and e_w <= 1e-4


def test_grad_outputs_are_optional():
    g, r, G, w = _small()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    grf, gc, gw = plan.das_backward(_to_dev(r), _to_dev(G), apod=_to_dev(w), want_rf=False)
    assert grf is None and gc is not None and gw is not None
    _, want_c, want_w = oracle.das_grad(g, r, G, w=w, want_rf=False)
    assert abs(float(gc.item()) - want_c) <= 1e-3 * abs(want_c)


def test_autograd_function():
    g, r, G, w = _small(fnum=0.5)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    dr = _to_dev(r).requires_grad_(True)
    dw = _to_dev(w).requires_grad_(True)
    c = torch.tensor(1520.0, device="cuda", requires_grad=True)
    img = rc.das_autograd(plan, dr, dw, c)
    (img * _to_dev(G)).sum().backward()
    want_rf, want_c, want_w = oracle.das_grad(g, r, G, w=w, c=1520.0)
    assert rel_l2(dr.grad.cpu().numpy(), want_rf) <= 1e-4
    assert rel_l2(dw.grad.cpu().numpy(), want_w) <= 1e-4
    assert abs(float(c.grad.item()) - want_c) <= 1e-3 * abs(want_c)


def test_autofocus_speed_of_sound_gradient():
    # complex RF synthesised at c = 1480 m/s, beamformed at 1540 m/s; loss =
    # -sum |I|^2. The analytic dL/dc (adjoint kernel) against central finite
    # differences with a 1e-3 relative step, on the GPU forward and on the
    # FP64 oracle forward, and against the oracle's analytic gradient.
    fr = frame("autofocus")
    g = fr.geometry
    r = fr.decoded.astype(np.complex128)
    c0 = 1540.0
    plan = rc.Plan(rc.make_params(g, decoded_dtype="cf32"))
    dec = _to_dev(fr.decoded)
    img = plan.das(dec, c=c0)
    G = -2.0 * img                                   # dL/dI for L = -sum |I|^2, both planes
    _, gc, gw = plan.das_backward(dec, G, c=c0, want_rf=False)
    gc = float(gc.item())

    def loss_gpu(c):
        im = plan.das(dec, c=c).double()
        return -float((im * im).sum().item())

    h = 1e-3 * c0
    fd_gpu = (loss_gpu(c0 + h) - loss_gpu(c0 - h)) / (2 * h)

    def loss_oracle(c):
        im = oracle.das(g, r, c=c)
        return -float(np.sum(np.abs(im) ** 2))

    fd_oracle = (loss_oracle(c0 + h) - loss_oracle(c0 - h)) / (2 * h)
    im64 = oracle.das(g, r, c=c0)
    _, gc64, gw64 = oracle.das_grad(g, r, -2.0 * im64, c=c0, want_rf=False)
    print("autofocus dL/dc: adjoint %.6e  FD(gpu) %.6e  FD(oracle) %.6e  oracle analytic %.6e"
          % (gc, fd_gpu, fd_oracle, gc64))
    print("  rel: vs FD(gpu) %.2e  vs FD(oracle) %.2e  vs oracle analytic %.2e  dw rel-L2 %.2e"
          % (abs(gc - fd_gpu) / abs(fd_gpu), abs(gc - fd_oracle) / abs(fd_oracle),
             abs(gc - gc64) / abs(gc64), rel_l2(gw.cpu().numpy(), gw64)))
    assert abs(gc - gc64) <= 1e-3 * abs(gc64)
    assert rel_l2(gw.cpu().numpy(), gw64) <= 1e-3
    assert abs(gc - fd_oracle) <= 1e-3 * abs(fd_oracle)
