"""The usage example of the README, run as written: decode and DAS of the
full-size B-scan, then one autofocus gradient through the adjoint kernel."""
import numpy as np
import pytest

import synth

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


def test_readme_usage_example():
    g = synth.full_bscan_geometry()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f16"))
    rf = torch.from_numpy(synth.full_bscan(2).rf).cuda()
    image = plan.das(plan.decode(rf))
    assert tuple(image.shape) == (g.out_dims[2], g.out_dims[1], g.out_dims[0])
    assert torch.isfinite(image).all() and image.abs().max() > 0

    dec = plan.decode(rf).float().requires_grad_()
    w = torch.ones(g.n_ch, device="cuda", requires_grad=True)
    c = torch.tensor(1540.0, device="cuda", requires_grad=True)
    p32 = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    rc.envelope_loss(rc.das_autograd(p32, dec, w, c)).backward()
    assert dec.grad is not None and tuple(dec.grad.shape) == tuple(dec.shape)
    assert torch.isfinite(dec.grad).all() and dec.grad.abs().max() > 0
    assert np.isfinite(w.grad.cpu().numpy()).all() and np.isfinite(float(c.grad))
