"""Failure detection of the tiled DAS on the GPU without a fault: the bounded
waits of rcbf_das report their expiry through the plan's status word.
rcbf_plan_set_wait's test hook withholds the first window copy of every voxel
tile, so each tile's first wait runs out after the (short) bound; the kernel
stops those tiles and returns, rcbf_plan_status reads RCBF_ETIMEOUT, and the
next call, with the hook off, succeeds on the same plan and context."""
import numpy as np
import pytest

import oracle
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


def _tiny():
    fr = frame("tiny")
    g = fr.geometry
    r = oracle.decode(fr.rf).astype(np.float64) / g.n_tx
    return g, r, torch.from_numpy(r.astype(np.float32)).cuda()


def test_forward_das_wait_expires_and_the_next_call_succeeds():
    g, r, dec = _tiny()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    assert plan.info()["tiled"]
    want = plan.das(dec).cpu().numpy()
    assert plan.status() == rc.OK
    plan.set_wait(2_000_000, withhold=1)          # 2 ms bound; every tile's first copy withheld
    plan.das(dec)
    assert plan.status() == rc.ETIMEOUT
    plan.set_wait(1_000_000_000, withhold=0)
    got = plan.das(dec).cpu().numpy()
    assert plan.status() == rc.OK                 # the next call clears the word
    np.testing.assert_array_equal(got, want)
    assert rel_l2(got, oracle.das(g, r)) <= 1e-4


def test_adjoint_clears_and_reports_its_status():
    g, r, dec = _tiny()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    plan.set_wait(2_000_000, withhold=1)
    plan.das(dec)
    assert plan.status() == rc.ETIMEOUT
    plan.set_wait(1_000_000_000, withhold=0)
    G = torch.ones(plan.image_shape, device="cuda")
    plan.das_backward(dec, G)
    assert plan.status() == rc.OK                 # the adjoint's own waits all completed


def test_set_wait_validates():
    g, _, _ = _tiny()
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    with pytest.raises(rc.RcbfError):
        plan.set_wait(0)
    with pytest.raises(rc.RcbfError):
        plan.set_wait(1000, withhold=2)
