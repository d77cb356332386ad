"""The upload ring (rcbf_pipeline_*) on the GPU: several steps through three
slots with distinct inputs per step, pinned and pageable host memory, every
step's images equal to the single-frame entry points on the same data, and
the argument checks."""
import numpy as np
import pytest

import synth
from synth import MM
from tests._frames import rel_l2

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


def _frames():
    g1 = synth.tiny_bscan_geometry()
    g2 = synth.Geometry(n_tx=64, n_ch=64, n_samples=2048, hadamard_order=64, out_dims=(256, 1, 256),
                        out_min=(-3.2 * MM, 0.0, 4 * MM), out_max=(3.2 * MM, 0.0, 20 * MM))
    return [synth.make_frame(g1, 31, 5), synth.make_frame(g2, 32, 5)]


@pytest.mark.parametrize("pinned", [True, False])
def test_pipeline_steps_match_single_frames(pinned):
    frames = _frames()
    # different tile extents: the batch of every slot runs two phases (the
    # second a programmatic dependent), captured in the slot's graph
    plans = [rc.Plan(rc.make_params(f.geometry, decoded_dtype="f16", tile=t))
             for f, t in zip(frames, [(64, 1, 16), (32, 1, 32)])]
    pipe = rc.Pipeline(plans, n_slots=3)
    steps = 7                               # every slot is reused at least twice
    inputs, images = [], []
    for s in range(steps):
        scale = (-1) ** s                   # distinct inputs per step (exact in int16)
        ins = [torch.from_numpy(np.ascontiguousarray(scale * f.rf)) for f in frames]
        outs = [torch.empty(p.image_shape, dtype=torch.float32) for p in plans]
        if pinned:
            ins = [t.pin_memory() for t in ins]
            outs = [t.pin_memory() for t in outs]
        pipe.submit(ins, outs)
        inputs.append(ins)
        images.append(outs)
    pipe.wait()
    for s in range(steps):
        for f, p in enumerate(plans):
            want = p.das(p.decode(inputs[s][f].cuda())).cpu().numpy()
            err = rel_l2(images[s][f].numpy(), want)
            assert err <= 1e-5, (s, f, err)
    pipe.close()


def test_pipeline_argument_checks():
    frames = _frames()
    plans = [rc.Plan(rc.make_params(f.geometry, decoded_dtype="f16", tile=(64, 1, 16))) for f in frames]
    for n_slots in (1, 9):
        with pytest.raises(rc.RcbfError) as e:
            rc.Pipeline(plans, n_slots=n_slots)
        assert e.value.code == rc.EINVAL
    cub = rc.Plan(rc.make_params(frames[0].geometry, decoded_dtype="f16", tile=(64, 1, 16), interp="cubic"))
    with pytest.raises(rc.RcbfError) as e:
        rc.Pipeline([cub], n_slots=2)
    assert e.value.code == rc.EUNSUPPORTED
