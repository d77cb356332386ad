"""The geometry affines on the GPU: the world -> array transform (the paper's
corner-element origin, §METHODS "Data Processing") and the voxel-index ->
world transform (Fig. "das_dispatch"), tiled and plain DAS forms against the
FP64 oracle at relative L2 1e-4. The oracle's reading of both matrices is
pinned by hand-computed delays in tests/test_oracle_pins.py."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth
from synth import MM
from tests._frames import frame, rel_l2

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
    return oracle.decode(fr.rf).astype(np.float64) / fr.geometry.n_tx


def _gpu(g, r, variant, xdc=None, vox=None):
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32", das_variant=variant,
                                  xdc_transform=None if xdc is None else np.asarray(xdc).tolist(),
                                  voxel_transform=None if vox is None else np.asarray(vox).tolist()))
    img = plan.das(torch.from_numpy(r.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64), plan.info()


def _corner(g):
    # world origin at the centre of element 0 of both families: world ->
    # centred array frame is a translation by minus the corner's offset
    X = np.eye(4)
    X[0, 3] = -(g.n_ch - 1) / 2 * g.rx_pitch      # columns: lateral x
    X[1, 3] = -(g.n_tx - 1) / 2 * g.tx_pitch      # rows: lateral y
    return X


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
def test_corner_element_origin(variant):
    # the tiny acquisition imaged on a grid given in the corner-element frame:
    # the same world points as the centred grid, so the oracle image in both
    # frames agrees to rounding, and the GPU follows the oracle in each
    fr = frame("tiny")
    g = fr.geometry
    r = _exact(fr)
    X = _corner(g)
    gw = dataclasses.replace(g, out_min=tuple(np.add(g.out_min, [-X[0, 3], -X[1, 3], 0.0])),
                             out_max=tuple(np.add(g.out_max, [-X[0, 3], -X[1, 3], 0.0])))
    want = oracle.das(gw, r, xdc_transform=X)
    np.testing.assert_allclose(want, oracle.das(g, r), rtol=0, atol=1e-9 * np.abs(want).max())
    got, info = _gpu(gw, r, variant, xdc=X)
    assert info["tiled"] == (variant == rc.DAS_TILED)
    err = rel_l2(got, want)
    print("corner origin v%d: rel-L2 %.3e" % (variant, err))
    assert err <= TOL


def _swapped_volume():
    # index axis 0 -> world y, index axis 1 -> world x, axis 2 -> z: a volume
    # whose lane axis (transmit lateral and z constant) is index axis 1
    g = synth.Geometry(n_tx=32, n_ch=32, n_samples=1024, out_dims=(16, 64, 96),
                       out_min=(0.0, 0.0, 0.0), out_max=(0.0, 0.0, 0.0))
    M = np.zeros((4, 4))
    M[1, 0], M[1, 3] = 1.0 * MM / 15, -0.5 * MM          # 16 points over y in [-0.5, 0.5] mm
    M[0, 1], M[0, 3] = 3.0 * MM / 63, -1.5 * MM          # 64 points over x in [-1.5, 1.5] mm
    M[2, 2], M[2, 3] = 4.0 * MM / 95, 5.0 * MM           # 96 points over z in [5, 9] mm
    M[3, 3] = 1.0
    r = np.random.default_rng(41).normal(size=(32, 32, 1024))
    return g, M, r


@pytest.mark.parametrize("variant", [rc.DAS_TILED, rc.DAS_PLAIN])
def test_axis_permuting_voxel_affine(variant):
    g, M, r = _swapped_volume()
    want = oracle.das(g, r, voxel_transform=M)
    got, info = _gpu(g, r, variant, vox=M)
    assert info["tiled"] == (variant == rc.DAS_TILED)
    err = rel_l2(got, want)
    print("permuted voxel affine v%d: rel-L2 %.3e tile %s" % (variant, err, info["tile"]))
    assert err <= TOL
    # the transposed matrix puts the voxels elsewhere: a large difference
    assert rel_l2(oracle.das(g, r, voxel_transform=M.T), want) > 0.1


def test_rotated_array_runs_plain_form():
    # the array turned by 30 degrees about z: the transmit lateral coordinate
    # changes along both image axes, so no lane axis exists: the tiled form
    # is refused (RCBF_EUNSUPPORTED) and the plain form holds the bound
    g = synth.Geometry(n_tx=16, n_ch=16, n_samples=768, out_dims=(24, 20, 48),
                       out_min=(-1 * MM, -1 * MM, 4 * MM), out_max=(1 * MM, 1 * MM, 8 * MM), f_number=0.7)
    a = math.radians(30.0)
    X = np.eye(4)
    X[0, 0], X[0, 1], X[1, 0], X[1, 1] = math.cos(a), math.sin(a), -math.sin(a), math.cos(a)
    X[0, 3], X[1, 3] = 0.1 * MM, -0.2 * MM
    r = np.random.default_rng(43).normal(size=(16, 16, 768))
    want = oracle.das(g, r, xdc_transform=X)
    with pytest.raises(rc.RcbfError) as e:
        _gpu(g, r, rc.DAS_TILED, xdc=X)
    assert e.value.code == rc.EUNSUPPORTED
    got, info = _gpu(g, r, rc.DAS_PLAIN, xdc=X)
    assert not info["tiled"]
    err = rel_l2(got, want)
    print("rotated array (plain form): rel-L2 %.3e" % err)
    assert err <= TOL
