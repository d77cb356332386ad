"""Decode parity on the GPU: the library's decode (through the C ABI) must
equal the oracle's exact integer decode bit for bit, for every output type and
both the tensor-core and the plain form."""
import numpy as np
import pytest

import oracle
import synth
from tests._frames import frame

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


def _geom(n, n_ch, n_s):
    return synth.Geometry(n_tx=n, n_ch=n_ch, n_samples=n_s, hadamard_order=n)


def _run(g, rf, dtype, variant, matrix=None):
    plan = rc.Plan(rc.make_params(g, decoded_dtype=dtype, decode_variant=variant), decode_matrix=matrix)
    out = plan.decode(torch.from_numpy(rf).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _assert_bit_exact(got, D, n, dtype):
    want = oracle.decoded_as(D, n, dtype)
    if dtype == "f16":
        np.testing.assert_array_equal(got.view(np.uint16), want.view(np.uint16))
    else:
        np.testing.assert_array_equal(got, want)


VARIANTS = [rc.DECODE_MMA_I8, rc.DECODE_MMA_F16, rc.DECODE_PLAIN]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dtype", ["i32", "f32", "f16"])
@pytest.mark.parametrize("n,n_ch,n_s", [(32, 32, 1024), (64, 5, 136), (128, 3, 1000), (256, 3, 520),
                                        (32, 1, 8), (128, 1, 24)])
def test_decode_random_full_int16_range(variant, dtype, n, n_ch, n_s):
    # full-range random int16 exercises the sign of the high byte and the
    # largest sums; n_ch * n_s spans several 128-column tiles and a ragged tail
    rf = synth.random_int_rf(n, n_ch, n_s, seed=n + n_ch + n_s)
    g = _geom(n, n_ch, n_s)
    _assert_bit_exact(_run(g, rf, dtype, variant), oracle.decode(rf), n, dtype)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dtype", ["i32", "f32", "f16"])
def test_decode_extreme_values(variant, dtype):
    # every acquisition at -32768 or +32767: the largest |D| = n * 32768
    n = 256
    rf = np.full((n, 2, 64), -32768, dtype=np.int16)
    rf[::2, 0, :] = 32767
    g = _geom(n, 2, 64)
    _assert_bit_exact(_run(g, rf, dtype, variant), oracle.decode(rf), n, dtype)


@pytest.mark.parametrize("variant", [rc.DECODE_MMA_I8, rc.DECODE_MMA_F16])
@pytest.mark.parametrize("name", ["tiny", "bscan", "volume"])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_decode_workloads(variant, name, dtype):
    fr = frame(name)
    g = fr.geometry
    _assert_bit_exact(_run(g, fr.rf, dtype, variant), oracle.decode(fr.rf), g.n_tx, dtype)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", [32, 64, 128, 256])
def test_decode_round_trip(variant, n):
    rng = np.random.default_rng(100 + n)
    lim = 32767 // n
    r = rng.integers(-lim, lim + 1, size=(n, 4, 256)).astype(np.int64)
    s = np.einsum("ki,ics->kcs", synth.sylvester_kron(n), r).astype(np.int16)
    got = _run(_geom(n, 4, 256), s, "i32", variant)
    np.testing.assert_array_equal(got, (n * r).astype(np.int32))


def test_decode_custom_matrix():
    n = 64
    rng = np.random.default_rng(7)
    H = (synth.sylvester_kron(n)[rng.permutation(n)] * rng.choice([-1, 1], n)[None, :]).astype(np.int8)
    rf = synth.random_int_rf(n, 3, 128, seed=8)
    for variant in VARIANTS:
        plan = rc.Plan(rc.make_params(_geom(n, 3, 128), decoded_dtype="i32", decode_variant=variant),
                       decode_matrix=H)
        got = plan.decode(torch.from_numpy(rf).cuda()).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.decode(rf, H).astype(np.int32))


def test_decode_rejects_misaligned():
    g = _geom(32, 1, 64)
    plan = rc.Plan(rc.make_params(g, decoded_dtype="f32"))
    buf = torch.zeros(32 * 64 + 8, dtype=torch.int16, device="cuda")
    with pytest.raises(rc.RcbfError) as e:
        plan.decode(buf[1:1 + 32 * 64])
    assert e.value.code == rc.EINVAL
