"""The tcgen05 decode (RCBF_DECODE_TC: tensor-memory accumulators, TMA tensor
loads and stores) against the oracle's exact integer decode, bit for bit, for
every output type: full-range random int16 (the sign of the high byte and the
largest sums), ragged column counts, the extreme values, the Hadamard round
trip, a non-Sylvester +-1 matrix, and the three acquisition workloads (many
64-column tiles per CTA, so the 4-stage ring and both accumulator sets wrap
around many times)."""
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


def _run(g, rf, dtype, matrix=None):
    plan = rc.Plan(rc.make_params(g, decoded_dtype=dtype, decode_variant=rc.DECODE_TC), decode_matrix=matrix)
    out = plan.decode(torch.from_numpy(np.ascontiguousarray(rf)).cuda())
    torch.cuda.synchronize()
    assert plan.status() == rc.OK
    return out.cpu().numpy()


def _assert_bit_exact(got, D, n, dtype):
    want = oracle.decoded_as(D, n, dtype)
    if dtype == "f16":
        np.testing.assert_array_equal(got.view(np.uint16), want.view(np.uint16))
    else:
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("dtype", ["i32", "f32", "f16"])
@pytest.mark.parametrize("n,n_ch,n_s", [(32, 32, 1024), (64, 5, 136), (128, 3, 1000), (128, 1, 24),
                                        (32, 1, 8), (128, 41, 2048)])
def test_tc_decode_random_full_int16_range(dtype, n, n_ch, n_s):
    rf = synth.random_int_rf(n, n_ch, n_s, seed=3 * n + n_ch + n_s)
    _assert_bit_exact(_run(_geom(n, n_ch, n_s), rf, dtype), oracle.decode(rf), n, dtype)


@pytest.mark.parametrize("dtype", ["i32", "f32", "f16"])
def test_tc_decode_extreme_values(dtype):
    # every acquisition at -32768 or +32767: the largest |D| = n * 32768
    n = 128
    rf = np.full((n, 2, 64), -32768, dtype=np.int16)
    rf[::2, 0, :] = 32767
    _assert_bit_exact(_run(_geom(n, 2, 64), rf, dtype), oracle.decode(rf), n, dtype)


@pytest.mark.parametrize("n", [32, 64, 128])
def test_tc_decode_round_trip(n):
    rng = np.random.default_rng(200 + n)
    lim = 32767 // n
    r = rng.integers(-lim, lim + 1, size=(n, 4, 256)).astype(np.int64)
    s = np.einsum("ki,ics->kcs", synth.sylvester_kron(n), r).astype(np.int16)
    np.testing.assert_array_equal(_run(_geom(n, 4, 256), s, "i32"), (n * r).astype(np.int32))


def test_tc_decode_custom_matrix():
    n = 64
    rng = np.random.default_rng(17)
    H = (synth.sylvester_kron(n)[rng.permutation(n)] * rng.choice([-1, 1], n)[None, :]).astype(np.int8)
    rf = synth.random_int_rf(n, 3, 128, seed=18)
    np.testing.assert_array_equal(_run(_geom(n, 3, 128), rf, "i32", matrix=H), oracle.decode(rf, H).astype(np.int32))


@pytest.mark.parametrize("name", ["tiny", "bscan", "volume"])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_tc_decode_workloads(name, dtype):
    fr = frame(name)
    g = fr.geometry
    _assert_bit_exact(_run(g, fr.rf, dtype), oracle.decode(fr.rf), g.n_tx, dtype)


def test_tc_decode_rejects_order_256():
    with pytest.raises(rc.RcbfError) as e:
        rc.Plan(rc.make_params(_geom(256, 2, 64), decoded_dtype="f32", decode_variant=rc.DECODE_TC))
    assert e.value.code == rc.EUNSUPPORTED
