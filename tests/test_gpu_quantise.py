"""The fixed-point conversion of the seeding step on the GPU against the oracle's
(the bit-exactness contract of A1: the paper seeds in native pad and time
coordinates, Sec. 1; the reading is pad_q = rint(64 pad), t_q = rint(64 time),
ties to even).

Every float bit pattern with 2^-8 <= |v| <= 131072 goes through the device
conversion (tpc_debug_quantize, the same function the neighbour kernels use) and
through the oracle's or_quantize, and the two must agree bit for bit; below 2^-8
(where 64 v rounds to zero) a dense stride of patterns, signed zeros and
subnormals.  131072 bins is the top of the validated time range, 1024 pads that of
the pad range.  A planted round-half-up conversion must disagree on the exact
halves, so the sweep would notice that mistake."""
import numpy as np
import pytest

import oracle as orc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tpcca():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_08862_gb300 import _build, tpcca
    _build.build()
    return tpcca


def _gpu_q(tpcca, v_host):
    dev = torch.device("cuda", 0)
    v = torch.from_numpy(v_host).to(dev)
    q = torch.empty(v.numel(), dtype=torch.int32, device=dev)
    assert tpcca.tpc_debug_quantize(v.data_ptr(), v.numel(), q.data_ptr(), 0) == tpcca.TPC_OK, tpcca.tpc_last_error()
    return q.cpu().numpy()


def _oracle_q(v):
    rows = np.zeros(v.shape[0], np.uint16)
    pq, tq, _, _ = orc.quantize(rows, v, v)
    assert np.array_equal(pq, tq)
    return pq


LO, HI = np.float32(2.0 ** -8).view(np.uint32), np.float32(131072.0).view(np.uint32)
CHUNK = 1 << 25


def test_every_pattern_in_the_validated_range(tpcca):
    total = 0
    for sign in (0, 0x80000000):
        for a in range(int(LO), int(HI) + 1, CHUNK):
            bits = np.arange(a, min(a + CHUNK, int(HI) + 1), dtype=np.uint32) | np.uint32(sign)
            v = bits.view(np.float32)
            g, o = _gpu_q(tpcca, v), _oracle_q(v)
            bad = np.nonzero(g != o)[0]
            assert bad.size == 0, (v[bad[:5]], g[bad[:5]], o[bad[:5]])
            total += v.size
    assert total == 2 * (int(HI) - int(LO) + 1)


def test_small_values_zeros_and_subnormals(tpcca):
    bits = np.concatenate([np.arange(0, int(LO), 4099, dtype=np.uint32), np.arange(0, 64, dtype=np.uint32)])
    bits = np.concatenate([bits, bits | np.uint32(0x80000000)])
    v = bits.view(np.float32)
    g, o = _gpu_q(tpcca, v), _oracle_q(v)
    assert np.array_equal(g, o)
    assert np.all(g == 0)


def test_round_half_up_would_be_noticed(tpcca):
    # exact halves 64 v = k + 1/2 for k in [-2^22, 2^22)
    k = np.arange(-(1 << 22), 1 << 22, dtype=np.int64)
    v = ((2 * k + 1).astype(np.float64) / 128.0).astype(np.float32)
    assert np.all((v.astype(np.float64) * 64.0) == k + 0.5)   # exact
    g = _gpu_q(tpcca, v)
    assert np.array_equal(g, _oracle_q(v))
    even = np.where(k % 2 == 0, k, k + 1)                        # ties to even
    assert np.array_equal(g, even)
    half_up = np.floor(v.astype(np.float64) * 64.0 + 0.5).astype(np.int64)
    assert np.count_nonzero(half_up != g) == k.size // 2         # the planted mistake differs on half of them
