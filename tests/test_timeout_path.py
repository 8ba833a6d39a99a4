"""The failure path of the bounded device waits, run on the GPU without any
fault: with the data-wait limit set to 1 ns (bolt_set_wait_limit_ns), the
streaming top-k kernel's waits for its code copies give up, the kernel drains
its copies in flight and marks the query (every index -2, which check_topk
turns into BOLT_ETIMEOUT), and the tensor-core encoder reports
n_rechecked = -1.  With the default limit restored, the same calls on the
same context return correct results."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1706_10283_gb300 import bolt, synth

pytestmark = pytest.mark.gpu


@pytest.fixture()
def tiny_wait_limit():
    L = bolt.lib()
    assert L.bolt_set_wait_limit_ns(C.c_uint64(1)) == bolt.OK
    try:
        yield L
    finally:
        assert L.bolt_set_wait_limit_ns(C.c_uint64(0)) == bolt.OK


def test_streaming_topk_times_out_cleanly(tiny_wait_limit):
    import torch

    assert torch.cuda.is_available()
    rng = np.random.default_rng(3)
    n, M, k = 6_000_000, 16, 100  # one query, 155 blocks per CTA: beyond the shared-memory class
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, 256, (1, M, 16)).astype(np.uint8)
    blocked = bolt.pack_codes(torch.from_numpy(codes).cuda())
    L = torch.from_numpy(luts).cuda()
    s, i = bolt.topk(blocked, n, M, L, k, bolt.METRIC_L2)
    torch.cuda.synchronize()
    assert (i.cpu().numpy() == -2).all()
    with pytest.raises(bolt.BoltError) as e:
        bolt.check_topk(i)
    assert e.value.code == bolt.ETIMEOUT
    # the default limit back: the same call is correct on the same context
    tiny_wait_limit.bolt_set_wait_limit_ns(C.c_uint64(0))
    s, i = bolt.topk(blocked, n, M, L, k, bolt.METRIC_L2, check=True)
    rs, ri = oracle.topk(oracle.scan(codes, luts), k, oracle.METRIC_L2)
    np.testing.assert_array_equal(i.cpu().numpy(), ri)
    np.testing.assert_array_equal(s.cpu().numpy(), rs)


def test_tensor_core_encoder_times_out_cleanly(tiny_wait_limit):
    import torch

    assert torch.cuda.is_available()
    n, J, M = 200_000, 256, 32
    X = synth.mixture(n, J, 9)
    C_ = oracle.kmeans(X[:4000], M, 3, synth.kmeans_init_rows(4000, 9))
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C_).cuda()
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    bolt.encode(Xd, Cd, bolt.PREC_BF16_RECHECK, n_rechecked=cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == -1
    tiny_wait_limit.bolt_set_wait_limit_ns(C.c_uint64(0))
    cnt.zero_()
    codes = bolt.encode(Xd, Cd, bolt.PREC_BF16_RECHECK, n_rechecked=cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) >= 0
    np.testing.assert_array_equal(bolt.unpack_codes(codes, n, M).cpu().numpy(), oracle.encode(X, C_))
