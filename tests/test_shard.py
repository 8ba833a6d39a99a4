"""Sharded top-k on the GPU: logical shards of one database, each with its
own bolt_topk, merged by bolt_topk_merge -- bit-identical to the unsharded
top-k and to the oracle, including shards smaller than k, uneven shards,
heavy ties across shard boundaries, and both metrics."""
import numpy as np
import pytest

import oracle
from paper_1706_10283_gb300 import bolt, shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bolt.lib()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("metric", [bolt.METRIC_L2, bolt.METRIC_DOT])
@pytest.mark.parametrize("n,M,k,nshard,ties", [(100_003, 16, 100, 3, False), (100_003, 16, 10, 8, True),
                                                (5_000, 8, 1, 2, False), (1_000, 32, 100, 4, False),
                                                (700, 16, 300, 3, True), (70_000, 64, 37, 5, False)])
def test_sharded_equals_unsharded(torch_cuda, metric, n, M, k, nshard, ties):
    torch = torch_cuda
    rng = np.random.default_rng(n + M + k + nshard + metric)
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    hi = 2 if ties else 256
    luts = rng.integers(0, hi, (4, M, 16)).astype(np.uint8)
    blocked = bolt.pack_codes(dev(torch, codes))
    L = dev(torch, luts)
    s1, i1 = bolt.topk(blocked, n, M, L, k, metric)
    s2, i2 = shard.sharded_topk(blocked, n, M, L, k, metric, nshard)
    np.testing.assert_array_equal(i2.cpu().numpy(), i1.cpu().numpy())
    np.testing.assert_array_equal(s2.view(torch.int16).cpu().numpy(), s1.view(torch.int16).cpu().numpy())
    rs, ri = oracle.topk(oracle.scan(codes, luts), k, metric)
    np.testing.assert_array_equal(i2.cpu().numpy(), ri)
    np.testing.assert_array_equal(s2.cpu().numpy(), rs)


def test_merge_pads_and_propagates_failure(torch_cuda):
    """Union smaller than k: padding as bolt_topk (sum 0, index -1); a shard
    row marked -2 (failed wait) marks the merged row -2."""
    torch = torch_cuda
    k, M = 8, 4
    sums = np.zeros((2, 2, k), np.uint16)
    idx = np.full((2, 2, k), -1, np.int64)
    sums[0, 0, :2], idx[0, 0, :2] = [3, 5], [0, 1]
    sums[1, 0, :1], idx[1, 0, :1] = [4], [0]
    idx[1, 1, :] = -2
    offs = dev(torch, np.array([0, 100], np.int64))
    s, i = bolt.topk_merge(dev(torch, sums.view(np.int16)).view(torch.uint16), dev(torch, idx), offs, M,
                           bolt.METRIC_L2)
    np.testing.assert_array_equal(i.cpu().numpy()[0], [0, 100, 1, -1, -1, -1, -1, -1])
    np.testing.assert_array_equal(s.cpu().numpy()[0], [3, 4, 5, 0, 0, 0, 0, 0])
    assert np.all(i.cpu().numpy()[1] == -2)
