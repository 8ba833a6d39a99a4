"""The library's basic usage sequence from Python -- fit codebooks and the
quantizer on the GPU, encode, build L2 tables, fused top-k, dequantize -- on a
200,000-vector mixture, with the codes and the top-k checked against the
oracle on the same codebooks and tables."""
import numpy as np
import pytest

import oracle
from paper_1706_10283_gb300 import bolt, synth

pytestmark = pytest.mark.gpu


def test_readme_example():
    import torch

    assert torch.cuda.is_available()
    n, J, M = 200_000, 128, 16
    X = synth.mixture_torch(n, J, seed=0)
    Q = torch.from_numpy(synth.mixture(16, J, 1)).cuda()
    C = bolt.fit_codebooks(X[:100_000].contiguous(), M, 8, synth.kmeans_init_rows(100_000, 0))
    a, b, _ = bolt.fit_quantizer(X[:256].contiguous(), C, bolt.METRIC_L2)
    codes = bolt.encode(X, C)
    luts = bolt.build_luts(Q, C, bolt.METRIC_L2, a, b)
    sums, idx = bolt.topk(codes, X.shape[0], M, luts, 100, bolt.METRIC_L2)
    dist = bolt.dequantize(sums, a, b)
    assert sums.shape == (16, 100) and idx.shape == (16, 100) and dist.shape == (16, 100)
    oc = bolt.unpack_codes(codes, n, M).cpu().numpy()
    np.testing.assert_array_equal(oc, oracle.encode(X.cpu().numpy(), C.cpu().numpy()))
    rs, ri = oracle.topk(oracle.scan(oc, luts.cpu().numpy()), 100, oracle.METRIC_L2)
    np.testing.assert_array_equal(idx.cpu().numpy(), ri)
    np.testing.assert_array_equal(sums.cpu().numpy(), rs)
    assert (np.diff(dist.cpu().numpy(), axis=1) >= 0).all()
