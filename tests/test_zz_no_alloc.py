"""bolt_topk_noalloc: the allocation-free top-k entry point (for callers that
cannot allocate device memory during a call, such as code running under a
strict CUDA-graph capture or allocator-free serving loops).

Called directly through the C ABI and compared with bolt_topk, the entry point
that takes caller-provided scratch, on two calls in a row (the fixed scratch
array is shared and reused between calls).  The file is named to be collected
last; it also passes when run alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1706_10283_gb300 import bolt

pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_topk_noalloc_matches_topk_twice():
    import torch

    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    L = bolt.lib()
    rng = np.random.default_rng(123)
    n, M, k, nq = 150_001, 16, 100, 2
    codes = bolt.pack_codes(torch.from_numpy(rng.integers(0, 16, (n, M)).astype(np.uint8)).cuda())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, metric in enumerate((bolt.METRIC_L2, bolt.METRIC_DOT)):
        luts = torch.from_numpy(rng.integers(0, 256, (nq, M, 16)).astype(np.uint8)).cuda()
        ref_s, ref_i = bolt.topk(codes, n, M, luts, k, metric)
        out_s = torch.full((nq, k), 7, dtype=torch.uint16, device="cuda")
        out_i = torch.full((nq, k), -9, dtype=torch.int64, device="cuda")
        rc = L.bolt_topk_noalloc(_p(codes), n, M, _p(luts), nq, k, metric, _p(out_s), _p(out_i), stream)
        assert rc == bolt.OK, L.bolt_last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out_i.cpu().numpy(), ref_i.cpu().numpy(), err_msg="call %d" % call)
        np.testing.assert_array_equal(out_s.cpu().numpy(), ref_s.cpu().numpy(), err_msg="call %d" % call)


def test_topk_noalloc_multi_query_layout():
    """Five queries over 4,000,003 vectors take the multi-query plan (sample
    bound, filter, select, streaming fallback), whose scratch is split into
    several regions inside the fixed array; compared with bolt_topk on two
    calls in a row."""
    import torch

    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    L = bolt.lib()
    rng = np.random.default_rng(321)
    n, M, k, nq = 4_000_003, 16, 10, 5
    assert bolt.topk_workspace_bytes(n, M, nq, k) <= 4 << 20
    codes = bolt.pack_codes(torch.from_numpy(rng.integers(0, 16, (n, M)).astype(np.uint8)).cuda())
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, metric in enumerate((bolt.METRIC_DOT, bolt.METRIC_L2)):
        luts = torch.from_numpy(rng.integers(0, 256, (nq, M, 16)).astype(np.uint8)).cuda()
        ref_s, ref_i = bolt.topk(codes, n, M, luts, k, metric)
        out_s = torch.full((nq, k), 7, dtype=torch.uint16, device="cuda")
        out_i = torch.full((nq, k), -9, dtype=torch.int64, device="cuda")
        rc = L.bolt_topk_noalloc(_p(codes), n, M, _p(luts), nq, k, metric, _p(out_s), _p(out_i), stream)
        assert rc == bolt.OK, L.bolt_last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out_i.cpu().numpy(), ref_i.cpu().numpy(), err_msg="call %d" % call)
        np.testing.assert_array_equal(out_s.cpu().numpy(), ref_s.cpu().numpy(), err_msg="call %d" % call)


def test_topk_noalloc_rejects_oversized_request():
    """Too many queries for the fixed array: BOLT_ENOMEM before any launch.
    Every buffer is sized for the request it describes (a small database,
    tables and outputs for all 1,024 queries), so even a call that wrongly
    launched would stay inside its buffers."""
    import torch

    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    L = bolt.lib()
    n, M, k, nq = 5_000, 16, 1000, 1024  # the request is oversized through nq and k, not n
    assert bolt.topk_workspace_bytes(n, M, nq, k) > 4 << 20
    codes = torch.zeros(bolt.codes_bytes(n, M), dtype=torch.uint8, device="cuda")
    luts = torch.zeros((nq, M, 16), dtype=torch.uint8, device="cuda")
    out_s = torch.zeros((nq, k), dtype=torch.uint16, device="cuda")
    out_i = torch.zeros((nq, k), dtype=torch.int64, device="cuda")
    rc = L.bolt_topk_noalloc(_p(codes), n, M, _p(luts), nq, k, bolt.METRIC_L2, _p(out_s), _p(out_i),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bolt.ENOMEM
    assert b"4194304" in L.bolt_last_error()
