"""Host-only checks of the C ABI: the library builds, loads and exports
every entry point include/bolt.h declares; host-side helpers and argument
validation work without a GPU (no kernel is launched here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_1706_10283_gb300 import bolt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bolt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bolt_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = bolt.lib()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
        assert name in bolt.exported_symbols(), name
    assert b"sm_103a" in L.bolt_version()


def test_codes_bytes_layout_arithmetic():
    # ceil(n/256) blocks of M rows of 128 bytes
    assert bolt.codes_bytes(0, 16) == 0
    assert bolt.codes_bytes(1, 16) == 16 * 128
    assert bolt.codes_bytes(256, 8) == 8 * 128
    assert bolt.codes_bytes(257, 8) == 2 * 8 * 128
    assert bolt.codes_bytes(1_000_000, 16) == 3907 * 16 * 128
    # M/2 bytes per vector once blocks are full (the paper's 8B/16B/32B codes)
    for M, nbytes in ((16, 8), (32, 16), (64, 32)):
        assert bolt.codes_bytes(256 * 1000, M) == 256 * 1000 * nbytes
    assert bolt.lib().bolt_codes_bytes(-1, 4) == -1
    assert bolt.lib().bolt_codes_bytes(10, 257) == 257 * 128  # up to 4096 codebooks (uint32 sums)
    assert bolt.lib().bolt_codes_bytes(10, 4096) == 4096 * 128
    assert bolt.lib().bolt_codes_bytes(10, 4097) == -1
    assert bolt.lib().bolt_codes_bytes(10, 0) == -1


def test_dequant_params_match_oracle():
    rng = np.random.default_rng(0)
    for M in (1, 8, 32, 256, 1000):
        a = np.float32(rng.uniform(0.01, 10))
        b = rng.standard_normal(M).astype(np.float32) * 100
        assert bolt.dequant_params(a, b) == tuple(float(v) for v in oracle.dequant_params(a, b))


def test_invalid_arguments_are_rejected_on_host():
    L = bolt.lib()
    nul = C.c_void_p(0)
    # J not a multiple of M
    rc = L.bolt_encode(nul, 10, 30, 8, nul, 0, nul, nul, nul)
    assert rc == bolt.EUNSUPPORTED and b"multiple" in L.bolt_last_error()
    # M > 256
    assert L.bolt_scan_l2(nul, 10, 300, nul, 1, nul, nul) == bolt.EUNSUPPORTED
    # bad metric
    assert L.bolt_build_luts(nul, 1, 8, 2, nul, 7, C.c_float(1.0), nul, nul, nul, nul) == bolt.EINVAL
    # k out of range
    assert L.bolt_topk_workspace_bytes(100, 8, 1, 0) == -1
    assert L.bolt_topk_workspace_bytes(100, 8, 1, 5000) == -1
    # top-k keeps uint16 sums: M <= 256 (the uint32 scan takes up to 4096)
    assert L.bolt_topk_workspace_bytes(100, 257, 1, 10) == -1
    assert L.bolt_scan_u32(nul, 10, 4097, nul, 1, nul, nul) == bolt.EUNSUPPORTED
    assert L.bolt_scan_u32(nul, 10, 4096, nul, 1, nul, nul) == bolt.EINVAL  # passes the M check, then null
    assert L.bolt_encode(nul, 10, 8194, 4097, nul, 0, nul, nul, nul) == bolt.EUNSUPPORTED
    # non-positive scale
    ia, bb = C.c_float(), C.c_float()
    arr = np.zeros(4, np.float32)
    assert L.bolt_dequant_params(C.c_float(0.0), arr.ctypes.data_as(C.c_void_p), 4, C.byref(ia), C.byref(bb)) \
        == bolt.EINVAL


def test_binding_fails_loudly_without_cuda():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(bolt.BoltError):
        bolt.encode(torch.zeros(4, 8), torch.zeros(2, 16, 4))


def _coll(n, M, nq, ld=None, qt=0, upw=0, codes=0x10000, luts=0x20000, sums=0x30000, sum_bits=0):
    return bolt.Collection(codes, luts, sums, n, nq, bolt.sums_ld(n) if ld is None else ld, M, qt, upw, sum_bits)


def _plan_bytes(*colls):
    arr = (bolt.Collection * max(1, len(colls)))(*colls)
    return int(bolt.lib().bolt_batch_plan_bytes(C.cast(arr, C.c_void_p), len(colls)))


def test_batch_planner_task_counts():
    """Host planner: 64-byte header, a 48-byte record per collection and a
    24-byte task per (query group, block range)."""
    H, R, T = 64, 48, 24
    assert _plan_bytes() == H
    # 64 blocks, 16 queries, qt 8: one group of 2 tiles; 8 warps x 4 units
    # per task = 32 units = 16 blocks x 2 tiles -> 4 tasks
    assert _plan_bytes(_coll(64 * 256, 16, 16, qt=8, upw=4)) == H + R + 4 * T
    # 37 queries at qt 8: tiles 8,8,8,8 (one group) + 4 + 1; 1 block each
    assert _plan_bytes(_coll(100, 16, 37, qt=8, upw=4)) == H + R + 3 * T
    # M = 256: 16 x 256 table rows exceed the 1024 staged, so qt drops to 4
    # and a group holds one tile: 9 queries -> tiles 4, 4, 1 -> 3 groups
    assert _plan_bytes(_coll(256, 256, 9, qt=16, upw=1)) == H + R + 3 * T
    # empty collections have no tasks but keep their record
    assert _plan_bytes(_coll(0, 8, 5), _coll(100, 8, 0)) == H + 2 * R
    # uint32 sums: at most 2 queries per tile; M = 300 stages one query's
    # 300 table rows per group (5 queries -> tiles 2, 2, 1, one per group);
    # M = 2048 (too large to stage) also tiles of 2
    assert _plan_bytes(_coll(256, 300, 5, qt=16, upw=1, sum_bits=32)) == H + R + 3 * T
    assert _plan_bytes(_coll(256, 2048, 4, qt=8, upw=1, sum_bits=32)) == H + R + 2 * T
    # both lists in one plan: the uint16 tasks, then the uint32 ones
    assert _plan_bytes(_coll(100, 16, 37, qt=8, upw=4), _coll(256, 300, 5, qt=16, upw=1, sum_bits=32)) == \
        H + 2 * R + 6 * T


def test_batch_planner_rejects_bad_collections():
    L = bolt.lib()
    bad = [_coll(100, 0, 2), _coll(100, 257, 2), _coll(100, 8, 2, ld=100), _coll(100, 8, 2, ld=96),
           _coll(100, 8, 2, qt=3), _coll(100, 8, 2, upw=65), _coll(100, 8, 2, sum_bits=1),
           _coll(100, 8, 2, sum_bits=8), _coll(100, 4097, 2, sum_bits=32), _coll(100, 257, 2, sum_bits=16),
           _coll(100, 8, 2, codes=0x10001), _coll(100, 8, 2, sums=0), _coll(-1, 8, 2)]
    for c in bad:
        assert _plan_bytes(c) < 0
        assert L.bolt_last_error()
    # a bad record anywhere fails the whole batch
    assert _plan_bytes(_coll(100, 8, 2), _coll(100, 8, 2, qt=5)) < 0
    assert L.bolt_scan_batched(C.c_void_p(0), C.c_void_p(0)) == bolt.EINVAL


def test_topk_workspace_query_host_only():
    """The workspace query plans on the host: positive for every size class,
    growing with the number of queries, -1 for invalid shapes."""
    L = bolt.lib()
    for n, M, k in ((1, 1, 1), (1000, 16, 10), (1_000_000, 16, 100), (50_000_000, 16, 100), (3_000_000, 32, 1000),
                    (10, 256, 1)):
        sizes = [L.bolt_topk_workspace_bytes(n, M, nq, k) for nq in (1, 4, 64)]
        assert all(v > 0 for v in sizes) and sizes[0] <= sizes[1] <= sizes[2], (n, M, k, sizes)
    assert L.bolt_topk_workspace_bytes(-1, 16, 1, 10) == -1
    assert L.bolt_topk_workspace_bytes(100, 0, 1, 10) == -1
    assert L.bolt_topk_workspace_bytes(100, 16, -1, 10) == -1
