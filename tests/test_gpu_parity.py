"""GPU parity: every stage of the CUDA path against the CPU oracle on the
same seeded inputs.  Integer outputs (codes, table bytes, sums, top-k) must be
bit-exact; float outputs use the canonical fp32 order on both sides and are
compared bit-exact too, with the fp64 oracle as a 1e-5 relative check.
"""
import numpy as np
import pytest

import oracle
from paper_1706_10283_gb300 import bolt, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bolt.lib()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def decode_blocked(buf, n, M):
    """Independent numpy reading of the blocked layout in include/bolt.h."""
    nb = (n + 255) // 256
    words = np.frombuffer(buf.tobytes(), dtype="<u4").reshape(nb, M, 32)
    nib = (words[..., None] >> (4 * np.arange(8, dtype=np.uint32))) & 15  # (nb, M, 32, 8)
    return nib.transpose(0, 2, 3, 1).reshape(nb * 256, M)[:n].astype(np.uint8)


def problem(n, J, M, seed, kind="mixture", nq=5):
    X = synth.mixture(n, J, seed) if kind == "mixture" else synth.iid(n, J, seed)
    Q = synth.mixture(nq, J, seed + 100) if kind == "mixture" else synth.iid(nq, J, seed + 100)
    nfit = min(n, 4000)
    if nfit >= 16:
        C_ = oracle.kmeans(X[:nfit], M, 4, synth.kmeans_init_rows(nfit, seed))
    else:  # too few rows to seed 16 centroids: random codebooks
        C_ = synth.iid(M * 16, J // M, seed + 7).reshape(M, 16, J // M)
    return X, Q, C_


SHAPES = [(10_000, 32, 8, "iid"), (1_037, 128, 16, "mixture"), (513, 24, 4, "mixture"), (300, 64, 64, "mixture"),
          (257, 16, 1, "mixture"), (40, 256, 32, "mixture"), (5, 8, 2, "iid"), (1000, 6, 3, "iid"),
          (3000, 512, 32, "mixture")]


# ------------------------------------------------------------------ layout
def test_pack_unpack_roundtrip(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(0)
    for n, M in ((1, 1), (255, 3), (256, 16), (1000, 32), (70_001, 8)):
        codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
        blocked = bolt.pack_codes(dev(torch, codes))
        assert blocked.numel() == bolt.codes_bytes(n, M)
        np.testing.assert_array_equal(decode_blocked(blocked.cpu().numpy(), n, M), codes)
        # padding codes are zero
        tail = decode_blocked(blocked.cpu().numpy(), ((n + 255) // 256) * 256, M)[n:]
        assert not tail.any()
        np.testing.assert_array_equal(bolt.unpack_codes(blocked, n, M).cpu().numpy(), codes)


# ------------------------------------------------------------------ encoder
@pytest.mark.parametrize("n,J,M,kind", SHAPES)
def test_encode_fp32_bitexact(torch_cuda, n, J, M, kind):
    torch = torch_cuda
    X, _, C_ = problem(n, J, M, 1, kind)
    got = bolt.encode(dev(torch, X), dev(torch, C_), bolt.PREC_FP32)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(decode_blocked(got.cpu().numpy(), n, M), oracle.encode(X, C_))


def test_encode_adversarial_ties(torch_cuda):
    """Exact ties (duplicated centroids, points on centroids) resolve to the
    lower index on both sides."""
    torch = torch_cuda
    rng = np.random.default_rng(5)
    C_ = rng.integers(-4, 4, (4, 16, 4)).astype(np.float32)
    C_[:, 9] = C_[:, 3]
    pick = rng.integers(0, 16, (3000, 4))
    X = np.concatenate([C_[m, pick[:, m]] for m in range(4)], axis=1)
    X[::7] += np.float32(0.5)  # half-way points between integer centroids
    got = bolt.encode(dev(torch, X), dev(torch, C_))
    np.testing.assert_array_equal(decode_blocked(got.cpu().numpy(), len(X), 4), oracle.encode(X, C_))


TC_SHAPES = [(10_000, 32, 8), (1_037, 128, 16), (40, 256, 32), (513, 64, 4), (777, 64, 2), (3000, 512, 32),
             (1, 128, 16), (129, 128, 16), (257, 128, 16), (20_000, 256, 32),
             # centroids too large for the shared-memory copy: the re-check reads them from global memory
             (3000, 1024, 32), (3000, 1024, 64)]


@pytest.mark.parametrize("n,J,M", TC_SHAPES)
def test_encode_tensor_core_bitexact(torch_cuda, n, J, M):
    """bf16 tensor-core scores + fp32 re-check give the canonical fp32 codes."""
    torch = torch_cuda
    X, _, C_ = problem(n, J, M, 4)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    got = bolt.encode(dev(torch, X), dev(torch, C_), bolt.PREC_BF16_RECHECK, n_rechecked=cnt)
    np.testing.assert_array_equal(decode_blocked(got.cpu().numpy(), n, M), oracle.encode(X, C_))
    assert 0 <= int(cnt.item()) <= n * M


@pytest.mark.parametrize("scale", [1e-3, 1.0, 1e3])
def test_encode_tensor_core_near_ties(torch_cuda, scale):
    """Points at and near the midpoints between centroids, duplicated
    centroids and exact centroid hits: the re-check must resolve every one
    exactly as the fp32 encoder does."""
    torch = torch_cuda
    rng = np.random.default_rng(int(scale * 7) + 1)
    M, s = 16, 8
    C_ = (rng.standard_normal((M, 16, s)) * scale).astype(np.float32)
    C_[:, 5] = C_[:, 2]  # duplicate
    n = 4096
    a = rng.integers(0, 16, (n, M))
    b = rng.integers(0, 16, (n, M))
    w = rng.uniform(0.45, 0.55, (n, M, 1))
    eps = rng.choice([0.0, 1e-7, -1e-7, 1e-5, -1e-5, 1e-3], (n, M, 1))
    sub = np.stack([C_[m, a[:, m]] * (w[:, m] + eps[:, m]) + C_[m, b[:, m]] * (1 - w[:, m] - eps[:, m])
                    for m in range(M)], axis=1)
    sub[::5] = np.stack([C_[m, a[::5, m]] for m in range(M)], axis=1)  # exact hits
    X = sub.reshape(n, M * s).astype(np.float32)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    got = bolt.encode(dev(torch, X), dev(torch, C_), bolt.PREC_BF16_RECHECK, n_rechecked=cnt)
    np.testing.assert_array_equal(decode_blocked(got.cpu().numpy(), n, M), oracle.encode(X, C_))
    assert int(cnt.item()) > 0


# ------------------------------------------------------------------ LUT
@pytest.mark.parametrize("metric", [bolt.METRIC_L2, bolt.METRIC_DOT, bolt.METRIC_L1])
@pytest.mark.parametrize("n,J,M,kind", SHAPES[:5])
def test_luts_bitexact(torch_cuda, metric, n, J, M, kind):
    torch = torch_cuda
    X, Q, C_ = problem(n, J, M, 2, kind, nq=37)
    Dtr = oracle.lut_f32(X[:256], C_, metric)
    a, b, _, _ = oracle.fit_quant(Dtr)
    luts, f32 = bolt.build_luts(dev(torch, Q), dev(torch, C_), metric, a, b, out_f32=True)
    D = oracle.lut_f32(Q, C_, metric)
    np.testing.assert_array_equal(f32.cpu().numpy(), D)
    np.testing.assert_array_equal(luts.cpu().numpy(), oracle.quantize(D, a, b))
    D64 = oracle.lut_f64(Q, C_, metric)
    # 1e-5 relative to the magnitude of the terms summed (|q||c| scale)
    scale = np.abs(D64) if metric != bolt.METRIC_DOT else (
        np.abs(Q).reshape(37, M, 1, -1) * np.abs(C_)[None]).sum(-1)
    assert np.all(np.abs(f32.cpu().numpy() - D64) <= 1e-5 * np.maximum(scale, 1e-30))


# ------------------------------------------------------------------ scan
@pytest.mark.parametrize("n,M", [(1, 1), (300, 3), (4096, 16), (10_007, 8), (70_000, 32), (1000, 256)])
def test_scan_sums_bitexact(torch_cuda, n, M):
    torch = torch_cuda
    rng = np.random.default_rng(n + M)
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, 256, (3, M, 16)).astype(np.uint8)
    blocked = bolt.pack_codes(dev(torch, codes))
    ref = oracle.scan(codes, luts)
    for fn in (bolt.scan_l2, bolt.scan_dot):
        got = fn(blocked, n, M, dev(torch, luts))
        np.testing.assert_array_equal(got.cpu().numpy(), ref)


@pytest.mark.parametrize("n,M,nq", [(150_001, 16, 21), (40_000, 64, 6), (60_000, 8, 9), (3_000, 128, 2)])
def test_scan_sums_query_tiles(torch_cuda, n, M, nq):
    """Scans of several queries run over tiles of up to 8 queries (each code
    word prepared once per tile) split evenly over the CTAs; ragged last
    tiles, shares that span two tiles and a ragged last block, against the
    oracle."""
    torch = torch_cuda
    rng = np.random.default_rng(n + M + nq)
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, 256, (nq, M, 16)).astype(np.uint8)
    got = bolt.scan_l2(bolt.pack_codes(dev(torch, codes)), n, M, dev(torch, luts))
    np.testing.assert_array_equal(got.cpu().numpy(), oracle.scan(codes, luts))


@pytest.mark.parametrize("n,J,M", [(10_000, 32, 8), (1_037, 128, 16), (70_001, 64, 32), (300, 64, 64), (257, 16, 1)])
def test_scan_float_bitexact(torch_cuda, n, J, M):
    """Bolt No Quantize: fp32 sums over the fp32 tables, bit-exact against
    the oracle's sequential sum in codebook order."""
    torch = torch_cuda
    X, Q, C_ = problem(n, J, M, 6, "mixture", nq=9)
    for metric in (bolt.METRIC_L2, bolt.METRIC_DOT):
        codes = oracle.encode(X, C_)
        D = oracle.lut_f32(Q, C_, metric)
        got = bolt.scan_float(bolt.pack_codes(dev(torch, codes)), n, M, dev(torch, D))
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.scan_float(codes, D))


def test_scan_extreme_tables(torch_cuda):
    """All-255 tables at M = 256 reach the largest sum 65280; all-zero give 0."""
    torch = torch_cuda
    n, M = 777, 256
    codes = np.random.default_rng(1).integers(0, 16, (n, M)).astype(np.uint8)
    luts = np.stack([np.full((M, 16), 255, np.uint8), np.zeros((M, 16), np.uint8)])
    got = bolt.scan_l2(bolt.pack_codes(dev(torch, codes)), n, M, dev(torch, luts)).cpu().numpy()
    assert np.all(got[0] == 65280) and np.all(got[1] == 0)


# ------------------------------------------------------------------ top-k
def check_topk(torch, codes, luts, k, metric, workspace=None):
    n, M = codes.shape
    blocked = bolt.pack_codes(dev(torch, codes))
    s, i = bolt.topk(blocked, n, M, dev(torch, luts), k, metric, workspace=workspace)
    rs, ri = oracle.topk(oracle.scan(codes, luts), k, metric)
    np.testing.assert_array_equal(i.cpu().numpy(), ri)
    np.testing.assert_array_equal(s.cpu().numpy(), rs)


@pytest.mark.parametrize("metric", [bolt.METRIC_L2, bolt.METRIC_DOT])
@pytest.mark.parametrize("n,M,k", [(5, 4, 10), (256, 8, 1), (1000, 8, 10), (10_003, 16, 100), (70_000, 16, 37),
                                   (1539, 16, 10), (100_003, 16, 100), (25_603, 8, 64),
                                   (200_000, 8, 100), (50_000, 32, 1000), (20_000, 64, 50), (3000, 128, 20),
                                   (600, 256, 5), (6_000_000, 16, 100), (3_000_000, 32, 10),
                                   (2_600_000, 8, 1024), (400_000, 64, 50), (200_000, 16, 300)])
def test_topk_bitexact(torch_cuda, metric, n, M, k):
    rng = np.random.default_rng(n * 7 + M + k + metric)
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, 256, (3, M, 16)).astype(np.uint8)
    check_topk(torch_cuda, codes, luts, k, metric)


@pytest.mark.parametrize("metric", [bolt.METRIC_L2, bolt.METRIC_DOT])
@pytest.mark.parametrize("hi,nq", [(2, 4), (16, 5), (256, 37), (16, 1), (2, 1)])
def test_topk_large_database_paths(torch_cuda, metric, hi, nq):
    """4,000,000 vectors (103 blocks per CTA: beyond the shared-memory size
    class, which holds up to ~3.3M vectors at M = 16, k = 100).  With 4 or
    more queries: sample bound, multi-query filter and select, tables drawn
    from [0, hi): hi = 2 makes every sum tie (candidate overflow: the exact
    streaming fallback runs), hi = 16 makes hundreds of ties at the k-th sum
    (ordered by index), hi = 256 is the ordinary case; 37 queries span tiles
    of 16, 16, 4 and 1.  One query: the fused streaming kernel."""
    rng = np.random.default_rng(hi * 10 + nq + metric)
    n, M, k = 4_000_000, 16, 100
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, hi, (nq, M, 16)).astype(np.uint8)
    check_topk(torch_cuda, codes, luts, k, metric)


@pytest.mark.parametrize("n,M,k,nq", [(1000, 8, 10, 1), (100_003, 16, 100, 2), (4_000_000, 16, 50, 5)])
def test_topk_l1_tables_rank_ascending(torch_cuda, n, M, k, nq):
    """L1 tables (the L_p family with p = 1): top-k ranks by ascending sum,
    through every size class (shared-memory, streaming, multi-query)."""
    rng = np.random.default_rng(n + M + k)
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, 256, (nq, M, 16)).astype(np.uint8)
    check_topk(torch_cuda, codes, luts, k, bolt.METRIC_L1)


@pytest.mark.parametrize("p", [0.5, 1.5, 3.0])
def test_lp_tables_fit_and_topk(torch_cuda, p):
    """L_p tables (delta = |q - c|^p): the GPU's fp32 entries (CUDA powf)
    within 1e-5 of the oracle's fp64 tables; its bytes equal the oracle's
    quantization of those fp32 entries; the quantizer fit over L_p tables
    equals the oracle's fit of the same fp32 tables; and top-k with the L_p
    metric over the GPU's bytes equals the oracle's, in the shared-memory,
    streaming and multi-query size classes."""
    torch = torch_cuda
    rng = np.random.default_rng(int(p * 10))
    J, M = 64, 16
    X = synth.mixture(30_000, J, 71)
    C_ = oracle.kmeans(X[:5_000], M, 4, synth.kmeans_init_rows(5_000, 71))
    Qtr = X[synth.train_query_rows(30_000, 71)]
    Q = synth.mixture(5, J, 72)
    Cd = dev(torch, C_)
    # fit: over the GPU's own fp32 tables of the training queries
    _, Dtr = bolt.build_luts_lp(dev(torch, Qtr), Cd, p, 1.0, np.zeros(M, np.float32), out_f32=True)
    a, b, ai = bolt.fit_quantizer_lp(dev(torch, Qtr), Cd, p)
    oa, ob, oai, _ = oracle.fit_quant(Dtr.cpu().numpy())
    assert (a, ai) == (np.float32(oa), oai)
    np.testing.assert_array_equal(b, ob)
    luts, D = bolt.build_luts_lp(dev(torch, Q), Cd, p, a, b, out_f32=True)
    Dg = D.cpu().numpy()
    ref = oracle.lut_lp_f64(Q, C_, p)
    np.testing.assert_allclose(Dg, ref, rtol=1e-5, atol=1e-5 * float(np.abs(ref).max()))
    lg = luts.cpu().numpy()
    np.testing.assert_array_equal(lg, oracle.quantize(Dg, a, b))
    for n in (10_003, 4_000_000):
        codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
        blocked = bolt.pack_codes(dev(torch, codes))
        for nq in (1, 5):
            s_, i_ = bolt.topk(blocked, n, M, luts[:nq], 100, bolt.METRIC_LP)
            rs, ri = oracle.topk(oracle.scan(codes, lg[:nq]), 100, oracle.METRIC_LP)
            np.testing.assert_array_equal(i_.cpu().numpy(), ri)
            np.testing.assert_array_equal(s_.cpu().numpy(), rs)


@pytest.mark.parametrize("metric", [bolt.METRIC_L2, bolt.METRIC_DOT])
def test_topk_heavy_ties(torch_cuda, metric):
    """Tables with 2 distinct values: huge tie groups decided by index."""
    rng = np.random.default_rng(3)
    n, M = 100_000, 8
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, 2, (2, M, 16)).astype(np.uint8)
    check_topk(torch_cuda, codes, luts, 100, metric)
    luts0 = np.zeros((1, M, 16), np.uint8)  # every sum equal
    check_topk(torch_cuda, codes, luts0, 64, metric)


@pytest.mark.parametrize("metric", [bolt.METRIC_L2, bolt.METRIC_DOT])
def test_topk_small_class_winners_in_one_range(torch_cuda, metric):
    """Shared-memory size class with the best sums all in the first rows
    (rows ordered by their sum under the query's tables): the first CTA's list
    holds every winner, more than the merge's 16-key prefix, so the merge
    takes its exact path (global histogram, searches past the prefix)."""
    rng = np.random.default_rng(11 + metric)
    n, M, k = 100_003, 16, 100
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, 256, (2, M, 16)).astype(np.uint8)
    S = luts[0][np.arange(M)[None, :], codes].astype(np.int64).sum(axis=1)
    order = np.argsort(S if metric == bolt.METRIC_L2 else -S, kind="stable")
    check_topk(torch_cuda, codes[order], luts, k, metric)


def test_topk_sorted_input_worst_case(torch_cuda):
    """Sums decreasing with the index: every block improves the threshold."""
    torch = torch_cuda
    n, M = 60_000, 16
    codes = np.zeros((n, M), np.uint8)
    val = (15 - (np.arange(n) * 16 // n)).astype(np.uint8)
    codes[:, :] = val[:, None]
    luts = np.tile(np.arange(16, dtype=np.uint8) * 16, (1, M, 1))
    check_topk(torch, codes, luts, 100, bolt.METRIC_L2)


@pytest.mark.parametrize("pattern", ["concentrated", "sorted"])
@pytest.mark.parametrize("metric", [bolt.METRIC_L2, bolt.METRIC_DOT])
def test_topk_streaming_kernel_stress(torch_cuda, pattern, metric):
    """The streaming kernel (one query, 4,000,000 vectors) where one CTA's
    range decides the top k: "concentrated" puts 20,000 vectors with small,
    sparsely tied sums inside one range (its local thresholds meet the
    global k-th sum, where warps out of lockstep matter); "sorted" makes the
    sums decrease with the index (every block improves the threshold).
    Twelve repeated launches must all equal the oracle."""
    torch = torch_cuda
    rng = np.random.default_rng(71 + metric)
    n, M, k = 4_000_000, 16, 100
    luts = rng.integers(0, 256, (1, M, 16)).astype(np.uint8)
    if pattern == "concentrated":
        codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
        # rows whose codes pick each table's 3 best entries: small sums, few ties each
        order = np.argsort(luts[0] if metric == bolt.METRIC_L2 else -luts[0].astype(np.int32), axis=1)
        pick = rng.integers(0, 3, (20_000, M))
        codes[1_000_000:1_020_000] = order[np.arange(M)[None, :], pick].astype(np.uint8)
    else:
        luts = np.tile((np.arange(16, dtype=np.uint8) * 16)[None, None, :], (1, M, 1))
        val = (15 - (np.arange(n) * 16 // n)).astype(np.uint8)
        if metric == bolt.METRIC_DOT:
            val = 15 - val
        codes = np.repeat(val[:, None], M, axis=1)
        codes[::7] = rng.integers(0, 16, (len(codes[::7]), M))  # break the exact ties a little
    blocked = bolt.pack_codes(dev(torch, codes))
    L = dev(torch, luts)
    rs, ri = oracle.topk(oracle.scan(codes, luts), k, metric)
    for _ in range(12):
        s, i = bolt.topk(blocked, n, M, L, k, metric)
        np.testing.assert_array_equal(i.cpu().numpy(), ri)
        np.testing.assert_array_equal(s.cpu().numpy(), rs)


def test_topk_explicit_workspace(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(4)
    n, M, k = 30_000, 16, 50
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, 256, (4, M, 16)).astype(np.uint8)
    ws = torch.empty(bolt.topk_workspace_bytes(n, M, 4, k), dtype=torch.uint8, device="cuda")
    for _ in range(2):  # reuse of one workspace
        check_topk(torch, codes, luts, k, bolt.METRIC_L2, workspace=ws)
    with pytest.raises(bolt.BoltError):
        small = torch.empty(16, dtype=torch.uint8, device="cuda")
        blocked = bolt.pack_codes(dev(torch, codes))
        bolt.topk(blocked, n, M, dev(torch, luts), k, bolt.METRIC_L2, workspace=small)


# ------------------------------------------------------------------ dequantize / matmul
def test_dequantize_bitexact(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(6)
    S = rng.integers(0, 65281, 10_001).astype(np.uint16)
    a, b = np.float32(0.37), rng.standard_normal(16).astype(np.float32)
    got = bolt.dequantize(dev(torch, S), a, b).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.dequant(S, a, b))


@pytest.mark.parametrize("rows,n,J,M", [(37, 1000, 64, 8), (8, 257, 32, 32), (100, 5000, 128, 16)])
def test_approx_matmul_bitexact(torch_cuda, rows, n, J, M):
    torch = torch_cuda
    B = synth.mixture(n, J, 0)
    A = synth.iid(rows, J, 9)
    C_ = oracle.kmeans(B, M, 4, synth.kmeans_init_rows(n, 0))
    a, b, _, _ = oracle.fit_quant(oracle.lut_f32(A, C_, oracle.METRIC_DOT))
    codes = oracle.encode(B, C_)
    blocked = bolt.pack_codes(dev(torch, codes))
    got = bolt.approx_matmul(dev(torch, A), blocked, n, dev(torch, C_), a, b).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.matmul(A, codes, C_, a, b))


# ------------------------------------------------------------------ fit
@pytest.mark.parametrize("n,J,M,iters", [(5000, 32, 8, 8), (3000, 64, 16, 5), (10_000, 16, 1, 6)])
def test_kmeans_matches_oracle(torch_cuda, n, J, M, iters):
    torch = torch_cuda
    X = synth.mixture(n, J, 3)
    rows = synth.kmeans_init_rows(n, 3)
    got = bolt.fit_codebooks(dev(torch, X), M, iters, rows).cpu().numpy()
    ref, obj = oracle.kmeans(X, M, iters, rows, return_objective=True)
    # fp64 means summed in a different (fixed) order: equal up to the last bit
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6)
    codes_g = oracle.encode(X, got)
    xh = oracle.decode(codes_g, got).astype(np.float64)
    obj_g = ((X.astype(np.float64) - xh) ** 2).sum()
    assert abs(obj_g - obj[-1]) <= 1e-5 * obj[-1]


def test_kmeans_million_rows_matches_oracle(torch_cuda):
    """k-means at scale: 1,000,000 x 128 mixture rows, M = 16, 4 Lloyd
    iterations from the seeded init (Sec. 3.1 background).  The GPU sums the
    fp64 centroid means over 489 fixed chunks of 2,048 rows, the oracle in
    row order: centroids within rtol 1e-5 and the objective of the GPU
    centroids within 1e-5 of the oracle's."""
    torch = torch_cuda
    n, J, M, iters = 1_000_000, 128, 16, 4
    X = synth.mixture(n, J, 4)
    rows = synth.kmeans_init_rows(n, 4)
    got = bolt.fit_codebooks(dev(torch, X), M, iters, rows).cpu().numpy()
    ref, obj = oracle.kmeans(X, M, iters, rows, return_objective=True)
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6)
    from oracle import parallel

    xh = oracle.decode(parallel.encode(X, got), got).astype(np.float64)
    obj_g = ((X.astype(np.float64) - xh) ** 2).sum()
    assert abs(obj_g - obj[-1]) <= 1e-5 * obj[-1]


@pytest.mark.parametrize("metric", [bolt.METRIC_L2, bolt.METRIC_DOT])
def test_fit_quantizer_matches_oracle(torch_cuda, metric):
    torch = torch_cuda
    X, Q, C_ = problem(3000, 64, 8, 7)
    Qtr = X[synth.train_query_rows(len(X), 7)]
    a, b, ai = bolt.fit_quantizer(dev(torch, Qtr), dev(torch, C_), metric)
    ra, rb, rai, _ = oracle.fit_quant(oracle.lut_f32(Qtr, C_, metric))
    assert ai == rai
    assert a == ra
    np.testing.assert_array_equal(b, rb)


# ------------------------------------------------------------------ workloads
def test_small_iid_workload_end_to_end(torch_cuda):
    """10,000 x 32 i.i.d. N(0,1), M = 8, 16 queries, top-10 (L2): fit, encode,
    tables and top-k on the GPU against the oracle."""
    torch = torch_cuda
    cfg = synth.CONFIGS["small_iid_l2"]
    X = synth.iid(cfg["n"], cfg["J"], 0)
    Q = synth.iid(cfg["nq"], cfg["J"], 1)
    rows = synth.kmeans_init_rows(cfg["n"], 0)
    Qtr = X[synth.train_query_rows(cfg["n"], 0)]
    Cg, ag, bg = bolt.fit_codebooks(dev(torch, X), cfg["M"], cfg["iters"], rows, Qtrain=dev(torch, Qtr))
    Co = oracle.kmeans(X, cfg["M"], cfg["iters"], rows)
    np.testing.assert_allclose(Cg.cpu().numpy(), Co, rtol=1e-5, atol=1e-6)
    # downstream parity feeds the same centroids and quantizer to both sides
    a, b, _, _ = oracle.fit_quant(oracle.lut_f32(Qtr, Co, oracle.METRIC_L2))
    Cd = dev(torch, Co)
    codes = bolt.encode(dev(torch, X), Cd)
    luts = bolt.build_luts(dev(torch, Q), Cd, bolt.METRIC_L2, a, b)
    s, i = bolt.topk(codes, cfg["n"], cfg["M"], luts, cfg["k"], bolt.METRIC_L2)
    oc = oracle.encode(X, Co)
    ol = oracle.quantize(oracle.lut_f32(Q, Co, oracle.METRIC_L2), a, b)
    rs, ri = oracle.topk(oracle.scan(oc, ol), cfg["k"], oracle.METRIC_L2)
    np.testing.assert_array_equal(decode_blocked(codes.cpu().numpy(), cfg["n"], cfg["M"]), oc)
    np.testing.assert_array_equal(luts.cpu().numpy(), ol)
    np.testing.assert_array_equal(i.cpu().numpy(), ri)
    np.testing.assert_array_equal(s.cpu().numpy(), rs)


def test_mixture_1m_workload_full_size(torch_cuda):
    """1,000,000 x 128 mixture, M = 16, top-100 L2 and dot, launched as in
    the benchmark (one query per launch): all codes against the oracle, and
    the top-k of a seeded sample of the 1,000 queries."""
    torch = torch_cuda
    cfg = synth.CONFIGS["mixture_1m"]
    n, J, M, k = cfg["n"], cfg["J"], cfg["M"], cfg["k"]
    X = synth.mixture(n, J, 0)
    Q = synth.mixture(cfg["nq"], J, 1)
    rows = synth.kmeans_init_rows(n, 0)
    Co = oracle.kmeans(X[:20_000], M, 4, synth.kmeans_init_rows(20_000, 0))
    Cd = dev(torch, Co)
    codes = bolt.encode(dev(torch, X), Cd)
    oc = oracle.encode(X, Co)
    np.testing.assert_array_equal(decode_blocked(codes.cpu().numpy(), n, M), oc)
    Qtr = X[synth.train_query_rows(n, 0)]
    sample = np.random.default_rng(11).choice(cfg["nq"], 6, replace=False)
    for metric in (oracle.METRIC_L2, oracle.METRIC_DOT):
        a, b, _, _ = oracle.fit_quant(oracle.lut_f32(Qtr, Co, metric))
        luts = bolt.build_luts(dev(torch, Q), Cd, metric, a, b)
        ol = oracle.quantize(oracle.lut_f32(Q, Co, metric), a, b)
        np.testing.assert_array_equal(luts.cpu().numpy(), ol)
        for qi in sample:
            s, i = bolt.topk(codes, n, M, luts[qi:qi + 1], k, metric)
            rs, ri = oracle.topk(oracle.scan(oc, ol[qi:qi + 1]), k, metric)
            np.testing.assert_array_equal(i.cpu().numpy(), ri)
            np.testing.assert_array_equal(s.cpu().numpy(), rs)
    del rows


def clustered_codes(n, M, seed, clusters=256, chunk=5_000_000):
    """Codes with the structure of an encoded mixture: each row belongs to
    one of `clusters` groups and takes its group's code in a codebook with
    probability 1/2, else a uniform code."""
    rng = np.random.default_rng(seed)
    pref = rng.integers(0, 16, (clusters, M), dtype=np.uint8)
    out = np.empty((n, M), np.uint8)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        g = rng.integers(0, clusters, hi - lo)
        r = rng.integers(0, 32, (hi - lo, M), dtype=np.uint8)
        out[lo:hi] = np.where(r < 16, r, pref[g])
    return out


def test_serve_50m_full_size_topk(torch_cuda):
    """50,000,000 vectors, M = 16, top-100 (the serving database), launched
    as the benchmark times it: one query per launch (fused streaming kernel)
    and an 8-query batch (multi-query pipeline), L2 and dot tables built by
    the oracle from mixture queries; every result against the oracle."""
    torch = torch_cuda
    cfg = synth.CONFIGS["serve_50m"]
    n, J, M, k = cfg["n"], cfg["J"], cfg["M"], 100
    codes = clustered_codes(n, M, 50)
    blocked = bolt.pack_codes(dev(torch, codes))
    torch.cuda.synchronize()
    X = synth.mixture(20_000, J, 51)
    Co = oracle.kmeans(X, M, 4, synth.kmeans_init_rows(20_000, 51))
    Q = synth.mixture(8, J, 52)
    for metric in (oracle.METRIC_L2, oracle.METRIC_DOT):
        a, b, _, _ = oracle.fit_quant(oracle.lut_f32(X[:2000], Co, metric))
        ol = oracle.quantize(oracle.lut_f32(Q, Co, metric), a, b)
        rs, ri = oracle.topk(oracle.scan(codes, ol), k, metric)
        L = dev(torch, ol)
        for qi in range(2):
            s, i = bolt.topk(blocked, n, M, L[qi:qi + 1], k, metric)
            np.testing.assert_array_equal(i.cpu().numpy(), ri[qi:qi + 1])
            np.testing.assert_array_equal(s.cpu().numpy(), rs[qi:qi + 1])
        s, i = bolt.topk(blocked, n, M, L, k, metric)
        np.testing.assert_array_equal(i.cpu().numpy(), ri)
        np.testing.assert_array_equal(s.cpu().numpy(), rs)


def test_encode_10m_full_size(torch_cuda):
    """10,000,000 x 256 mixture rows, M = 32, encoded in one launch by the
    fp32 encoder and by the tensor-core encoder with fp32 re-check, as the
    benchmark times them: the two encoders' codes equal everywhere, and the
    codes of a seeded sample of 16,384 rows equal the oracle's."""
    torch = torch_cuda
    cfg = synth.CONFIGS["encode_10m"]
    n, J, M = cfg["n"], cfg["J"], cfg["M"]
    X = synth.mixture_torch(n, J, seed=0)
    Co = oracle.kmeans(X[:20_000].cpu().numpy(), M, 4, synth.kmeans_init_rows(20_000, 0))
    Cd = dev(torch, Co)
    c32 = bolt.encode(X, Cd, bolt.PREC_FP32)
    ctc = bolt.encode(X, Cd, bolt.PREC_BF16_RECHECK)
    assert torch.equal(c32, ctc)
    rows = np.sort(np.random.default_rng(12).choice(n, 16_384, replace=False))
    Xs = X[torch.from_numpy(rows).cuda()].cpu().numpy()
    del X
    blocks = np.unique(rows // 256)
    got_blocks = c32.view(-1, M * 128)[torch.from_numpy(blocks).cuda()].cpu().numpy()
    dec = decode_blocked(got_blocks, len(blocks) * 256, M)
    pos = np.searchsorted(blocks, rows // 256) * 256 + rows % 256
    np.testing.assert_array_equal(dec[pos], oracle.encode(Xs, Co))


def test_approx_matmul_full_size(torch_cuda):
    """A (4,096 x 512) times the encoded B (100,000 x 512, M = 32), one call
    as the benchmark and the serving mix issue it: a seeded sample of 16
    output rows against the oracle."""
    torch = torch_cuda
    cfg = synth.CONFIGS["matmul_4096x512_100k"]
    rows, n, J, M = cfg["rows"], cfg["n"], cfg["J"], cfg["M"]
    B = synth.mixture(n, J, 31)
    A = synth.mixture(rows, J, 32)
    C_ = oracle.kmeans(B[:20_000], M, 4, synth.kmeans_init_rows(20_000, 31))
    a, b, _, _ = oracle.fit_quant(oracle.lut_f32(A[:256], C_, oracle.METRIC_DOT))
    codes = oracle.encode(B, C_)
    blocked = bolt.pack_codes(dev(torch, codes))
    got = bolt.approx_matmul(dev(torch, A), blocked, n, dev(torch, C_), a, b)
    sample = np.sort(np.random.default_rng(33).choice(rows, 16, replace=False))
    np.testing.assert_array_equal(got[torch.from_numpy(sample).cuda()].cpu().numpy(),
                                  oracle.matmul(A[sample], codes, C_, a, b))


# ------------------------------------------------------------------ more than 256 codebooks
@pytest.mark.parametrize("n,M", [(1, 1), (1000, 16), (300, 256), (5000, 257), (2049, 300), (777, 1024),
                                 (300, 4096)])
def test_scan_u32_bitexact(torch_cuda, n, M):
    """uint32 sums for any M up to 4096 (chunks of 256 codebooks in the
    uint16 form, added in 32 bits) against the oracle; for M <= 256 also the
    uint16 scan; and the uint32 dequantization."""
    torch = torch_cuda
    rng = np.random.default_rng(n + M)
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, 256, (3, M, 16)).astype(np.uint8)
    luts[1] = 255  # the largest sums: 255 M
    blocked = bolt.pack_codes(dev(torch, codes))
    L = dev(torch, luts)
    got = bolt.scan_u32(blocked, n, M, L)
    want = oracle.scan_u32(codes, luts)
    np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32), want)
    if M <= 256:
        np.testing.assert_array_equal(bolt.scan_l2(blocked, n, M, L).cpu().numpy(), want.astype(np.uint16))
    b = rng.standard_normal(M).astype(np.float32)
    np.testing.assert_array_equal(bolt.dequantize_u32(got, 0.37, b).cpu().numpy(), oracle.dequant_u32(want, 0.37, b))


@pytest.mark.parametrize("metric", [bolt.METRIC_L2, bolt.METRIC_DOT, bolt.METRIC_L1])
@pytest.mark.parametrize("n,M,k,nq,hi", [(1, 257, 1, 1, 256), (5, 300, 10, 2, 256), (20_003, 257, 100, 3, 256),
                                          (70_001, 512, 1024, 2, 256), (300_001, 512, 100, 2, 256),
                                          (4_100, 4096, 1, 2, 256), (50_000, 512, 100, 2, 2),
                                          (40_000, 300, 64, 2, 1)])
def test_topk_u32_bitexact(torch_cuda, metric, n, M, k, nq, hi):
    """Fused top-k over uint32 sums for more than 256 codebooks (M up to
    4096) against the oracle's selection over its own uint32 scan: ragged
    n, k > n (padding), k = 1 and 1024, tables drawn from [0, hi) -- hi = 2
    makes long tie runs at the k-th sum, hi = 1 makes every sum equal (the
    first k indices) -- and the dot order; the sums exceed 65,535."""
    torch = torch_cuda
    rng = np.random.default_rng(n + M + k + metric)
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, hi, (nq, M, 16)).astype(np.uint8)
    if hi == 256:
        luts[0] = np.maximum(luts[0], 200)  # large sums: up to 255 M
    blocked = bolt.pack_codes(dev(torch, codes))
    s, i = bolt.topk_u32(blocked, n, M, dev(torch, luts), k, metric)
    rs, ri = oracle.topk_u32(oracle.scan_u32(codes, luts), k, metric)
    np.testing.assert_array_equal(i.cpu().numpy(), ri)
    np.testing.assert_array_equal(s.cpu().numpy().view(np.uint32), rs)


def test_topk_u32_explicit_workspace_twice(torch_cuda):
    """A caller-provided workspace reused by two calls in a row (the
    histograms and counters are cleared by each call)."""
    torch = torch_cuda
    rng = np.random.default_rng(5)
    n, M, k = 100_003, 512, 50
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    blocked = bolt.pack_codes(dev(torch, codes))
    ws = torch.empty(bolt.topk_u32_workspace_bytes(n, M, 2, k), dtype=torch.uint8, device="cuda")
    for metric in (bolt.METRIC_L2, bolt.METRIC_DOT):
        luts = rng.integers(0, 256, (2, M, 16)).astype(np.uint8)
        s, i = bolt.topk_u32(blocked, n, M, dev(torch, luts), k, metric, workspace=ws)
        rs, ri = oracle.topk_u32(oracle.scan_u32(codes, luts), k, metric)
        np.testing.assert_array_equal(i.cpu().numpy(), ri)
        np.testing.assert_array_equal(s.cpu().numpy().view(np.uint32), rs)


def test_more_than_256_codebooks_end_to_end(torch_cuda):
    """M = 512 codebooks of s = 2 dims: codes (both precisions run the fp32
    encoder), layout round trip, L2 and dot tables with the oracle's fitted
    a and b, uint32 sums and their dequantization, all against the oracle;
    the uint16-sum entry points refuse M > 256."""
    torch = torch_cuda
    n, M, s = 3000, 512, 2
    J = M * s
    X = synth.mixture(n, J, 71)
    Q = synth.mixture(5, J, 72)
    C_ = oracle.kmeans(X, M, 3, synth.kmeans_init_rows(n, 71))
    Xd, Cd = dev(torch, X), dev(torch, C_)
    oc = oracle.encode(X, C_)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for prec in (bolt.PREC_FP32, bolt.PREC_BF16_RECHECK):
        blocked = bolt.encode(Xd, Cd, prec, n_rechecked=cnt)
        np.testing.assert_array_equal(decode_blocked(blocked.cpu().numpy(), n, M), oc)
        assert int(cnt.item()) == 0
    np.testing.assert_array_equal(bolt.unpack_codes(blocked, n, M).cpu().numpy(), oc)
    for metric in (oracle.METRIC_L2, oracle.METRIC_DOT):
        a, b, _, _ = oracle.fit_quant(oracle.lut_f32(X[:64], C_, metric))
        luts = bolt.build_luts(dev(torch, Q), Cd, metric, a, b)
        ol = oracle.quantize(oracle.lut_f32(Q, C_, metric), a, b)
        np.testing.assert_array_equal(luts.cpu().numpy(), ol)
        S = bolt.scan_u32(blocked, n, M, luts)
        oS = oracle.scan_u32(oc, ol)
        np.testing.assert_array_equal(S.cpu().numpy().view(np.uint32), oS)
        np.testing.assert_array_equal(bolt.dequantize_u32(S, a, b).cpu().numpy(), oracle.dequant_u32(oS, a, b))
        for fn in (lambda: bolt.scan_l2(blocked, n, M, luts), lambda: bolt.topk(blocked, n, M, luts, 10, metric)):
            with pytest.raises(bolt.BoltError):
                fn()
