"""Batched multi-collection scan (one persistent launch over many
collections) against the CPU oracle: codes, tables and sums bit-exact.

The workload: collections with N log-uniform in [1e3, 2e6], J in {64, 128,
256}, M in {8, 16, 32}, 1..256 queries each, Gaussian-mixture data
(``synth.collections``).  A scaled-down batch is compared element by
element; the full 64-collection batch is compared on seeded samples of rows
(every query) in the launch configuration the benchmark times.
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


def decode_rows(buf, rows, M):
    """Codes of the given rows from the blocked layout (numpy reading of
    include/bolt.h): row r is nibble r % 8 of word (r % 256) // 8 in row m of
    block r // 256."""
    words = np.frombuffer(buf.tobytes(), dtype="<u4").reshape(-1, M, 32)
    rows = np.asarray(rows)
    w = words[rows // 256, :, (rows % 256) // 8]  # (len(rows), M)
    return ((w >> (4 * (rows % 8))[:, None].astype(np.uint32)) & 15).astype(np.uint8)


def oracle_params(X_fit, Qtr, M, seed, metric):
    """Centroids (oracle k-means, 4 iterations on the fit rows) and the
    quantizer fitted by the oracle: the inputs both sides share."""
    nf = X_fit.shape[0]
    Co = oracle.kmeans(X_fit, M, 4, synth.kmeans_init_rows(nf, seed))
    a, b, _, _ = oracle.fit_quant(oracle.lut_f32(Qtr, Co, metric))
    return Co, a, b


SMALL_SPECS = synth.collections(seed=5, count=10, n_hi=3e4)


def u16(torch, shape, fill=0):
    """uint16 device tensor filled with `fill` (torch fills int16; same bits)."""
    v = fill - 65536 if fill >= 32768 else fill
    return torch.full(shape, v, dtype=torch.int16, device="cuda").view(torch.uint16)


def small_batch(torch, specs):
    """Per collection: GPU codes and tables, oracle codes and tables."""
    out = []
    for ci, sp in enumerate(specs):
        n, J, M, nq = sp["n"], sp["J"], sp["M"], sp["nq"]
        metric = ci % 2
        X = synth.mixture(n, J, sp["data_seed"])
        Q = synth.mixture(nq, J, sp["query_seed"])
        nf = min(n, 4000)
        Qtr = X[synth.train_query_rows(n, sp["data_seed"])]
        Co, a, b = oracle_params(X[:nf], Qtr, M, sp["data_seed"], metric)
        Cd = dev(torch, Co)
        codes = bolt.encode(dev(torch, X), Cd)
        luts = bolt.build_luts(dev(torch, Q), Cd, metric, a, b)
        oc = oracle.encode(X, Co)
        ol = oracle.quantize(oracle.lut_f32(Q, Co, metric), a, b)
        out.append(dict(n=n, M=M, nq=nq, codes=codes, luts=luts, oc=oc, ol=ol, ref=oracle.scan(oc, ol)))
    return out


@pytest.fixture(scope="module")
def small_data(torch_cuda):
    return small_batch(torch_cuda, SMALL_SPECS)


def fresh(torch, batch):
    """The collections with new sums matrices (filled with 0xBEEF)."""
    return [dict(c, sums=u16(torch, (c["nq"], bolt.sums_ld(c["n"])), 0xBEEF)) for c in batch]


def entries(batch):
    return [(c["codes"], c["n"], c["M"], c["luts"], c["sums"]) for c in batch]


def check_small(batch):
    for c in batch:
        n, M = c["n"], c["M"]
        np.testing.assert_array_equal(decode_rows(c["codes"].cpu().numpy(), np.arange(n), M), c["oc"])
        np.testing.assert_array_equal(c["luts"].cpu().numpy(), c["ol"])
        np.testing.assert_array_equal(c["sums"][:, :n].cpu().numpy(), c["ref"])


def test_batched_small_bitexact(torch_cuda, small_data):
    """Ten mixed collections (N up to 3e4, every (J, M) kind), default
    tiles: codes, tables and every sum against the oracle."""
    torch = torch_cuda
    batch = fresh(torch, small_data)
    plan = bolt.BatchPlan(entries(batch))
    plan.run()
    torch.cuda.synchronize()
    check_small(batch)


@pytest.mark.parametrize("qt,upw", [(1, 1), (2, 3), (4, 8), (16, 1), (16, 64)])
def test_batched_tiles_change_no_result(torch_cuda, small_data, qt, upw):
    """Every tile choice gives the same sums (the autotuner's knobs change
    speed only)."""
    torch = torch_cuda
    batch = fresh(torch, small_data[:5])
    plan = bolt.BatchPlan(entries(batch), tuning=[(qt, upw)] * len(batch))
    plan.run()
    torch.cuda.synchronize()
    check_small(batch)


def test_batched_autotune_and_graph(torch_cuda, small_data):
    """Autotuned plan captured in a CUDA graph: replays give the oracle's
    sums."""
    torch = torch_cuda
    batch = fresh(torch, small_data[:6])
    plan = bolt.BatchPlan(entries(batch))
    ms = plan.autotune()
    assert ms > 0
    for qt, upw in plan.tuning():
        assert qt in (4, 8, 16) and upw in (1, 2, 4, 8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.run(stream=s)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    for _ in range(2):
        for c in batch:
            c["sums"].view(torch.int16).fill_(0)
        g.replay()
        torch.cuda.synchronize()
        check_small(batch)


def test_batched_edge_cases(torch_cuda):
    """Empty collections, one vector, odd codebook counts (M = 1, 3, 5), the
    largest M (tiles shrink to fit the staged tables), many queries, wide
    row strides, and sums packed at offsets inside one buffer."""
    torch = torch_cuda
    rng = np.random.default_rng(17)
    shapes = [(0, 8, 5), (100, 8, 0), (1, 16, 3), (257, 1, 7), (1000, 3, 33), (5000, 5, 17), (700, 256, 9),
              (3000, 64, 300), (256, 32, 1), (70_001, 16, 2)]
    specs = []
    total = 0
    for n, M, nq in shapes:
        ld = bolt.sums_ld(n) + (24 if n % 3 == 0 else 0)
        specs.append((n, M, nq, ld, total))
        total += nq * ld + 8  # next matrix starts 16 bytes further on
    big = u16(torch, (total,), 0x1234)
    ents, refs = [], []
    for n, M, nq, ld, off in specs:
        codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
        luts = rng.integers(0, 256, (nq, M, 16)).astype(np.uint8)
        blocked = bolt.pack_codes(dev(torch, codes)) if n else torch.zeros(16, dtype=torch.uint8, device="cuda")
        sums = big[off:off + nq * ld].view(nq, ld) if nq else big[off:off + 8].view(1, 8)[:0]
        ents.append((blocked, n, M, dev(torch, luts), sums))
        refs.append(oracle.scan(codes, luts) if n and nq else None)
    plan = bolt.BatchPlan(ents)
    plan.run()
    torch.cuda.synchronize()
    host = big.cpu().numpy()
    for (n, M, nq, ld, off), ref in zip(specs, refs):
        if ref is None:
            continue
        got = host[off:off + nq * ld].reshape(nq, ld)[:, :n]
        np.testing.assert_array_equal(got, ref)
    # the 8 entries between matrices are never written
    for n, M, nq, ld, off in specs:
        np.testing.assert_array_equal(host[off + nq * ld:off + nq * ld + 8], 0x1234)


def test_batched_uint32_sums_large_M(torch_cuda):
    """Collections with uint32 sums in the same plan as uint16 ones: M above
    256 (300, 1030: tables staged; 2048: tables read from global memory, too
    large to stage), ragged n, 1..5 queries, and a uint32 collection with
    M = 16; every sum against the oracle's uint32 scan.  The uint16
    collections' results are unchanged by the wide tasks beside them, and a
    tuned plan gives the same sums."""
    torch = torch_cuda
    rng = np.random.default_rng(23)
    shapes = [(5_003, 300, 3, True), (2_049, 1030, 2, True), (777, 2048, 5, True), (10_007, 16, 4, True),
              (20_001, 16, 7, False), (3_001, 8, 33, False)]
    ents, refs, outs = [], [], []
    for n, M, nq, wide in shapes:
        codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
        luts = rng.integers(0, 256, (nq, M, 16)).astype(np.uint8)
        ld = bolt.sums_ld(n)
        if wide:
            sums = torch.full((nq, ld), -1, dtype=torch.int32, device="cuda")
            refs.append(oracle.scan_u32(codes, luts).astype(np.uint32))
        else:
            sums = u16(torch, (nq, ld), 0xBEEF)
            refs.append(oracle.scan(codes, luts))
        ents.append((bolt.pack_codes(dev(torch, codes)), n, M, dev(torch, luts), sums))
        outs.append((sums, n, wide))

    def check():
        for (sums, n, wide), ref in zip(outs, refs):
            got = sums[:, :n].cpu().numpy()
            np.testing.assert_array_equal(got.view(np.uint32) if wide else got, ref)

    plan = bolt.BatchPlan(ents)
    plan.run()
    torch.cuda.synchronize()
    check()
    for sums, n, wide in outs:
        sums.fill_(0)
    plan.autotune()
    plan.run()
    torch.cuda.synchronize()
    check()


def test_batched_invalid_arguments(torch_cuda):
    torch = torch_cuda
    codes = torch.zeros(bolt.codes_bytes(100, 8), dtype=torch.uint8, device="cuda")
    luts = torch.zeros((2, 8, 16), dtype=torch.uint8, device="cuda")
    sums = u16(torch, (2, 104))
    with pytest.raises(bolt.BoltError):
        bolt.BatchPlan([(codes, 100, 8, luts, u16(torch, (2, 100)))])  # ld 100 is not a multiple of 8
    with pytest.raises(bolt.BoltError):
        bolt.BatchPlan([(codes, 100, 8, luts, sums)], tuning=[(3, 1)])  # qt_max 3
    with pytest.raises(bolt.BoltError):
        bolt.BatchPlan([(codes[1:], 100, 8, luts, sums)])  # misaligned codes
    big = torch.zeros(bolt.codes_bytes(100, 300), dtype=torch.uint8, device="cuda")
    bl = torch.zeros((2, 300, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(bolt.BoltError):
        bolt.BatchPlan([(big, 100, 300, bl, sums)])  # M > 256 needs uint32 sums


# ------------------------------------------------------------------ full size
def test_batched_64_collections_full_size(torch_cuda):
    """The full 64-collection batch (N up to 2e6, 1..256 queries each; about
    13.7M vectors, 1.4e9 distances, 3.6e10 table lookups) in one launch with
    autotuned tiles: on every collection, the codes of 40 seeded sample rows
    (plus the first and last) and their sums for every query match the
    oracle."""
    torch = torch_cuda
    specs = synth.collections(seed=3)
    rng = np.random.default_rng(23)
    batch = []
    for ci, sp in enumerate(specs):
        n, J, M, nq = sp["n"], sp["J"], sp["M"], sp["nq"]
        metric = ci % 2
        X = synth.mixture_torch(n, J, sp["data_seed"])
        Q = synth.mixture(nq, J, sp["query_seed"])
        nf = min(n, 4000)
        Xfit = X[:nf].cpu().numpy()
        Qtr = X[torch.from_numpy(synth.train_query_rows(n, sp["data_seed"])).cuda()].cpu().numpy()
        Co, a, b = oracle_params(Xfit, Qtr, M, sp["data_seed"], metric)
        Cd = dev(torch, Co)
        codes = bolt.encode(X, Cd)
        luts = bolt.build_luts(dev(torch, Q), Cd, metric, a, b)
        rows = np.unique(np.concatenate([rng.choice(n, 40, replace=False), [0, n - 1]]))
        Xs = X[torch.from_numpy(rows).cuda()].cpu().numpy()
        del X
        oc = oracle.encode(Xs, Co)
        ol = oracle.quantize(oracle.lut_f32(Q, Co, metric), a, b)
        sums = u16(torch, (nq, bolt.sums_ld(n)))
        batch.append(dict(n=n, M=M, codes=codes, luts=luts, sums=sums, rows=rows, oc=oc, ol=ol))
    plan = bolt.BatchPlan(entries(batch))
    plan.autotune()
    for c in batch:
        c["sums"].view(torch.int16).fill_(0)
    plan.run()
    torch.cuda.synchronize()
    for c in batch:
        np.testing.assert_array_equal(decode_rows(c["codes"].cpu().numpy(), c["rows"], c["M"]), c["oc"])
        np.testing.assert_array_equal(c["luts"].cpu().numpy(), c["ol"])
        got = c["sums"].view(torch.int16)[:, torch.from_numpy(c["rows"]).cuda()].cpu().numpy().view(np.uint16)
        np.testing.assert_array_equal(got, oracle.scan(c["oc"], c["ol"]))
