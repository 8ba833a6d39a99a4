"""The benchmark's timed steps, built exactly as bench.py builds them
(pipeline.SearchStep: one query per launch round-robin on several streams
with one workspace per stream, the step captured in CUDA graphs and
replayed), checked against the oracle on every query after several
replays, and through run_from_host (pinned host buffers in and out).

Two configurations: the shared-memory size class on a mixture database
with 8 streams (the 1,000,000-vector step's form, at 262,147 vectors), and
the 50,000,000-vector resident database with a 1,000,064-row insert batch
encoded into its last rows each step, on 4 streams (the headline step).
"""
import numpy as np
import pytest

import oracle
from oracle import parallel
from paper_1706_10283_gb300 import bolt, synth
from paper_1706_10283_gb300.pipeline import SearchStep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bolt.lib()
    return torch


def oracle_results(codes, Q, C, quant, k, metrics):
    """Per metric: oracle tables, then the top-k sums, indices and
    dequantized values of every query (threaded oracle driver)."""
    out = {}
    for m in metrics:
        a, b = quant[m]
        ol = oracle.quantize(oracle.lut_f32(Q, C, m), a, b)
        rs = np.empty((len(Q), k), np.uint16)
        ri = np.empty((len(Q), k), np.int64)
        for qi in range(len(Q)):
            s_, i_ = parallel.scan_topk(codes, ol[qi:qi + 1], k, m)
            rs[qi], ri[qi] = s_[0], i_[0]
        out[m] = (ol, rs, ri, oracle.dequant(rs, a, b))
    return out


def check_step(torch, step, want):
    for m, (ol, rs, ri, rd) in want.items():
        np.testing.assert_array_equal(step.luts[m].cpu().numpy(), ol)
        np.testing.assert_array_equal(step.idx[m].cpu().numpy(), ri)
        np.testing.assert_array_equal(step.sums[m].cpu().numpy(), rs)
        np.testing.assert_array_equal(step.dist[m].cpu().numpy(), rd)


def test_search_step_eight_streams_graph_replay(torch_cuda):
    torch = torch_cuda
    n, J, M, nq, k = 262_147, 128, 16, 96, 100
    X = synth.mixture(n, J, 0)
    Q = synth.mixture(nq, J, 1)
    C = oracle.kmeans(X[:20_000], M, 4, synth.kmeans_init_rows(20_000, 0))
    Qtr = X[synth.train_query_rows(n, 0)]
    quant = {}
    for m in (oracle.METRIC_L2, oracle.METRIC_DOT):
        a, b, _, _ = oracle.fit_quant(oracle.lut_f32(Qtr, C, m))
        quant[m] = (a, b)
    step = SearchStep(n, J, M, nq, k, torch.from_numpy(C).cuda(), quant, streams=8)
    step.set_inputs(torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda())
    step.capture()
    for _ in range(3):
        step.replay(timed=True)
    torch.cuda.synchronize()
    oc = parallel.encode(X, C)
    np.testing.assert_array_equal(bolt.unpack_codes(step.codes, n, M).cpu().numpy(), oc)
    want = oracle_results(oc, Q, C, quant, k, step.metrics)
    check_step(torch, step, want)
    # end to end from pinned host buffers
    oi = [torch.full((nq, k), -7, dtype=torch.int64).pin_memory() for _ in step.metrics]
    od = [torch.zeros((nq, k), dtype=torch.float32).pin_memory() for _ in step.metrics]
    step.run_from_host(torch.from_numpy(X).pin_memory(), torch.from_numpy(Q).pin_memory(), oi, od)
    torch.cuda.synchronize()
    for j, m in enumerate(step.metrics):
        np.testing.assert_array_equal(oi[j].numpy(), want[m][2])
        np.testing.assert_array_equal(od[j].numpy(), want[m][3])


def clustered_codes(n, M, seed, clusters=256, chunk=5_000_000):
    """Codes with the structure of an encoded mixture (see test_gpu_parity)."""
    rng = np.random.default_rng(seed)
    pref = rng.integers(0, 16, (clusters, M), dtype=np.uint8)
    out = np.empty((n, M), np.uint8)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        g = rng.integers(0, clusters, hi - lo)
        r = rng.integers(0, 32, (hi - lo, M), dtype=np.uint8)
        out[lo:hi] = np.where(r < 16, r, pref[g])
    return out


def test_search_step_50m_insert_four_streams(torch_cuda):
    """The headline step at full size: 50,000,000 resident codes, the insert
    batch of 1,000,064 mixture rows encoded into rows 48,999,936 .. 50M each
    step, L2 and dot tables, one-query top-100 launches round-robin on 4
    streams, dequantize; 3 graph replays, then every query against the
    oracle over the whole database (its last rows re-encoded by the oracle),
    then two end-to-end steps from pinned host buffers back to back (the
    second step's upload overlaps the first step's searches)."""
    torch = torch_cuda
    cfg = synth.CONFIGS["serve_50m"]
    n, J, M, k, nq = cfg["n"], cfg["J"], cfg["M"], 100, 6
    nx = 1_000_064
    row0 = n - nx
    codes = clustered_codes(n, M, 50)
    Xf = synth.mixture(20_000, J, 51)
    C = oracle.kmeans(Xf, M, 4, synth.kmeans_init_rows(20_000, 51))
    quant = {}
    for m in (oracle.METRIC_L2, oracle.METRIC_DOT):
        a, b, _, _ = oracle.fit_quant(oracle.lut_f32(Xf[:2000], C, m))
        quant[m] = (a, b)
    Xins = synth.mixture(nx, J, 52)
    Q = synth.mixture(nq, J, 53)
    dcodes = bolt.pack_codes(torch.from_numpy(codes).cuda())
    step = SearchStep(n, J, M, nq, k, torch.from_numpy(C).cuda(), quant, streams=4, codes=dcodes,
                      insert_row0=row0, insert_rows=nx)
    step.set_inputs(torch.from_numpy(Xins).cuda(), torch.from_numpy(Q).cuda())
    step.capture()
    for _ in range(3):
        step.replay(timed=True)
    torch.cuda.synchronize()
    codes[row0:] = parallel.encode(Xins, C)
    got = bolt.unpack_codes(dcodes, n, M)
    np.testing.assert_array_equal(got[row0 - 1000:].cpu().numpy(), codes[row0 - 1000:])  # insert + neighbours
    del got
    want = oracle_results(codes, Q, C, quant, k, step.metrics)
    check_step(torch, step, want)
    oi = [torch.full((nq, k), -7, dtype=torch.int64).pin_memory() for _ in step.metrics]
    od = [torch.zeros((nq, k), dtype=torch.float32).pin_memory() for _ in step.metrics]
    # a first step from other inputs, then the checked one: its upload may
    # start while the first step's searches run, never before its encode
    Xh, Qh = torch.from_numpy(Xins).pin_memory(), torch.from_numpy(Q).pin_memory()
    Xz, Qz = torch.zeros_like(Xh).pin_memory(), torch.zeros_like(Qh).pin_memory()
    oz = [torch.empty_like(t).pin_memory() for t in oi]
    dz = [torch.empty_like(t).pin_memory() for t in od]
    step.run_from_host(Xz, Qz, oz, dz)
    step.run_from_host(Xh, Qh, oi, od)
    torch.cuda.synchronize()
    for j, m in enumerate(step.metrics):
        np.testing.assert_array_equal(oi[j].numpy(), want[m][2])
        np.testing.assert_array_equal(od[j].numpy(), want[m][3])
