"""Serving loop on the GPU: every request's results are the same when it is
served in the mix (continuous batching over several streams, requests
arriving while others run, a tight HBM budget) as when it runs alone, and
match the oracle.  Search results (indices, dequantized distances) and
matmul outputs are compared bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1706_10283_gb300 import bolt, serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bolt.lib()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def world(torch_cuda):
    """Two search collections and one matmul operand, with oracle-fitted
    parameters shared by both sides, plus oracle codes."""
    torch = torch_cuda
    out = {}
    for name, (n, J, M, seed) in {"db": (60_000, 64, 16, 31), "db2": (9_001, 32, 8, 32),
                                  "B": (5_000, 128, 32, 33)}.items():
        X = synth.mixture(n, J, seed)
        Co = oracle.kmeans(X[:4000], M, 4, synth.kmeans_init_rows(4000, seed))
        Qtr = X[synth.train_query_rows(n, seed)]
        quant = {}
        for m in (bolt.METRIC_L2, bolt.METRIC_DOT):
            a, b, _, _ = oracle.fit_quant(oracle.lut_f32(Qtr, Co, m))
            quant[m] = (a, b)
        Cd = dev(torch, Co)
        out[name] = dict(n=n, J=J, M=M, Co=Co, Cd=Cd, quant=quant, codes=bolt.encode(dev(torch, X), Cd),
                         oc=oracle.encode(X, Co))
    return out


def make_server(torch, world, budget, slots, max_queries=512):
    srv = serve.Server(budget, slots=slots, policy=serve.BatchPolicy(max_queries=max_queries))
    for name, w in world.items():
        srv.add_collection(name, w["codes"], w["n"], w["M"], w["Cd"], w["quant"])
    return srv


def make_trace(seed, count, rate):
    tr = synth.poisson_trace(seed, count, rate, 64, max_q=200, matmul_frac=0.1, J_mm=128, max_rows=40)
    reqs = []
    for i, r in enumerate(tr):
        if r["kind"] == "matmul":
            coll = "B"
        else:
            coll = "db" if i % 3 else "db2"
            if coll == "db2":
                r["Q"] = np.ascontiguousarray(r["Q"][:, :32])
        reqs.append(serve.Request(i, coll, r["Q"], kind=r["kind"], metric=r["metric"], k=r["k"],
                                  t_arrival=r["t_arrival"]))
    return reqs


def alone(torch, world, r):
    """The request by itself, through the library entry points."""
    w = world[r.collection]
    Qd = dev(torch, r.Q)
    if r.kind == serve.MATMUL:
        a, b = w["quant"][bolt.METRIC_DOT]
        return bolt.approx_matmul(Qd, w["codes"], w["n"], w["Cd"], a, b).cpu().numpy()
    a, b = w["quant"][r.metric]
    luts = bolt.build_luts(Qd, w["Cd"], r.metric, a, b)
    s, i = bolt.topk(w["codes"], w["n"], w["M"], luts, r.k, r.metric)
    return i.cpu().numpy(), bolt.dequantize(s, a, b).cpu().numpy()


def check_same(torch, world, done):
    for r in done:
        ref = alone(torch, world, r)
        if r.kind == serve.MATMUL:
            np.testing.assert_array_equal(r.out, ref)
        else:
            np.testing.assert_array_equal(r.idx, ref[0])
            np.testing.assert_array_equal(r.dist, ref[1])


def test_mixed_trace_same_as_alone(torch_cuda, world):
    """120 Poisson requests (1..200 queries, L2 and dot, k 10..100, 10%
    matmul) through 3 slots: batching happens (fewer batches than
    requests), and every result equals the request served alone."""
    torch = torch_cuda
    srv = make_server(torch, world, budget=2 << 30, slots=3)
    reqs = make_trace(5, 120, rate=2000.0)
    done = serve.run_trace(srv, reqs)
    assert len(done) == len(reqs) and srv.idle()
    assert srv.batches < len(reqs)
    assert max(np.bincount([r.batch_id for r in done])) > 1
    assert srv.budget.used == sum(c.nbytes for c in srv.collections.values())
    check_same(torch, world, done)


def test_tight_budget_serializes_but_results_hold(torch_cuda, world):
    """A budget that fits the collections and about one batch: requests wait
    for memory, the books never exceed the budget, results are unchanged."""
    torch = torch_cuda
    resident = sum(serve.Collection(nm, w["codes"], w["n"], w["M"], w["Cd"], w["quant"]).nbytes
                   for nm, w in world.items())
    reqs = make_trace(6, 60, rate=5000.0)
    probe = make_server(torch, world, budget=2 << 30, slots=1)
    largest = max(serve.batch_bytes(probe.collections[r.collection], r.kind, r.nq, r.k) for r in reqs)
    budget = resident + largest + (1 << 20)
    srv = make_server(torch, world, budget=budget, slots=4)
    done = serve.run_trace(srv, reqs)
    assert len(done) == len(reqs)
    assert srv.budget.peak <= budget
    check_same(torch, world, done)


def test_served_search_matches_oracle(torch_cuda, world):
    torch = torch_cuda
    srv = make_server(torch, world, budget=2 << 30, slots=2)
    reqs = [r for r in make_trace(7, 40, rate=1e4) if r.kind == serve.SEARCH][:12]
    done = serve.run_trace(srv, reqs)
    for r in done:
        w = world[r.collection]
        a, b = w["quant"][r.metric]
        ol = oracle.quantize(oracle.lut_f32(r.Q, w["Co"], r.metric), a, b)
        rs, ri = oracle.topk(oracle.scan(w["oc"], ol), r.k, r.metric)
        np.testing.assert_array_equal(r.idx, ri)
        np.testing.assert_array_equal(r.dist, oracle.dequant(rs, a, b))


def test_admission_by_budget(torch_cuda, world):
    torch = torch_cuda
    w = world["db"]
    small = serve.Collection("db", w["codes"], w["n"], w["M"], w["Cd"], w["quant"]).nbytes
    srv = serve.Server(small + 1000, slots=1)
    srv.add_collection("db", w["codes"], w["n"], w["M"], w["Cd"], w["quant"])
    with pytest.raises(serve.AdmissionError):
        srv.add_collection("db2", world["db2"]["codes"], world["db2"]["n"], world["db2"]["M"], world["db2"]["Cd"],
                           world["db2"]["quant"])
    with pytest.raises(serve.AdmissionError):  # its working memory can never fit
        srv.submit(serve.Request(0, "db", np.zeros((100, 64), np.float32), k=10))
    srv.remove_collection("db")
    assert srv.budget.used == 0
