"""Online changes to a resident collection (vectors added, changed and
deleted while it serves, Sec. 1.3): after deletes, inserts that reuse the
deleted rows, appends and in-place updates, every search through the
server equals the oracle's top-k over the live rows with their current
vectors."""
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


def oracle_topk_live(X, live, Co, Q, metric, quant, k):
    """Top-k by (key, row id) over the live rows, from oracle codes."""
    a, b = quant[metric]
    rows = np.nonzero(live)[0]
    codes = oracle.encode(X[rows], Co)
    luts = oracle.quantize(oracle.lut_f32(Q, Co, metric), a, b)
    s, pos = oracle.topk(oracle.scan(codes, luts), k, metric)
    idx = np.where(pos >= 0, rows[np.maximum(pos, 0)], -1)
    return s, idx, a, b


def test_insert_update_delete_then_search(torch_cuda):
    torch = torch_cuda
    n, J, M, cap = 20_000, 64, 16, 26_000
    X = np.zeros((cap, J), np.float32)
    X[:n] = synth.mixture(n, J, 41)
    Co = oracle.kmeans(X[:4000], M, 4, synth.kmeans_init_rows(4000, 41))
    Qtr = X[synth.train_query_rows(n, 41)]
    quant = {m: oracle.fit_quant(oracle.lut_f32(Qtr, Co, m))[:2] for m in (bolt.METRIC_L2, bolt.METRIC_DOT)}
    Cd = dev(torch, Co)
    codes = torch.zeros(bolt.codes_bytes(cap, M), dtype=torch.uint8, device="cuda")
    codes[:bolt.codes_bytes(n, M)] = bolt.encode(dev(torch, X[:n]), Cd)
    srv = serve.Server(1 << 30, slots=2)
    srv.add_collection("db", codes, n, M, Cd, quant, capacity=cap)
    live = np.zeros(cap, bool)
    live[:n] = True
    rng = np.random.default_rng(42)
    dead = rng.choice(n, 300, replace=False)
    srv.delete("db", dead)
    live[dead] = False
    Xn = synth.mixture(500, J, 43)
    ids = srv.insert("db", Xn)
    assert sorted(ids[:300].tolist()) == sorted(dead.tolist()) and ids[300:].tolist() == list(range(n, n + 200))
    X[ids] = Xn
    live[ids] = True
    upd = rng.choice(np.nonzero(live)[0], 100, replace=False)
    Xu = synth.mixture(100, J, 44)
    srv.update("db", upd, Xu)
    X[upd] = Xu
    more_dead = rng.choice(np.nonzero(live)[0], 50, replace=False)
    srv.delete("db", more_dead)
    live[more_dead] = False
    assert srv.collections["db"].n == n + 200 and srv.collections["db"].n_dead == 50
    reqs = []
    for i, (nq, k, metric) in enumerate([(1, 10, 0), (7, 100, 1), (3, 37, 0), (12, 64, 1)]):
        reqs.append(serve.Request(i, "db", synth.mixture(nq, J, 60 + i), metric=metric, k=k))
    done = serve.run_trace(srv, reqs)
    for r in done:
        rs, ri, a, b = oracle_topk_live(X[:n + 200], live[:n + 200], Co, r.Q, r.metric, quant, r.k)
        np.testing.assert_array_equal(r.idx, ri)
        np.testing.assert_array_equal(r.dist, oracle.dequant(rs, a, b))
        assert not np.isin(r.idx, np.nonzero(~live)[0]).any()


def test_write_codes_rejects_bad_rows_and_codes(torch_cuda):
    torch = torch_cuda
    blocked = torch.zeros(bolt.codes_bytes(300, 4), dtype=torch.uint8, device="cuda")
    rc = torch.tensor([[1, 2, 3, 4]], dtype=torch.uint8, device="cuda")
    with pytest.raises(bolt.BoltError):
        bolt.write_codes(rc, torch.tensor([300], dtype=torch.int64, device="cuda"), blocked, 300)
    with pytest.raises(bolt.BoltError):
        bolt.write_codes(rc + 15, torch.tensor([5], dtype=torch.int64, device="cuda"), blocked, 300)
    assert int(blocked.sum()) == 0
    bolt.write_codes(rc, torch.tensor([257], dtype=torch.int64, device="cuda"), blocked, 300)
    np.testing.assert_array_equal(bolt.unpack_codes(blocked, 300, 4).cpu().numpy()[257], [1, 2, 3, 4])


def test_topk_filter_drops_dead_rows(torch_cuda):
    torch = torch_cuda
    idx = torch.tensor([[5, 1, 9, 3, 7], [2, -2, 4, 6, 8]], dtype=torch.int64, device="cuda")
    sums = torch.tensor([[1, 2, 3, 4, 5], [1, 1, 1, 1, 1]], dtype=torch.int16, device="cuda").view(torch.uint16)
    bits = np.zeros(1, np.uint32)
    bits[0] = (1 << 1) | (1 << 9) | (1 << 7)
    dead = torch.from_numpy(bits.view(np.int32)).cuda()
    s, i = bolt.topk_filter(sums, idx, dead, 32, 3)
    assert i.cpu().tolist()[0] == [5, 3, -1] and s.cpu().numpy().tolist()[0] == [1, 4, 0]
    assert i.cpu().tolist()[1] == [-2, -2, -2]
