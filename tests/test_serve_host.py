"""Host logic of the serving loop (no GPU): the batching policy, the HBM
budget's books, and the seeded Poisson trace."""
from collections import deque

import numpy as np
import pytest

from paper_1706_10283_gb300 import synth
from paper_1706_10283_gb300.serve import MATMUL, SEARCH, BatchPolicy, Budget, Request


def req(rid, nq, coll="a", kind=SEARCH, metric=0, k=10):
    return Request(rid, coll, np.zeros((nq, 4), np.float32), kind=kind, metric=metric, k=k)


def test_policy_groups_same_collection_kind_metric_in_order():
    q = deque([req(0, 10), req(1, 5, metric=1), req(2, 7), req(3, 3, coll="b"), req(4, 1)])
    b = BatchPolicy(max_queries=512).take(q)
    assert [r.rid for r in b] == [0, 2, 4]
    assert [r.rid for r in q] == [1, 3]  # the rest keep their order


def test_policy_respects_query_cap_and_lookahead():
    q = deque([req(0, 300), req(1, 300), req(2, 200), req(3, 12)])
    b = BatchPolicy(max_queries=512).take(q)
    assert [r.rid for r in b] == [0, 2, 3]  # 300 + 200 + 12 = 512
    assert [r.rid for r in q] == [1]
    q = deque([req(i, 1) for i in range(10)])
    b = BatchPolicy(max_queries=512, lookahead=3).take(q)
    assert [r.rid for r in b] == [0, 1, 2, 3]
    assert [r.rid for r in q] == [4, 5, 6, 7, 8, 9]


def test_policy_matmul_and_oversized_run_alone():
    q = deque([req(0, 4, kind=MATMUL), req(1, 4, kind=MATMUL)])
    assert [r.rid for r in BatchPolicy().take(q)] == [0]
    q = deque([req(0, 600), req(1, 1)])
    assert [r.rid for r in BatchPolicy(max_queries=512).take(q)] == [0]
    assert BatchPolicy().take(deque()) == []


def test_budget_books():
    b = Budget(100)
    assert b.reserve(60) and not b.reserve(41) and b.reserve(40)
    assert b.used == 100 and b.peak == 100
    b.release(60)
    assert b.used == 40 and b.peak == 100
    with pytest.raises(AssertionError):
        b.release(41)


def test_poisson_trace_is_seeded_and_in_range():
    a = synth.poisson_trace(3, 400, 50.0, 16, max_q=512, k_lo=10, k_hi=100, matmul_frac=0.2, J_mm=8)
    b = synth.poisson_trace(3, 400, 50.0, 16, max_q=512, k_lo=10, k_hi=100, matmul_frac=0.2, J_mm=8)
    assert [r["nq"] for r in a] == [r["nq"] for r in b]
    assert all(np.array_equal(x["Q"], y["Q"]) for x, y in zip(a, b))
    t = np.array([r["t_arrival"] for r in a])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.2 / 50.0  # mean inter-arrival 1/rate
    assert all(1 <= r["nq"] <= 512 and 10 <= r["k"] <= 100 and r["metric"] in (0, 1) for r in a)
    mm = [r for r in a if r["kind"] == "matmul"]
    assert 40 <= len(mm) <= 120 and all(r["Q"].shape[1] == 8 for r in mm)
    assert all(r["Q"].shape == (r["nq"], 16) for r in a if r["kind"] == "search")


def test_check_topk_flags_timed_out_rows():
    from paper_1706_10283_gb300 import bolt

    ok = np.array([[3, 1, 2], [0, 5, -1]], np.int64)  # -1 is padding (k > n), not a failure
    bolt.check_topk(ok)
    bad = ok.copy()
    bad[1] = -2
    with pytest.raises(bolt.BoltError) as e:
        bolt.check_topk(bad)
    assert e.value.code == bolt.ETIMEOUT


def test_retire_fails_a_request_whose_rows_timed_out():
    """A batch whose second request's rows came back as -2 (a bounded device
    wait gave up): that request is failed with ETIMEOUT and carries no
    results; the first request of the same batch is returned normally."""
    from types import SimpleNamespace

    import torch

    from paper_1706_10283_gb300 import bolt
    from paper_1706_10283_gb300.serve import Server

    r0, r1 = req(0, 2, k=3), req(1, 1, k=3)
    idx = torch.tensor([[4, 5, 6], [7, 8, 9], [-2, -2, -2]], dtype=torch.int64)
    dist = torch.arange(9, dtype=torch.float32).reshape(3, 3)
    srv = Server.__new__(Server)
    srv.budget = Budget(100)
    assert srv.budget.reserve(10)
    slot = SimpleNamespace(busy=True, event=SimpleNamespace(query=lambda: True), reqs=[(r0, 0), (r1, 2)],
                           host_view=(idx, dist), nbytes=10, keep=None)
    srv.slots = [slot]
    done = srv._retire()
    assert [r.rid for r in done] == [0, 1]
    assert r0.error is None and r0.idx.tolist() == [[4, 5, 6], [7, 8, 9]]
    assert isinstance(r1.error, bolt.BoltError) and r1.error.code == bolt.ETIMEOUT
    assert r1.idx is None and r1.dist is None
    assert srv.budget.used == 0 and not slot.busy
