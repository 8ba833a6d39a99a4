"""The multi-rank exchange on CPU: world_size-2 gloo ranks each hold one
shard of a database (oracle top-k on its own rows), exchange their lists
with shard.gather_lists, and the union's best k (merged here by sorting the
keys) is the oracle top-k of the whole database."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import oracle
from paper_1706_10283_gb300 import shard

N, M, NQ, K = 3000, 8, 3, 25


def _problem():
    rng = np.random.default_rng(9)
    codes = rng.integers(0, 16, (N, M)).astype(np.uint8)
    luts = rng.integers(0, 4, (NQ, M, 16)).astype(np.uint8)  # many ties
    return codes, luts


def _merge(sums, idx, offsets, metric):
    """Test-side merge of gathered lists: sort all keys (s', global index)."""
    world, nq, k = idx.shape
    out_s = np.zeros((nq, k), np.uint16)
    out_i = np.full((nq, k), -1, np.int64)
    for q in range(nq):
        keys = []
        for r in range(world):
            for p in range(k):
                if idx[r, q, p] >= 0:
                    S = int(sums[r, q, p])
                    keys.append((S if metric == 0 else 255 * M - S, int(offsets[r] + idx[r, q, p]), S))
        keys.sort()
        for j, (_, gi, S) in enumerate(keys[:k]):
            out_s[q, j], out_i[q, j] = S, gi
    return out_s, out_i


def _rank(rank, world, port, metric, result):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    codes, luts = _problem()
    lo, hi = shard.shard_bounds(N, world)[rank]
    s, i = oracle.topk(oracle.scan(codes[lo:hi], luts), K, metric)
    S, I, O = shard.gather_lists(torch.from_numpy(s.view(np.int16)).view(torch.uint16), torch.from_numpy(i), lo)
    if rank == 0:
        result["sums"] = S.view(torch.int16).numpy().view(np.uint16).copy()
        result["idx"] = I.numpy().copy()
        result["offsets"] = O.numpy().copy()
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_exchange_matches_unsharded():
    ctx = mp.get_context("spawn")
    for metric in (0, 1):
        with ctx.Manager() as mgr:
            result = mgr.dict()
            port = _free_port()
            procs = [ctx.Process(target=_rank, args=(r, 2, port, metric, result)) for r in range(2)]
            for p in procs:
                p.start()
            for p in procs:
                p.join(120)
                assert p.exitcode == 0
            S, I, O = result["sums"], result["idx"], result["offsets"]
        codes, luts = _problem()
        assert list(O) == [lo for lo, _ in shard.shard_bounds(N, 2)]
        ms, mi = _merge(S, I, O, metric)
        rs, ri = oracle.topk(oracle.scan(codes, luts), K, metric)
        np.testing.assert_array_equal(mi, ri)
        np.testing.assert_array_equal(ms, rs)


def test_shard_bounds_are_block_aligned_and_cover():
    for n, s in ((1, 1), (1000, 3), (256 * 7 + 5, 4), (100, 8), (10**6, 7)):
        b = shard.shard_bounds(n, s)
        assert len(b) == s and b[0][0] == 0 and b[-1][1] == n
        for (lo, hi), (lo2, _) in zip(b, b[1:]):
            assert hi == lo2 and lo % 256 == 0 and lo <= hi
