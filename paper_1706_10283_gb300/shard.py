"""Sharded search: one database split into contiguous row ranges.

Every approximate distance depends on one vector's codes only (Sec. 3.1), so
a database can be split by rows across GPUs (or across logical shards on one
GPU) with the codebooks and query tables replicated.  Each shard computes
its own exact top-k; the only exchange is k (sum, index) pairs per query and
shard, and ``bolt_topk_merge`` turns the shard lists into the top-k of the
whole database, bit-identical to the unsharded result.

Shard boundaries are multiples of the 256-vector code block, so a shard's
codes are a contiguous byte range of the whole database's blocked codes.
"""
from . import bolt


def shard_bounds(n, nshard):
    """Row ranges [(lo, hi), ...] of nshard shards covering [0, n): block
    aligned, as even as the 256-vector blocks allow (trailing shards may be
    empty when n has fewer blocks than shards)."""
    nb = (n + bolt.BLOCK - 1) // bolt.BLOCK
    out = []
    for s in range(nshard):
        b0 = nb * s // nshard
        b1 = nb * (s + 1) // nshard
        out.append((min(n, b0 * bolt.BLOCK), min(n, b1 * bolt.BLOCK)))
    return out


def shard_codes(codes, M, lo, hi):
    """The blocked codes of rows [lo, hi) (lo block aligned): a view."""
    row = M * 128
    b0 = lo // bolt.BLOCK
    return codes[b0 * row:b0 * row + bolt.codes_bytes(hi - lo, M)]


def sharded_topk(codes, n, M, luts, k, metric, nshard, stream=None):
    """Top-k over `nshard` logical shards of one database on this GPU: one
    bolt_topk per shard, then bolt_topk_merge.  Returns (sums, idx) (nq, k),
    identical to bolt.topk over the whole database."""
    import torch

    nq = luts.shape[0]
    dev = luts.device
    bounds = [b for b in shard_bounds(n, nshard) if b[1] > b[0]]
    sums = torch.empty((len(bounds), nq, k), dtype=torch.uint16, device=dev)
    idx = torch.empty((len(bounds), nq, k), dtype=torch.int64, device=dev)
    for s, (lo, hi) in enumerate(bounds):
        bolt.topk(shard_codes(codes, M, lo, hi), hi - lo, M, luts, k, metric, out_sums=sums[s], out_idx=idx[s],
                  stream=stream)
    offsets = torch.tensor([lo for lo, _ in bounds], dtype=torch.int64, device=dev)
    return bolt.topk_merge(sums, idx, offsets, M, metric, stream=stream)


def gather_lists(sums, idx, offset, group=None):
    """Exchange step across ranks (torch.distributed, any backend): every
    rank contributes its shard's top-k lists (sums (nq, k) uint16, local idx
    (nq, k) int64) and its global row offset; returns (sums (world, nq, k)
    uint16, idx (world, nq, k) int64, offsets (world,) int64) on every rank,
    in rank order, on the tensors' device."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    # collectives move int32 (no 16-bit integer type in every backend); the
    # int16 view and the narrowing cast back are bit-preserving
    s32 = sums.view(torch.int16).to(torch.int32)
    all_s = [torch.empty_like(s32) for _ in range(world)]
    all_i = [torch.empty_like(idx) for _ in range(world)]
    off = torch.tensor([offset], dtype=torch.int64, device=idx.device)
    all_o = [torch.empty_like(off) for _ in range(world)]
    dist.all_gather(all_s, s32, group=group)
    dist.all_gather(all_i, idx, group=group)
    dist.all_gather(all_o, off, group=group)
    return torch.stack(all_s).to(torch.int16).view(torch.uint16), torch.stack(all_i), torch.cat(all_o)
