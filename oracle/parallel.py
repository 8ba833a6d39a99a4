"""Multithreaded driver of the oracle's scan + top-k -- TEST INFRASTRUCTURE
ONLY (the timed CPU baseline of bench.py).

The database's rows are split into contiguous ranges, one per host thread;
each thread runs the oracle's own ``scan`` and ``topk`` on its range (the C
calls release the GIL, so the threads run in parallel), and the per-range
lists are reduced by ``topk`` over their concatenation.  The result equals
``topk(scan(codes, luts), k, metric)`` on the whole database: a vector's sum
depends on its own codes only (Sec. 3.1), every vector of the global top k is
in its range's top k, and the concatenation keeps ranges in row order, so
ties still go to the lower index.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import scan, topk


def host_threads():
    """Threads the CPU baseline may use: this process's CPU affinity."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - non-Linux
        return os.cpu_count() or 1


def scan_topk(codes, luts, k, metric, threads=None):
    """(sums (nq, k) uint16, idx (nq, k) int64) of the oracle's top-k over
    row-major codes (n, M) for tables luts (nq, M, 16)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    n = codes.shape[0]
    # every range holds at least k rows, so no per-range list is padded
    threads = max(1, min(int(threads or host_threads()), n // max(4096, k)))
    if threads == 1:
        return topk(scan(codes, luts), k, metric)
    bounds = [n * t // threads for t in range(threads + 1)]

    def one(t):
        lo, hi = bounds[t], bounds[t + 1]
        s, i = topk(scan(codes[lo:hi], luts), k, metric)
        return s, i + lo

    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(one, range(threads)))
    cs = np.concatenate([p[0] for p in parts], axis=1)
    ci = np.concatenate([p[1] for p in parts], axis=1)
    rs, pos = topk(cs, k, metric)
    return rs, np.take_along_axis(ci, pos, axis=1)


def encode(X, C, threads=None, chunk=65536):
    """The oracle's fp32 encoder on row chunks in host threads (the same
    per-row arithmetic, so the codes equal ``oracle.encode(X, C)``)."""
    from . import encode as encode_rows

    X = np.ascontiguousarray(X, dtype=np.float32)
    n = X.shape[0]
    starts = list(range(0, n, chunk))
    threads = max(1, min(int(threads or host_threads()), len(starts)))
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda lo: encode_rows(X[lo:lo + chunk], C), starts))
    return np.concatenate(parts, axis=0) if parts else np.empty((0, C.shape[0]), np.uint8)
