"""Serving loop over resident encoded databases.

The paper's query phase (Sec. 3.1: encode the query into tables, scan, keep
the best) is run here for a stream of requests that arrive at any time:

* ``search``: nq queries against one collection, L2 or dot, top-k (the
  nearest-neighbour / maximum-inner-product searches of Sec. 4.3), results
  dequantized (Sec. 3.2) and copied to host memory;
* ``matmul``: rows of a matrix A against an encoded matrix B (the
  approximate matrix product of Sec. 4.4), the full rows x n product copied
  to host memory.

Collections (codes, codebooks, quantizers) stay resident on the device.
Admission is by an HBM budget: a collection is admitted only if its bytes
fit, and a batch is dispatched only when its working memory (query tables,
top-k workspace, outputs) fits beside the resident collections and the
batches already in flight.  Batching is continuous: whenever one of
``slots`` CUDA streams is free and memory allows, the oldest waiting request
and the later waiting requests that can share its launches (same
collection, kind and metric) are merged into one batch -- one table build,
one top-k launch, one dequantize -- and enqueued on that stream, so batches
overlap on the device while new requests keep arriving.  Every kernel is a
libbolt.so entry point; this module only moves bytes and keeps books.

A batch's top-k uses the largest k of its requests; each request keeps the
first k of its rows, which is exactly its own top-k (ties are broken by
index, so the first k of a longer exact list are the exact top k).
"""
import time
from collections import deque

import numpy as np

from . import bolt

SEARCH, MATMUL = "search", "matmul"


class AdmissionError(RuntimeError):
    pass


class Budget:
    """Device bytes the server may hold: resident collections plus the working
    memory of batches in flight."""

    def __init__(self, total):
        self.total = int(total)
        self.used = 0
        self.peak = 0

    def reserve(self, nbytes):
        nbytes = int(nbytes)
        if self.used + nbytes > self.total:
            return False
        self.used += nbytes
        self.peak = max(self.peak, self.used)
        return True

    def release(self, nbytes):
        self.used -= int(nbytes)
        assert self.used >= 0


class Request:
    """One client request.  Q: (nq, J) float32 host array (queries, or rows
    of A for matmul).  After completion: ``idx`` (nq, k) int64 and ``dist``
    (nq, k) float32 for search, ``out`` (nq, n) float32 for matmul, and the
    host times ``t_arrival``, ``t_dispatch``, ``t_done`` (seconds).
    ``error`` is None, or the BoltError of a failed request (a search whose
    bounded device wait gave up: its rows would hold index -2); a failed
    request carries no results."""

    __slots__ = ("rid", "collection", "Q", "kind", "metric", "k", "t_arrival", "t_dispatch", "t_done", "idx",
                 "dist", "out", "batch_id", "error")

    def __init__(self, rid, collection, Q, kind=SEARCH, metric=bolt.METRIC_L2, k=10, t_arrival=0.0):
        self.rid = rid
        self.collection = collection
        self.Q = np.ascontiguousarray(Q, dtype=np.float32)
        self.kind = kind
        self.metric = metric
        self.k = int(k)
        self.t_arrival = float(t_arrival)
        self.t_dispatch = self.t_done = None
        self.idx = self.dist = self.out = None
        self.batch_id = None
        self.error = None

    @property
    def nq(self):
        return self.Q.shape[0]

    def key(self):
        return (self.collection, self.kind, self.metric)


class BatchPolicy:
    """Which waiting requests form the next batch (host logic only).

    The oldest waiting request leads.  Requests from the next ``lookahead``
    waiting ones join it, in arrival order, while they have the same
    collection, kind and metric and the batch stays within ``max_queries``
    queries.  A matmul request always runs alone (its output is a full
    rows x n matrix).  A request larger than ``max_queries`` runs alone.
    """

    def __init__(self, max_queries=512, lookahead=32):
        self.max_queries = int(max_queries)
        self.lookahead = int(lookahead)

    def take(self, queue):
        """Remove and return the next batch from ``queue`` (a deque)."""
        if not queue:
            return []
        head = queue.popleft()
        batch = [head]
        if head.kind == MATMUL or head.nq >= self.max_queries:
            return batch
        total = head.nq
        kept = []
        scanned = 0
        while queue and scanned < self.lookahead:
            r = queue.popleft()
            scanned += 1
            if r.key() == head.key() and total + r.nq <= self.max_queries:
                batch.append(r)
                total += r.nq
            else:
                kept.append(r)
        for r in reversed(kept):
            queue.appendleft(r)
        return batch


class Collection:
    """A resident encoded database: codes (blocked, device, room for
    `capacity` vectors), codebooks and per-metric quantizers (a, b).

    Rows [0, n) are in use; deleted rows are marked in a device bitmap
    (`dead`), kept in `free` for reuse by later inserts, and dropped from
    search results (top-(k + n_dead) followed by bolt_topk_filter, exact
    because at most n_dead dead rows can rank above a live one)."""

    def __init__(self, name, codes, n, M, centroids, quant, capacity=None):
        import torch

        self.name = name
        self.codes = codes
        self.n = int(n)
        self.M = int(M)
        self.capacity = int(capacity if capacity is not None else n)
        if codes.numel() < bolt.codes_bytes(self.capacity, self.M):
            raise AdmissionError("collection %r: codes hold fewer than %d vectors" % (name, self.capacity))
        self.C = centroids
        self.J = int(centroids.shape[0] * centroids.shape[2])
        self.quant = {m: (float(a), np.asarray(b, np.float32)) for m, (a, b) in quant.items()}
        self.dead_host = np.zeros((self.capacity + 31) // 32, np.uint32)
        self.dead = torch.zeros(len(self.dead_host), dtype=torch.int32, device=codes.device)
        self.free = []
        self.n_dead = 0
        self.nbytes = int(codes.numel() + centroids.numel() * 4 + self.dead.numel() * 4)

    def is_dead(self, i):
        return bool((self.dead_host[i >> 5] >> np.uint32(i & 31)) & np.uint32(1))

    def _set_dead(self, i, v):
        w, b = i >> 5, np.uint32(1 << (i & 31))
        self.dead_host[w] = (self.dead_host[w] | b) if v else (self.dead_host[w] & ~b)


def batch_bytes(coll, kind, nq, k):
    """Device bytes a batch holds while in flight (upper bound)."""
    q = nq * coll.J * 4
    if kind == MATMUL:
        return q + nq * coll.M * 16 + nq * coll.n * 4
    kr = k + coll.n_dead
    return (q + nq * coll.M * 16 + bolt.topk_workspace_bytes(coll.n, coll.M, nq, kr) + nq * kr * (2 + 8) * 2 +
            nq * k * 4)


class _Slot:
    def __init__(self, torch, device):
        self.stream = torch.cuda.Stream(device=device)
        self.event = torch.cuda.Event()
        self.busy = False
        self.reqs = []
        self.keep = None
        self.nbytes = 0
        self.host = {}
        self.host_view = None

    def pinned(self, torch, name, numel, dtype):
        buf = self.host.get(name)
        if buf is None or buf.numel() < numel:
            buf = torch.empty(max(numel, 1), dtype=dtype).pin_memory()
            self.host[name] = buf
        return buf[:numel]


class Server:
    """Continuous-batching server.  ``poll()`` is non-blocking: it retires
    finished batches and dispatches new ones; call it in the client loop."""

    def __init__(self, budget_bytes, slots=4, policy=None, device="cuda"):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.budget = Budget(budget_bytes)
        self.policy = policy or BatchPolicy()
        self.collections = {}
        self.queue = deque()
        self.slots = [_Slot(torch, self.device) for _ in range(slots)]
        self.batches = 0
        self.launches = 0
        self.resident = 0  # bytes of admitted collections

    # -------------------------------------------------------------- collections
    def add_collection(self, name, codes, n, M, centroids, quant, capacity=None):
        if name in self.collections:
            raise AdmissionError("collection %r already resident" % name)
        c = Collection(name, codes, n, M, centroids, quant, capacity)
        if not self.budget.reserve(c.nbytes):
            raise AdmissionError("collection %r (%d bytes) does not fit the HBM budget (%d of %d bytes used)" %
                                 (name, c.nbytes, self.budget.used, self.budget.total))
        self.collections[name] = c
        self.resident += c.nbytes
        return c

    def remove_collection(self, name):
        if any(s.busy and s.reqs[0][0].collection == name for s in self.slots) or any(
                r.collection == name for r in self.queue):
            raise AdmissionError("collection %r has requests pending" % name)
        c = self.collections.pop(name)
        self.budget.release(c.nbytes)
        self.resident -= c.nbytes

    # -------------------------------------------------------------- online changes
    def _quiesce(self, name):
        """Wait for the batches in flight on collection `name` (their results
        are retired by the next poll)."""
        for s in self.slots:
            if s.busy and s.reqs and s.reqs[0][0].collection == name:
                s.event.synchronize()

    def _encode_rows(self, c, X):
        torch = self.torch
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(self.device)
        if Xd.ndim != 2 or Xd.shape[1] != c.J:
            raise ValueError("vectors must be (count, %d)" % c.J)
        blocked = bolt.encode(Xd, c.C)
        return bolt.unpack_codes(blocked, Xd.shape[0], c.M)

    def insert(self, name, X):
        """Encode vectors X (count, J) and store them, reusing deleted rows
        first; returns their row ids.  Waits for the collection's batches in
        flight."""
        torch = self.torch
        c = self.collections[name]
        count = int(np.asarray(X).shape[0])
        reuse = min(count, len(c.free))
        fresh = count - reuse
        if c.n + fresh > c.capacity:
            raise AdmissionError("collection %r: %d rows free, %d needed" % (name, c.capacity - c.n + len(c.free),
                                                                            count))
        self._quiesce(name)
        rows = np.array(c.free[:reuse] + list(range(c.n, c.n + fresh)), np.int64)
        del c.free[:reuse]
        rowcodes = self._encode_rows(c, X)
        bolt.write_codes(rowcodes, torch.from_numpy(rows).to(self.device), c.codes, c.capacity)
        for i in rows[:reuse]:
            c._set_dead(int(i), False)
        c.n_dead -= reuse
        c.n += fresh
        if reuse:
            c.dead.copy_(torch.from_numpy(c.dead_host.view(np.int32)))
            torch.cuda.current_stream().synchronize()  # later batches run on other streams
        return rows

    def update(self, name, ids, X):
        """Replace the vectors of live rows `ids` by X (re-encoded)."""
        torch = self.torch
        c = self.collections[name]
        ids = np.asarray(ids, np.int64)
        if len(set(ids.tolist())) != len(ids) or any(i < 0 or i >= c.n or c.is_dead(int(i)) for i in ids):
            raise ValueError("update needs distinct live row ids")
        self._quiesce(name)
        bolt.write_codes(self._encode_rows(c, X), torch.from_numpy(ids).to(self.device), c.codes, c.capacity)

    def delete(self, name, ids):
        """Mark rows `ids` deleted: searches no longer return them and
        inserts reuse them."""
        torch = self.torch
        c = self.collections[name]
        ids = np.asarray(ids, np.int64)
        if any(i < 0 or i >= c.n for i in ids):
            raise ValueError("row id out of range")
        self._quiesce(name)
        for i in ids.tolist():
            if not c.is_dead(i):
                c._set_dead(i, True)
                c.free.append(i)
                c.n_dead += 1
        c.dead.copy_(torch.from_numpy(c.dead_host.view(np.int32)))
        torch.cuda.current_stream().synchronize()  # later batches run on other streams

    # -------------------------------------------------------------- requests
    def submit(self, req):
        c = self.collections.get(req.collection)
        if c is None:
            raise AdmissionError("unknown collection %r" % req.collection)
        if req.Q.ndim != 2 or req.Q.shape[1] != c.J:
            raise ValueError("request %r: queries must be (nq, %d)" % (req.rid, c.J))
        if req.kind == SEARCH and not 1 <= req.k <= 1024:
            raise ValueError("request %r: k=%d outside [1, 1024]" % (req.rid, req.k))
        if req.kind == SEARCH and req.k + c.n_dead > 1024:
            raise AdmissionError("request %r: k + %d deleted rows exceeds 1024; insert vectors to reuse them"
                                 % (req.rid, c.n_dead))
        if batch_bytes(c, req.kind, req.nq, req.k) + self.resident > self.budget.total:
            raise AdmissionError("request %r can never fit the HBM budget" % req.rid)
        self.queue.append(req)

    def idle(self):
        return not self.queue and not any(s.busy for s in self.slots)

    def poll(self):
        done = self._retire()
        self._dispatch()
        return done

    def drain(self):
        out = []
        while not self.idle():
            out += self.poll()
        return out

    # -------------------------------------------------------------- internals
    def _retire(self):
        done = []
        for s in self.slots:
            if not s.busy or not s.event.query():
                continue
            t = time.perf_counter()
            for r, row0 in s.reqs:
                if r.kind == MATMUL:
                    r.out = s.host_view.numpy().copy()
                else:
                    iv, dv = s.host_view
                    idx = iv[row0:row0 + r.nq, :r.k].numpy()
                    try:
                        bolt.check_topk(idx)
                        r.idx = idx.copy()
                        r.dist = dv[row0:row0 + r.nq, :r.k].numpy().copy()
                    except bolt.BoltError as e:  # fail the request, never return its -2 rows
                        r.error = e
                r.t_done = t
                done.append(r)
            self.budget.release(s.nbytes)
            s.busy, s.reqs, s.keep, s.host_view = False, [], None, None
        return done

    def _dispatch(self):
        while self.queue:
            slot = next((s for s in self.slots if not s.busy), None)
            if slot is None:
                return
            head = self.queue[0]
            c = self.collections[head.collection]
            batch = self.policy.take(self.queue)
            # the longest prefix of the batch whose working memory fits now
            while True:
                nq = sum(r.nq for r in batch)
                kb = max(r.k for r in batch)
                need = batch_bytes(c, head.kind, nq, kb)
                if self.budget.reserve(need):
                    break
                self.queue.appendleft(batch.pop())
                if not batch:
                    return  # even the oldest request must wait for memory
            self._launch(slot, c, batch, nq, kb, need)

    def _launch(self, slot, c, batch, nq, kb, need):
        torch = self.torch
        t = time.perf_counter()
        s = slot.stream
        J = c.J
        qh = slot.pinned(torch, "q", nq * J, torch.float32).view(nq, J)
        row = 0
        rows = []
        for r in batch:
            qh[row:row + r.nq].numpy()[:] = r.Q
            rows.append((r, row))
            r.t_dispatch = t
            r.batch_id = self.batches
            row += r.nq
        head = batch[0]
        with torch.cuda.stream(s):
            Qd = torch.empty((nq, J), dtype=torch.float32, device=self.device)
            Qd.copy_(qh, non_blocking=True)
            a, b = c.quant[head.metric if head.kind == SEARCH else bolt.METRIC_DOT]
            if head.kind == MATMUL:
                out = torch.empty((nq, c.n), dtype=torch.float32, device=self.device)
                bolt.approx_matmul(Qd, c.codes, c.n, c.C, a, b, out=out, stream=s)
                oh = slot.pinned(torch, "mm", nq * c.n, torch.float32).view(nq, c.n)
                oh.copy_(out, non_blocking=True)
                slot.keep = (Qd, out)
                slot.host_view = oh
                self.launches += 1
            else:
                luts = bolt.build_luts(Qd, c.C, head.metric, a, b, stream=s)
                kr = kb + c.n_dead  # deleted rows are filtered out of a longer list
                ws = torch.empty(bolt.topk_workspace_bytes(c.n, c.M, nq, kr), dtype=torch.uint8,
                                 device=self.device)
                sums, idx = bolt.topk(c.codes, c.n, c.M, luts, kr, head.metric, workspace=ws, stream=s)
                if c.n_dead:
                    sums, idx = bolt.topk_filter(sums, idx, c.dead, c.capacity, kb, stream=s)
                dist = bolt.dequantize(sums, a, b, stream=s)
                ih = slot.pinned(torch, "idx", nq * kb, torch.int64).view(nq, kb)
                dh = slot.pinned(torch, "dist", nq * kb, torch.float32).view(nq, kb)
                ih.copy_(idx, non_blocking=True)
                dh.copy_(dist, non_blocking=True)
                slot.keep = (Qd, luts, ws, sums, idx, dist)
                slot.host_view = (ih, dh)
                self.launches += 3
            slot.event.record(s)
        slot.busy, slot.reqs, slot.nbytes = True, rows, need
        self.batches += 1


# ------------------------------------------------------------------ plain form
def run_plain(collections, trace, device="cuda"):
    """The plain GPU form on the same trace: requests in arrival order, one
    query (or one row of A) per launch, one stream, each query's tables,
    top-k and dequantized results copied back before the next starts.
    ``collections``: name -> Collection.  Fills each request's results and
    times; returns the requests."""
    import torch

    dev = torch.device(device)
    s = torch.cuda.Stream(device=dev)
    t0 = time.perf_counter()
    base = t0
    reqs = sorted(trace, key=lambda r: r.t_arrival)
    ws_cache = {}
    with torch.cuda.stream(s):
        for r in reqs:
            while time.perf_counter() - base < r.t_arrival:
                pass
            r.t_dispatch = time.perf_counter()
            c = collections[r.collection]
            if r.kind == MATMUL:
                a, b = c.quant[bolt.METRIC_DOT]
                out = np.empty((r.nq, c.n), np.float32)
                for i in range(r.nq):
                    Qd = torch.from_numpy(r.Q[i:i + 1]).to(dev, non_blocking=False)
                    o = bolt.approx_matmul(Qd, c.codes, c.n, c.C, a, b, stream=s)
                    out[i] = o.cpu().numpy()[0]
                r.out = out
            else:
                a, b = c.quant[r.metric]
                key = (c.name, r.k)
                if key not in ws_cache:
                    ws_cache[key] = torch.empty(bolt.topk_workspace_bytes(c.n, c.M, 1, r.k), dtype=torch.uint8,
                                                device=dev)
                idx = np.empty((r.nq, r.k), np.int64)
                dist = np.empty((r.nq, r.k), np.float32)
                for i in range(r.nq):
                    Qd = torch.from_numpy(r.Q[i:i + 1]).to(dev)
                    luts = bolt.build_luts(Qd, c.C, r.metric, a, b, stream=s)
                    sm, ix = bolt.topk(c.codes, c.n, c.M, luts, r.k, r.metric, workspace=ws_cache[key], stream=s)
                    d = bolt.dequantize(sm, a, b, stream=s)
                    idx[i] = ix.cpu().numpy()[0]
                    dist[i] = d.cpu().numpy()[0]
                try:
                    bolt.check_topk(idx)
                    r.idx, r.dist = idx, dist
                except bolt.BoltError as e:
                    r.error = e
            r.t_done = time.perf_counter()
    for r in reqs:
        r.t_arrival += base
    return reqs


def run_trace(server, trace):
    """Submit each request at its arrival time (seconds after the start) and
    poll until all are done.  Arrival times are rewritten to absolute host
    times.  Returns the completed requests."""
    reqs = sorted(trace, key=lambda r: r.t_arrival)
    base = time.perf_counter()
    i = 0
    done = []
    while len(done) < len(reqs):
        now = time.perf_counter() - base
        while i < len(reqs) and reqs[i].t_arrival <= now:
            reqs[i].t_arrival += base
            server.submit(reqs[i])
            i += 1
        done += server.poll()
    return done


def latency_stats(reqs, n_of):
    """p50 / p99 / mean latency (ms) from arrival to results on the host,
    and throughput over the whole run.  n_of: collection name -> n."""
    lat = np.array([(r.t_done - r.t_arrival) * 1e3 for r in reqs])
    t_first = min(r.t_arrival for r in reqs)
    t_last = max(r.t_done for r in reqs)
    span = t_last - t_first
    queries = sum(r.nq for r in reqs)
    dists = sum(r.nq * n_of[r.collection] for r in reqs)
    return {"requests": len(reqs), "queries": int(queries), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "max_ms": round(float(lat.max()), 3), "span_s": round(span, 4),
            "queries_per_s": queries / span, "distances_per_s": dists / span}
