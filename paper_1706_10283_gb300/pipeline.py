"""One pass of the Bolt hot path as a reusable, graph-captured step.

``SearchStep`` owns device buffers for a database of n vectors and nq queries
and runs, in order (all in libbolt.so kernels):
  1. encode the database (Sec. 3.1 h, K = 16) -- or, for a resident database
     passed in as ``codes``, encode a batch of ``insert_rows`` new vectors
     into rows ``insert_row0 ..`` of it (an online insert, Sec. 1.3); by
     default on the tensor cores (bf16 split operands, fp32 accumulation and
     an fp32 re-check of near ties: the same codes as the fp32 encoder),
  2. build the uint8 query tables for each metric (Sec. 3.1 g, Sec. 3.2 beta),
  3. scan + exact top-k, one query per launch (the plain GPU form); the
     launches go round-robin to ``streams`` CUDA streams, each with its own
     workspace, so the next query's scan can start on the SMs that the
     previous query's final merge leaves idle,
  4. dequantize the k best sums to distances / inner products (Sec. 3.2).
The launch sequence is captured once into a CUDA graph and replayed, so the
per-launch host overhead of the thousands of small launches is paid once.
``run_from_host`` adds the host->device copy of the step's inputs from pinned
memory and the device->host copy of its results; the upload runs on its own
stream and waits only until the previous step's encode and table build have
read the input buffers, so consecutive steps overlap one step's upload with
the previous step's searches.
"""
import numpy as np
import torch

from . import bolt


class SearchStep:
    def __init__(self, n, J, M, nq, k, centroids, quant, metrics=(bolt.METRIC_L2, bolt.METRIC_DOT),
                 precision=bolt.PREC_BF16_RECHECK, device="cuda", streams=8, codes=None, insert_row0=0,
                 insert_rows=None):
        self.n, self.J, self.M, self.nq, self.k = n, J, M, nq, k
        self.metrics = tuple(metrics)
        self.quant = dict(quant)  # metric -> (a, b)
        self.precision = precision
        dev = torch.device(device)
        self.C = centroids
        nx = n if insert_rows is None else int(insert_rows)
        r0 = int(insert_row0)
        if r0 % 256 or r0 < 0 or r0 + nx > n or (r0 + nx != n and nx % 256):
            raise ValueError("insert rows [%d, %d) must start on a 256-vector block and end on one or at n"
                             % (r0, r0 + nx))
        if codes is None and nx != n:
            raise ValueError("an insert batch needs a resident database (codes)")
        self.row0, self.nx = r0, nx
        self.X = torch.empty((nx, J), dtype=torch.float32, device=dev)
        self.Q = torch.empty((nq, J), dtype=torch.float32, device=dev)
        if codes is None:
            codes = torch.empty(bolt.codes_bytes(n, M), dtype=torch.uint8, device=dev)
        if codes.numel() != bolt.codes_bytes(n, M):
            raise ValueError("codes hold %d bytes, the layout of %d vectors needs %d"
                             % (codes.numel(), n, bolt.codes_bytes(n, M)))
        self.codes = codes
        b0 = r0 // 256 * M * 128
        self.codes_x = codes[b0:b0 + bolt.codes_bytes(nx, M)]  # the rows the step encodes
        self.luts = {m: torch.empty((nq, M, 16), dtype=torch.uint8, device=dev) for m in self.metrics}
        self.sums = {m: torch.empty((nq, k), dtype=torch.uint16, device=dev) for m in self.metrics}
        self.idx = {m: torch.empty((nq, k), dtype=torch.int64, device=dev) for m in self.metrics}
        self.dist = {m: torch.empty((nq, k), dtype=torch.float32, device=dev) for m in self.metrics}
        self.side = [torch.cuda.Stream(device=dev) for _ in range(max(1, streams))]
        self.ws = [torch.empty(bolt.topk_workspace_bytes(n, M, 1, k), dtype=torch.uint8, device=dev)
                   for _ in self.side]
        self.graphs = None
        self.copy_stream = torch.cuda.Stream(device=dev)
        self._copied = torch.cuda.Event()
        # recorded on the current stream after every write or read of X and Q
        # there (set_inputs, the encode and table build of a replay): an
        # upload into X and Q waits for it
        self._inputs_read = torch.cuda.Event()
        self.launches_per_step = 1 + len(self.metrics) * (2 + nq)
        self.timing = []  # (start, end) event pairs around each top-k segment

    def set_inputs(self, X, Q):
        self.X.copy_(X)
        self.Q.copy_(Q)
        self._inputs_read.record()

    # The step in three kinds of segments, so that top-k launches can be timed
    # by ordinary stream events recorded between graph replays.
    def _pre(self):
        bolt.encode(self.X, self.C, self.precision, out=self.codes_x)
        for m in self.metrics:
            a, b = self.quant[m]
            bolt.build_luts(self.Q, self.C, m, a, b, out=self.luts[m])

    def _topk(self, m):
        cur = torch.cuda.current_stream()
        for s in self.side:
            s.wait_stream(cur)
        for q in range(self.nq):
            i = q % len(self.side)
            bolt.topk(self.codes, self.n, self.M, self.luts[m][q:q + 1], self.k, m,
                      out_sums=self.sums[m][q:q + 1], out_idx=self.idx[m][q:q + 1], workspace=self.ws[i],
                      stream=self.side[i])
        for s in self.side:
            cur.wait_stream(s)

    def _post(self):
        for m in self.metrics:
            a, b = self.quant[m]
            bolt.dequantize(self.sums[m], a, b, out=self.dist[m])

    def _segments(self):
        return [self._pre] + [(lambda m=m: self._topk(m)) for m in self.metrics] + [self._post]

    def run(self):
        """Enqueue one step on the current stream (no host synchronization)."""
        for seg in self._segments():
            seg()

    def capture(self):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()  # warm-up outside capture: sets kernel attributes once
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        graphs = []
        for seg in self._segments():
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, capture_error_mode="thread_local"):
                seg()
            graphs.append(g)
        self.graphs = graphs
        return graphs

    def replay(self, timed=False):
        if self.graphs is None:
            self.capture()
        self.graphs[0].replay()
        self._inputs_read.record()  # the encode and tables have read X and Q
        for g in self.graphs[1:-1]:
            if timed:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                g.replay()
                e1.record()
                self.timing.append((e0, e1))
            else:
                g.replay()
        self.graphs[-1].replay()

    def serial_topk_ms(self, launches=20, reps=10, metric=bolt.METRIC_L2):
        """Device time of one top-k launch by itself: `launches` launches on
        one stream, captured in a CUDA graph and replayed `reps` times
        between two events."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())

        def body():
            for q in range(launches):
                qq = q % self.nq
                bolt.topk(self.codes, self.n, self.M, self.luts[metric][qq:qq + 1], self.k, metric,
                          out_sums=self.sums[metric][qq:qq + 1], out_idx=self.idx[metric][qq:qq + 1],
                          workspace=self.ws[0], stream=s)

        with torch.cuda.stream(s):
            body()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            body()
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / (reps * launches)

    def flushed_topk_ms(self, launches=10, flush_bytes=512 << 20, metric=bolt.METRIC_L2):
        """Device time of one top-k launch with cold caches: before each
        launch a buffer of flush_bytes (several times the L2) is written, and
        only the launch (header memset + kernel) lies between the events."""
        buf = torch.empty(flush_bytes, dtype=torch.uint8, device="cuda")
        pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(launches)]
        for q, (e0, e1) in enumerate(pairs):
            qq = q % self.nq
            buf.zero_()
            e0.record()
            bolt.topk(self.codes, self.n, self.M, self.luts[metric][qq:qq + 1], self.k, metric,
                      out_sums=self.sums[metric][qq:qq + 1], out_idx=self.idx[metric][qq:qq + 1],
                      workspace=self.ws[0])
            e1.record()
        torch.cuda.synchronize()
        del buf
        return float(np.median([e0.elapsed_time(e1) for e0, e1 in pairs]))

    def topk_ms_per_launch(self):
        """Step time of the top-k segments divided by their launches (call
        after synchronizing): with launches overlapping on several streams
        this is the time per query of the step, not one launch's duration."""
        if not self.timing:
            return float("nan")
        tot = sum(e0.elapsed_time(e1) for e0, e1 in self.timing)
        return tot / (len(self.timing) * self.nq)

    def run_from_host(self, X_host, Q_host, out_idx_host, out_dist_host):
        """End to end: pinned host inputs -> device step -> host results
        (asynchronous; X_host and Q_host must stay unchanged, and the host
        outputs unread, until the current stream reaches this point).  The
        upload goes on copy_stream after the previous step's encode and
        tables have read the input buffers, so it overlaps that step's
        searches; the step itself waits for the upload."""
        cur = torch.cuda.current_stream()
        if self.graphs is None:
            self.capture()
        self.copy_stream.wait_event(self._inputs_read)
        with torch.cuda.stream(self.copy_stream):
            self.X.copy_(X_host, non_blocking=True)
            self.Q.copy_(Q_host, non_blocking=True)
            self._copied.record(self.copy_stream)
        cur.wait_event(self._copied)
        self.replay()
        for j, m in enumerate(self.metrics):
            out_idx_host[j].copy_(self.idx[m], non_blocking=True)
            out_dist_host[j].copy_(self.dist[m], non_blocking=True)

    def h2d_bytes(self):
        return self.X.numel() * 4 + self.Q.numel() * 4

    def d2h_bytes(self):
        return len(self.metrics) * self.nq * self.k * (8 + 4)
