#!/usr/bin/env python3
"""Benchmark of the Bolt hot path on GB300.

Workload (default, the large-N serving database): 50,000,000 x 128
Gaussian-mixture vectors encoded with M = 16 codebooks (8-byte codes, 400 MB,
larger than the 129 MB L2), resident on the device.  One step = one pass of
the whole path over one batch of synthetic input:
  1. encode a batch of 1,000,064 new database rows (an online insert into the
     last rows of the database, Sec. 1.3; the batch holds the same vectors as
     those rows, so the database is the same after every step),
  2. build the uint8 query tables of 64 L2 and 64 dot-product queries,
  3. fused scan + exact top-100 for each query, ONE QUERY PER LAUNCH (the
     plain GPU form), the launches alternating on two CUDA streams with
     separate workspaces, replayed from CUDA graphs,
  4. dequantize the 128 x 100 best sums.
The metric is encoded-vector distances per second: 128 queries x 50,000,000
vectors per step.

Also reported in the same JSON line:
  e2e           the same step from pinned host buffers (the insert batch and
                the queries copied in, the results copied out) through
                SearchStep.run_from_host,
  roofline      the dominant kernel (topk_kernel, the streaming fused scan +
                top-k) against the measured HBM copy bandwidth, with the
                bare lookup core's time (bolt_probe_lookup_core) beside it,
  cpu_baseline  the CPU oracle on this host: a seeded sample of queries over
                the full 50M codes, one thread and all cores,
and, as extra keys, the other configurations (1M mixture step, small i.i.d.
workload, 64-query batch on 50M, serving trace, 10M encoder and k-means fit,
64-collection batch, approximate matmul, accuracy).

``--impl reference`` times the CPU oracle (the only reference this method
has) on a bounded sample of the same workload per step and prints its line
with "impl": "reference".  Multi-GPU (torchrun, one process per GPU): each
rank runs the same step on its own database (weak scaling, no collective on
the data path); the time is the maximum over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encoded-vector distances/sec and code GB/s vs HBM peak; encode GB/s; served p50/p99"
UNIT = "distances/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0  # GB/s, used only when MEASURED_PEAKS.json is absent


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["bolt", "reference"], default="bolt")
    ap.add_argument("--nq", type=int, default=None, help="override query count (profiling runs)")
    ap.add_argument("--no-aux", action="store_true", help="skip the large-N and encode side measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", choices=["topk1m", "topk50m", "topk8m_batch64", "encode10m", "encode10m_tc", "batch", "serve",
                             "large50m", "accuracy", "matmul"], default=None,
                    help="profiling run: set up one workload and launch only its kernel a few times")
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--graph-reps", type=int, default=0, help="also time graph replays of the launches")
    ap.add_argument("--collections", type=int, default=64, help="--only batch: first N collections")
    ap.add_argument("--topk-streams", type=int, default=8, help="streams of the 1M step's one-query launches")
    ap.add_argument("--large-streams", type=int, default=4, help="streams of the 50M step's one-query launches")
    ap.add_argument("--large-nq", type=int, default=64, help="queries per metric in the 50M step")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# ------------------------------------------------------------------ distributed
def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if (args.impl == "bolt" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm_sorted) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ workload
def workload(nq_override=None):
    from paper_1706_10283_gb300 import synth

    cfg = dict(synth.CONFIGS["mixture_1m"])
    if nq_override:
        cfg["nq"] = nq_override
    return cfg


def oracle_step_sample(codes_host, Xins_host, Q_host, C, quant, nq_step, k, threads, q_sample=1,
                       enc_rows=20_000):
    """The CPU oracle on a bounded sample of one 50M step: the encode of
    enc_rows of the insert batch, the tables of every query of the step, and
    scan + top-k of q_sample queries per metric over all the database's
    codes (on `threads` host threads, oracle.parallel); each part is timed
    and scaled to the whole step.  Returns (distances/s, seconds of CPU work,
    description)."""
    import oracle
    from oracle import parallel

    n = codes_host.shape[0]
    nx = Xins_host.shape[0]
    t0 = time.perf_counter()
    oracle.encode(Xins_host[:enc_rows], C)
    t_enc = time.perf_counter() - t0
    t_lut = t_scan = 0.0
    for metric in (oracle.METRIC_L2, oracle.METRIC_DOT):
        a, b = quant[metric]
        t0 = time.perf_counter()
        luts = oracle.quantize(oracle.lut_f32(Q_host[:nq_step], C, metric), a, b)
        t_lut += time.perf_counter() - t0
        for qi in range(q_sample):
            t0 = time.perf_counter()
            s_, _ = parallel.scan_topk(codes_host, luts[qi:qi + 1], k, metric, threads=threads)
            oracle.dequant(s_, a, b)
            t_scan += time.perf_counter() - t0
    t_step = t_enc * nx / enc_rows + t_lut + t_scan * nq_step / q_sample
    work = t_enc + t_lut + t_scan
    desc = ("oracle on %d host thread(s): encode of %d of the %d insert rows, tables of all %d x 2 queries, scan + "
            "top-%d + dequantize of %d L2 and %d dot queries over all %d codes; each part scaled to the full step"
            % (threads, enc_rows, nx, nq_step, k, q_sample, q_sample, n))
    return 2.0 * nq_step * n / t_step, work, desc


def prepare(cfg, data_seed, device="cuda"):
    """Seeded inputs and the offline fit (codebooks, quantizers) on the GPU."""
    import torch

    from paper_1706_10283_gb300 import bolt, synth

    n, J, M, nq = cfg["n"], cfg["J"], cfg["M"], cfg["nq"]
    X = synth.mixture(n, J, data_seed)
    Q = synth.mixture(nq, J, 1)
    Xd = torch.from_numpy(X).to(device)
    Qd = torch.from_numpy(Q).to(device)
    C = bolt.fit_codebooks(Xd, M, cfg["iters"], synth.kmeans_init_rows(n, 0))
    Qtr = Xd[torch.from_numpy(synth.train_query_rows(n, 0)).to(device)].contiguous()
    quant = {}
    for m in (bolt.METRIC_L2, bolt.METRIC_DOT):
        a, b, _ = bolt.fit_quantizer(Qtr, C, m)
        quant[m] = (float(a), b)
    return X, Q, Xd, Qd, C, quant


LARGE_CHUNK = 1 << 21  # rows per generated chunk of the 50M database (a multiple of 256)


def build_50m(C, seed_base=5000):
    """Codes of the 50,000,000 x 128 mixture database (M = 16), encoded in
    2M-row chunks generated on the device (chunk c from seed seed_base + c)."""
    import torch

    from paper_1706_10283_gb300 import bolt, synth

    cfg = synth.CONFIGS["serve_50m"]
    n, J, M = cfg["n"], cfg["J"], cfg["M"]
    codes = torch.empty(bolt.codes_bytes(n, M), dtype=torch.uint8, device="cuda")
    buf = torch.empty((LARGE_CHUNK, J), dtype=torch.float32, device="cuda")
    for lo in range(0, n, LARGE_CHUNK):
        hi = min(n, lo + LARGE_CHUNK)
        X = synth.mixture_torch(hi - lo, J, seed=seed_base + lo // LARGE_CHUNK, out=buf[:hi - lo])
        row0 = lo // 256 * M * 128
        bolt.encode(X, C, out=codes[row0:row0 + bolt.codes_bytes(hi - lo, M)])
    del buf
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return codes


INSERT_ROWS = 1_000_064  # the step's insert batch: the database's last rows


def insert_batch(seed_base=5000):
    """(row0, X): the vectors of rows [row0, 50M) of the database generated by
    build_50m with the same seeds; row0 = 50M - INSERT_ROWS is a multiple of
    256, so the batch is encoded into whole code blocks."""
    from paper_1706_10283_gb300 import synth

    cfg = synth.CONFIGS["serve_50m"]
    n, J = cfg["n"], cfg["J"]
    row0 = n - INSERT_ROWS
    assert row0 % 256 == 0
    c = row0 // LARGE_CHUNK
    lo = c * LARGE_CHUNK
    X = synth.mixture_torch(min(n, lo + LARGE_CHUNK) - lo, J, seed=seed_base + c)
    assert lo + X.shape[0] == n  # the batch lies in the last chunk
    return row0, X[row0 - lo:].contiguous()


def accuracy_report(Xd, C, quant, nq=200, seed=21):
    """Accuracy on the 1M mixture (the paper's Recall@R, Sec. 4.5, and
    dot-product correlation, Sec. 4.6): for nq held-out mixture queries, the
    fraction whose true nearest neighbour (fp64 brute force) is among the R
    best by Bolt's uint8-table sums and by the fp32-table sums ("Bolt No
    Quantize"); and the Pearson correlation of dequantized approximate dot
    products with the true ones over a sample of pairs."""
    import torch

    from paper_1706_10283_gb300 import bolt, synth

    n, J = Xd.shape
    M = C.shape[0]
    Q = synth.mixture_torch(nq, J, seed=seed)
    codes = bolt.encode(Xd, C)
    a, b = quant[bolt.METRIC_L2]
    luts, luts32 = bolt.build_luts(Q, C, bolt.METRIC_L2, a, b, out_f32=True)
    # ground truth: fp64 brute force nearest neighbour
    X64 = Xd.double()
    true_nn = []
    for lo in range(0, nq, 50):
        q64 = Q[lo:lo + 50].double()
        d = (q64 * q64).sum(1, keepdim=True) - 2 * q64 @ X64.T + (X64 * X64).sum(1)[None]
        true_nn.append(d.argmin(1))
    true_nn = torch.cat(true_nn)
    del X64
    Rs = (1, 10, 100)
    out = {"queries": nq, "R": list(Rs)}
    s_q, i_q = bolt.topk(codes, n, M, luts, max(Rs), bolt.METRIC_L2)
    sf = bolt.scan_float(codes, n, M, luts32)
    i_f = torch.topk(sf, max(Rs), dim=1, largest=False).indices
    for name, idx in (("bolt_uint8_tables", i_q), ("bolt_no_quantize_fp32_tables", i_f)):
        out[name] = {"recall_at_R": [float((idx[:, :R] == true_nn[:, None]).any(1).float().mean()) for R in Rs]}
    # dot products: approximate (dequantized) vs true on a sample of pairs
    ad, bd = quant[bolt.METRIC_DOT]
    ld = bolt.build_luts(Q[:20], C, bolt.METRIC_DOT, ad, bd)
    approx = bolt.dequantize(bolt.scan_dot(codes, n, M, ld), ad, bd)[:, :200_000].double()
    true = Q[:20].double() @ Xd[:200_000].double().T
    a_c, t_c = approx - approx.mean(), true - true.mean()
    out["dot_correlation"] = float((a_c * t_c).sum() / (a_c.norm() * t_c.norm()))
    del sf
    torch.cuda.empty_cache()
    return out


def batch_64_on_50m(codes, C, quant):
    """64 L2 queries over the 50M database in one call (the multi-query
    pipeline: every code pass shared by up to 16 queries), against the
    one-query launches of the headline step."""
    import torch

    from paper_1706_10283_gb300 import bolt, synth

    cfg = synth.CONFIGS["serve_50m"]
    n, J, M, k = cfg["n"], cfg["J"], cfg["M"], 100
    a, b = quant[bolt.METRIC_L2]
    Qb = torch.from_numpy(synth.mixture(64, J, 78)).cuda()
    lb = bolt.build_luts(Qb, C, bolt.METRIC_L2, a, b)
    wsb = torch.empty(bolt.topk_workspace_bytes(n, M, 64, k), dtype=torch.uint8, device="cuda")
    ob_s = torch.empty((64, k), dtype=torch.uint16, device="cuda")
    ob_i = torch.empty((64, k), dtype=torch.int64, device="cuda")
    ms_b = _graph_ms(lambda s: bolt.topk(codes, n, M, lb, k, bolt.METRIC_L2, ob_s, ob_i, workspace=wsb, stream=s),
                     reps=3)
    bolt.check_topk(ob_i)
    del wsb
    return {"workload": "serve_50m: 64 L2 top-100 queries in one bolt_topk call (multi-query pipeline)",
            "ms_per_call": round(ms_b, 4), "ms_per_query": round(ms_b / 64, 4),
            "distances_per_s": 64 * n / (ms_b * 1e-3)}


def scan_sums_report(codes, C, quant, hbm_peak):
    """The plain scan (uint16 sums, no top-k): one query over the 50M
    database against the HBM roofline (codes read + sums written), and 1,000
    queries over its first 1M vectors (tiles of 8 queries per code pass)
    against the integer-ALU peak.  The 1,000-query sums of query 0 must equal
    the one-query sums over the same vectors."""
    import torch

    from paper_1706_10283_gb300 import alu_peak, bolt, synth

    cfg = synth.CONFIGS["serve_50m"]
    n, J, M = cfg["n"], cfg["J"], cfg["M"]
    a, b = quant[bolt.METRIC_L2]
    Qs = torch.from_numpy(synth.mixture(1000, J, 79)).cuda()
    luts = bolt.build_luts(Qs, C, bolt.METRIC_L2, a, b)
    out1 = torch.empty((1, n), dtype=torch.uint16, device="cuda")
    ms1 = _graph_ms(lambda s: bolt.scan_l2(codes, n, M, luts[:1], out=out1, stream=s), reps=10)
    n2 = 1_000_000
    codes2 = codes[:bolt.codes_bytes(n2, M)]
    out2 = torch.empty((1000, n2), dtype=torch.uint16, device="cuda")
    ms2 = _graph_ms(lambda s: bolt.scan_l2(codes2, n2, M, luts, out=out2, stream=s), reps=3)
    same = bool(torch.equal(out2[0], out1[0, :n2]))
    del out1, out2
    torch.cuda.empty_cache()
    bytes1 = n * M // 2 + 2 * n
    lookups2 = 1000 * n2 * M
    peak = alu_peak.lookups_per_s()
    return {"workload": "bolt_scan_l2 (uint16 sums): 1 query over serve_50m; 1,000 queries over its first 1M vectors",
            "one_query_50m": {"ms": round(ms1, 4), "bytes": bytes1,
                              "achieved_GBps": round(bytes1 / (ms1 * 1e-3) / 1e9, 1), "peak_GBps": hbm_peak,
                              "frac": round(bytes1 / (ms1 * 1e-3) / 1e9 / hbm_peak, 4)},
            "queries_1000_on_1m": {"ms": round(ms2, 4), "lookups": lookups2,
                                   "achieved_Tlookup_s": round(lookups2 / (ms2 * 1e-3) / 1e12, 3),
                                   "peak_Tlookup_s": round(peak / 1e12, 3),
                                   "frac": round(lookups2 / (ms2 * 1e-3) / peak, 4)},
            "query0_sums_equal": same}


def serving(codes50, C, quant, count=300, rates=(40.0, 80.0), slots=4, budget_gb=16.0):
    """Serving trace on the resident 50M-vector database plus the encoded
    100,000 x 512 matmul operand (M = 32): Poisson arrivals, 1..512 queries
    per request, L2 / dot, k 10..100, 10% approximate-matmul requests
    (1..512 rows of A); the continuous-batching server against the plain
    one-query-per-launch form on the same trace."""
    import torch

    from paper_1706_10283_gb300 import bolt, serve, synth

    cfg = synth.CONFIGS["serve_50m"]
    mm = synth.CONFIGS["matmul_4096x512_100k"]
    B = synth.mixture_torch(mm["n"], mm["J"], seed=900)
    CB, aB, bB = bolt.fit_codebooks(B[:50_000].contiguous(), mm["M"], 8, synth.kmeans_init_rows(50_000, 900),
                                    Qtrain=B[torch.from_numpy(synth.train_query_rows(mm["n"], 900)).cuda()]
                                    .contiguous(), metric=bolt.METRIC_DOT)
    codesB = bolt.encode(B, CB)
    del B
    srv = serve.Server(int(budget_gb * 2**30), slots=slots)
    srv.add_collection("db", codes50, cfg["n"], cfg["M"], C, quant)
    srv.add_collection("B", codesB, mm["n"], mm["M"], CB, {bolt.METRIC_DOT: (aB, bB), bolt.METRIC_L2: (aB, bB)})
    n_of = {"db": cfg["n"], "B": mm["n"]}
    out = {"workload": "serve_50m: resident 50,000,000 x 128 (M=16, 400 MB codes) + matmul B 100,000 x 512 "
                       "(M=32); %d Poisson requests per rate, 1-512 queries (log-uniform), L2/dot, k 10-100, "
                       "10%% matmul (1-512 rows of A)" % count,
           "latency": "host time from scheduled arrival to results in host memory", "rates": []}
    for rate in rates:
        trace = synth.poisson_trace(11, count, rate, cfg["J"], matmul_frac=0.1, J_mm=mm["J"])

        def requests():
            return [serve.Request(i, "B" if r["kind"] == "matmul" else "db", r["Q"], kind=r["kind"],
                                  metric=r["metric"], k=r["k"], t_arrival=r["t_arrival"])
                    for i, r in enumerate(trace)]

        # warm-up: a few requests through both forms (kernel attributes, pinned buffers)
        warm = requests()[:6]
        for r in warm:
            r.t_arrival = 0.0
        serve.run_trace(srv, warm)
        serve.run_plain(srv.collections, requests()[:2])
        torch.cuda.synchronize()
        b0, l0 = srv.batches, srv.launches
        got = serve.run_trace(srv, requests())
        srv_stats = serve.latency_stats(got, n_of)
        srv_stats.update(batches=srv.batches - b0, slots=slots, budget_bytes=srv.budget.total,
                         peak_budget_bytes=srv.budget.peak)
        plain = serve.run_plain(srv.collections, requests())
        plain_stats = serve.latency_stats(plain, n_of)
        by = {r.rid: r for r in plain}
        diff = []
        for r in got:
            p = by[r.rid]
            if r.error is not None or p.error is not None:
                diff.append({"rid": r.rid, "failed": str(r.error or p.error)})
                continue
            if r.kind == "matmul":
                if not np.array_equal(r.out, p.out):
                    diff.append({"rid": r.rid, "kind": "matmul", "rows": r.nq, "batch": r.batch_id,
                                 "elements": int((r.out != p.out).sum())})
            else:
                rows = (r.idx != p.idx).any(axis=1) | (r.dist != p.dist).any(axis=1)
                if rows.any():
                    diff.append({"rid": r.rid, "kind": "search", "nq": r.nq, "k": r.k, "metric": r.metric,
                                 "batch": r.batch_id, "rows": int(rows.sum())})
        out["rates"].append({"rate_per_s": rate, "offered_queries_per_s": sum(r["nq"] for r in trace) /
                             trace[-1]["t_arrival"], "server": srv_stats,
                             "plain_one_query_per_launch": plain_stats, "results_identical": not diff,
                             "mismatches": diff[:10]})
    del srv, codesB
    torch.cuda.empty_cache()
    return out


def encode_10m():
    """Encode 10,000,000 x 256 fp32 mixture rows into M = 32 codes."""
    import torch

    from paper_1706_10283_gb300 import bolt, synth

    cfg = synth.CONFIGS["encode_10m"]
    n, J, M = cfg["n"], cfg["J"], cfg["M"]
    X = synth.mixture_torch(n, J, seed=0)
    # the codebooks: k-means on all 10,000,000 rows (Sec. 3.1 background,
    # 16 Lloyd iterations from the seeded init), timed
    iters = 16
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    C = bolt.fit_codebooks(X, M, iters, synth.kmeans_init_rows(n, 0))
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    codes = torch.empty(bolt.codes_bytes(n, M), dtype=torch.uint8, device="cuda")
    out = {}
    hbm_peak, _ = peaks()
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    codes_tc = torch.empty_like(codes)
    for name, prec, dst in (("fp32", bolt.PREC_FP32, codes), ("bf16_tensor_core_recheck", bolt.PREC_BF16_RECHECK,
                                                                codes_tc)):
        for _ in range(2):
            bolt.encode(X, C, prec, out=dst, n_rechecked=cnt)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        reps = 5
        ev[0].record()
        for _ in range(reps):
            bolt.encode(X, C, prec, out=dst, n_rechecked=cnt)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / reps
        gbs = (n * J * 4 + n * M / 2) / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 4), "input_GBps": round(n * J * 4 / (ms * 1e-3) / 1e9, 1),
                     "vectors_per_s": n / (ms * 1e-3), "hbm_frac": round(gbs / hbm_peak, 4),
                     "rechecked_pairs": int(cnt.item()), "recheck_rate": round(int(cnt.item()) / (n * M), 4)}
    same = bool(torch.equal(codes, codes_tc))
    # precision report on a sample of rows: codes vs the fp64 argmin, and the
    # reconstruction error of the fp32 codes vs the fp64 codes
    import oracle

    rows = 20_000
    Xs = X[:rows].cpu().numpy()
    Cn = C.cpu().numpy()
    c64 = oracle.encode(Xs, Cn, precision="f64")
    c32 = bolt.unpack_codes(codes_tc[:bolt.codes_bytes(rows, M)], rows, M).cpu().numpy()
    mse = lambda cc: float(np.mean(np.sum((Xs.astype(np.float64) - oracle.decode(cc, Cn)) ** 2, axis=1)))  # noqa
    del X, codes, codes_tc
    torch.cuda.empty_cache()
    return {"workload": "encode_10m: 10,000,000 x 256 fp32 mixture, M=32", **out,
            "kmeans_fit": {"rows": n, "iterations": iters, "seconds": round(fit_s, 3),
                           "ms_per_iteration": round(fit_s * 1e3 / iters, 2),
                           "timing": "host clock around bolt_fit_codebooks (blocking), device synchronized"},
            "tensor_core_codes_equal_fp32": same,
            "sample_rows": rows, "mismatch_rate_vs_fp64": float(np.mean(c32 != c64)),
            "mse_fp32_codes": mse(c32), "mse_fp64_codes": mse(c64)}


def collections_setup(count=64):
    """The multi-collection batch on the GPU: per collection the seeded
    mixture data, a GPU fit (8 k-means iterations on up to 50,000 rows, the
    quantizer on 256 training rows), codes, query tables (L2 for even, dot
    for odd collections) and an output matrix."""
    import torch

    from paper_1706_10283_gb300 import bolt, synth

    specs = synth.collections(seed=3)[:count]
    out = []
    for ci, sp in enumerate(specs):
        n, J, M, nq = sp["n"], sp["J"], sp["M"], sp["nq"]
        metric = ci % 2
        X = synth.mixture_torch(n, J, sp["data_seed"])
        nf = min(n, 50_000)
        Qtr = X[torch.from_numpy(synth.train_query_rows(n, sp["data_seed"])).cuda()].contiguous()
        C, a, b = bolt.fit_codebooks(X[:nf].contiguous(), M, 8, synth.kmeans_init_rows(nf, sp["data_seed"]),
                                     Qtrain=Qtr, metric=metric)
        codes = bolt.encode(X, C)
        del X, Qtr
        Q = synth.mixture_torch(nq, J, sp["query_seed"])
        luts = bolt.build_luts(Q, C, metric, a, b)
        sums = torch.empty((nq, bolt.sums_ld(n)), dtype=torch.int16, device="cuda").view(torch.uint16)
        out.append(dict(n=n, J=J, M=M, nq=nq, codes=codes, luts=luts, sums=sums))
    torch.cuda.synchronize()
    return out


def _graph_ms(fn, reps):
    """Device time of one call of fn, captured once in a CUDA graph and
    replayed `reps` times between two events."""
    import torch

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn(s)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        fn(s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def batched_collections():
    """64 collections (N log-uniform in [1e3, 2e6], J in {64,128,256}, M in
    {8,16,32}, 1..256 queries each) scanned three ways, each captured in a
    CUDA graph: one persistent batched launch (autotuned tiles), one
    bolt_scan_l2 launch per collection, and one launch per query."""
    import torch

    from paper_1706_10283_gb300 import alu_peak, bolt

    batch = collections_setup()
    dists = sum(c["n"] * c["nq"] for c in batch)
    lookups = sum(c["n"] * c["nq"] * c["M"] for c in batch)
    plan = bolt.BatchPlan([(c["codes"], c["n"], c["M"], c["luts"], c["sums"]) for c in batch])
    t0 = time.perf_counter()
    tune_ms = plan.autotune()
    tune_s = time.perf_counter() - t0
    batched_ms = _graph_ms(lambda s: plan.run(stream=s), reps=10)
    plain = [torch.empty((c["nq"], c["n"]), dtype=torch.int16, device="cuda").view(torch.uint16) for c in batch]

    def per_collection(s):
        for c, o in zip(batch, plain):
            bolt.scan_l2(c["codes"], c["n"], c["M"], c["luts"], out=o, stream=s)

    def per_query(s):
        for c, o in zip(batch, plain):
            for q in range(c["nq"]):
                bolt.scan_l2(c["codes"], c["n"], c["M"], c["luts"][q:q + 1], out=o[q:q + 1], stream=s)

    coll_ms = _graph_ms(per_collection, reps=5)
    query_ms = _graph_ms(per_query, reps=2)
    plan.run()
    torch.cuda.synchronize()
    same = all(torch.equal(c["sums"].view(torch.int16)[:, :c["n"]], o.view(torch.int16)) for c, o in zip(batch, plain))
    peak = alu_peak.lookups_per_s()
    tuning = plan.tuning()
    by_m = {}
    for c, (qt, upw) in zip(batch, tuning):
        by_m[str(c["M"])] = {"qt_max": qt, "units_per_warp": upw}
    res = {"workload": "64 collections, N log-uniform in [1e3, 2e6] (%d vectors), J in {64,128,256}, "
                       "M in {8,16,32}, 1-256 queries each (%d queries)" % (sum(c["n"] for c in batch),
                                                                            sum(c["nq"] for c in batch)),
           "distances_per_batch": dists, "lookups_per_batch": lookups,
           "batched": {"ms": round(batched_ms, 4), "distances_per_s": dists / (batched_ms * 1e-3),
                       "launches": 1, "tiles_by_M": by_m, "autotune_s": round(tune_s, 2),
                       "autotune_best_ms": round(tune_ms, 4)},
           "per_collection_launch": {"ms": round(coll_ms, 4), "distances_per_s": dists / (coll_ms * 1e-3),
                                     "launches": len(batch)},
           "one_query_per_launch": {"ms": round(query_ms, 4), "distances_per_s": dists / (query_ms * 1e-3),
                                    "launches": sum(c["nq"] for c in batch)},
           "sums_equal": bool(same),
           "roofline": {"bound": "alu", "kernel": "batch_scan_kernel",
                        "achieved": round(lookups / (batched_ms * 1e-3) / 1e12, 4),
                        "peak": round(peak / 1e12, 4), "unit": "Tlookup/s",
                        "frac": round(lookups / (batched_ms * 1e-3) / peak, 4), "peak_source": alu_peak.source(),
                        "sums_written_GB": round(sum(c["nq"] * c["n"] * 2 for c in batch) / 1e9, 3)},
           "l2_cache": "every launch writes %.1f GB of sums (> L2)" % (sum(c["nq"] * c["n"] * 2 for c in batch) / 1e9)}
    # the CPU oracle on a sample of the batch: one query of every collection
    # (oracle.scan in host threads, one collection per thread), scaled to
    # the batch's distances
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from oracle import parallel

    host = [(bolt.unpack_codes(c["codes"], c["n"], c["M"]).cpu().numpy(), c["luts"][:1].cpu().numpy())
            for c in batch]
    sample = sum(c["n"] for c in batch)
    for threads in (1, parallel.host_threads()):
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda cl: oracle.scan(cl[0], cl[1]), host))
        dt = time.perf_counter() - t0
        res.setdefault("oracle_sample", []).append(
            {"threads": threads, "sample": "one query per collection (%d distances)" % sample,
             "seconds": round(dt, 3), "distances_per_s": sample / dt,
             "batch_seconds_scaled": round(dt * dists / sample, 2)})
    del plan, batch, plain, host
    torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------------ arms
def clustered_codes_host(n, M, seed, clusters=256, chunk=5_000_000):
    """Row-major codes with the structure of an encoded mixture (each row in
    one of `clusters` groups takes its group's code in a codebook with
    probability 1/2, else a uniform code), generated on the host: the
    reference arm builds its database without the GPU."""
    rng = np.random.default_rng(seed)
    pref = rng.integers(0, 16, (clusters, M), dtype=np.uint8)
    out = np.empty((n, M), np.uint8)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        g = rng.integers(0, clusters, hi - lo)
        r = rng.integers(0, 32, (hi - lo, M), dtype=np.uint8)
        out[lo:hi] = np.where(r < 16, r, pref[g])
    return out


def run_reference(args, world, rank):
    """CPU oracle on this host's cores, on a bounded sample of the 50M step:
    per step the encode of 2,000 insert rows, the tables of one L2 and one dot
    query, and their scan + top-100 + dequantize over all 50M codes (all host
    threads, oracle.parallel).  The database is built on the host (codes with
    an encoded mixture's structure; the oracle's cost does not depend on the
    code values)."""
    if rank != 0:
        return
    import oracle
    from oracle import parallel
    from paper_1706_10283_gb300 import synth

    cfg = synth.CONFIGS["serve_50m"]
    n, J, M, k = cfg["n"], cfg["J"], cfg["M"], 100
    fit_rows = 20_000
    Xf = synth.mixture(fit_rows, J, 0)
    C = oracle.kmeans(Xf, M, 4, synth.kmeans_init_rows(fit_rows, 0))
    Qtr = Xf[synth.train_query_rows(fit_rows, 0)]
    quant = {}
    for m in (oracle.METRIC_L2, oracle.METRIC_DOT):
        a, b, _, _ = oracle.fit_quant(oracle.lut_f32(Qtr, C, m))
        quant[m] = (a, b)
    codes = clustered_codes_host(n, M, 50)
    Xins = synth.mixture(2_000, J, 7)
    Q = synth.mixture(2 * (args.warmup + args.steps), J, 1)
    threads = parallel.host_threads()
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.encode(Xins, C)
        for j, m in enumerate((oracle.METRIC_L2, oracle.METRIC_DOT)):
            a, b = quant[m]
            luts = oracle.quantize(oracle.lut_f32(Q[2 * i + j:2 * i + j + 1], C, m), a, b)
            s_, _ = parallel.scan_topk(codes, luts, k, m, threads=threads)
            oracle.dequant(s_, a, b)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = float(np.mean(times)) * 1e3
    v = 2.0 * n / (ms * 1e-3)
    desc = ("oracle on %d host threads, per step: encode of 2,000 rows, tables and scan + top-%d + dequantize of "
            "1 L2 and 1 dot query over all %d codes (a sample of the 50M step, which has 64 + 64 queries and a "
            "1,000,064-row insert)" % (threads, k, n))
    conf = config_dict(args)
    conf["sampled"] = "per step: 2 of the 128 queries, 2,000 of the 1,000,064 insert rows"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": conf,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(args):
    from paper_1706_10283_gb300 import synth

    cfg = synth.CONFIGS["serve_50m"]
    return {"workload": "serve_50m", "n": cfg["n"], "dims": cfg["J"], "codebooks": cfg["M"],
            "code_bytes_per_vector": cfg["M"] // 2, "queries_per_step": 2 * args.large_nq, "k": 100,
            "metrics": ["l2", "dot"], "insert_rows_per_step": INSERT_ROWS,
            "launch": "one query per launch, alternating on %d CUDA streams (graph replay)" % args.large_streams,
            "l2_cache": "inputs larger than L2: every pass streams the 400 MB of codes (L2 is 129 MB)"}


def one_million_step(args, X, Q, Xd, Qd, C, quant, hbm_peak, peak_kind):
    """The 1,000,000 x 128 mixture step (encode all rows, tables of 1,000 L2
    and 1,000 dot queries, 2,000 one-query top-100 launches on several
    streams, dequantize): the codes stay in L2, so its bound is the integer
    pipe."""
    import torch

    from paper_1706_10283_gb300 import alu_peak
    from paper_1706_10283_gb300.pipeline import SearchStep

    cfg = workload(None)
    n, J, M, nq, k = cfg["n"], cfg["J"], cfg["M"], cfg["nq"], cfg["k"]
    step = SearchStep(n, J, M, nq, k, C, quant, streams=args.topk_streams)
    step.set_inputs(Xd, Qd)
    step.capture()
    for _ in range(3):
        step.replay()
    torch.cuda.synchronize()
    steps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step.replay(timed=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    per_query = step.topk_ms_per_launch()
    launch_ms = step.serial_topk_ms()
    cold_ms = step.flushed_topk_ms()
    peak = alu_peak.lookups_per_s()
    out = {"workload": "mixture_1m: 1,000,000 x 128 mixture, M=16, 1,000 queries, L2 + dot top-100, one query per "
                       "launch on %d streams" % len(step.side),
           "ms_per_step": round(ms, 4), "distances_per_s": 2.0 * nq * n / (ms * 1e-3),
           "topk_ms_per_launch": round(launch_ms, 5), "topk_ms_per_query_in_step": round(per_query, 5),
           "roofline": {"bound": "alu", "kernel": "topk_small_kernel",
                        "achieved": round(n * M / (launch_ms * 1e-3) / 1e12, 4), "peak": round(peak / 1e12, 4),
                        "unit": "Tlookup/s", "frac": round(n * M / (launch_ms * 1e-3) / peak, 4),
                        "peak_source": alu_peak.source()},
           "topk_l2_flushed": {"ms_per_launch": round(cold_ms, 5),
                               "code_GBps": round(n * M / 2 / (cold_ms * 1e-3) / 1e9, 1),
                               "hbm_frac": round(n * M / 2 / (cold_ms * 1e-3) / 1e9 / hbm_peak, 4),
                               "flush": "512 MB written before each launch (> 2x L2)"}}
    del step
    torch.cuda.empty_cache()
    return out


def small_iid_step():
    """Config 1: 10,000 x 32 i.i.d. N(0,1), M = 8, 16 queries, top-10: one
    step (encode, L2 tables, fused top-k of the 16 queries in one call,
    dequantize) replayed from a CUDA graph; latency-bound."""
    import torch

    from paper_1706_10283_gb300 import bolt, synth

    cfg = synth.CONFIGS["small_iid_l2"]
    n, J, M, nq, k = cfg["n"], cfg["J"], cfg["M"], cfg["nq"], cfg["k"]
    X = torch.from_numpy(synth.iid(n, J, 0)).cuda()
    Q = torch.from_numpy(synth.iid(nq, J, 1)).cuda()
    C = bolt.fit_codebooks(X, M, cfg["iters"], synth.kmeans_init_rows(n, 0))
    Qtr = X[torch.from_numpy(synth.train_query_rows(n, 0)).cuda()].contiguous()
    a, b, _ = bolt.fit_quantizer(Qtr, C, bolt.METRIC_L2)
    codes = torch.empty(bolt.codes_bytes(n, M), dtype=torch.uint8, device="cuda")
    luts = torch.empty((nq, M, 16), dtype=torch.uint8, device="cuda")
    ws = torch.empty(bolt.topk_workspace_bytes(n, M, nq, k), dtype=torch.uint8, device="cuda")
    os_ = torch.empty((nq, k), dtype=torch.uint16, device="cuda")
    oi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    od = torch.empty((nq, k), dtype=torch.float32, device="cuda")

    def step(s):
        bolt.encode(X, C, out=codes, stream=s)
        bolt.build_luts(Q, C, bolt.METRIC_L2, a, b, out=luts, stream=s)
        bolt.topk(codes, n, M, luts, k, bolt.METRIC_L2, os_, oi, workspace=ws, stream=s)
        bolt.dequantize(os_, a, b, out=od, stream=s)

    ms = _graph_ms(step, reps=50)
    topk_ms = _graph_ms(lambda s: bolt.topk(codes, n, M, luts, k, bolt.METRIC_L2, os_, oi, workspace=ws, stream=s),
                        reps=50)
    bolt.check_topk(oi)
    return {"workload": "small_iid_l2: 10,000 x 32 i.i.d. N(0,1), M=8, 16 queries, L2 top-10 (one top-k call)",
            "us_per_step": round(ms * 1e3, 2), "distances_per_s": nq * n / (ms * 1e-3),
            "topk_us_per_call": round(topk_ms * 1e3, 2), "timing": "CUDA graph replay, events around 50 replays"}


def approx_matmul_standalone(hbm_peak):
    """A (4096 x 512 fp32, i.i.d.) times encoded B (100,000 x 512 mixture,
    M = 32): the full 4096 x 100,000 fp32 product (Sec. 4.4), against its
    two bounds: integer lookups (4096 x 100,000 x 32) and the 1.64 GB
    output write."""
    import torch

    from paper_1706_10283_gb300 import alu_peak, bolt, synth

    mm = synth.CONFIGS["matmul_4096x512_100k"]
    rows, n, J, M = mm["rows"], mm["n"], mm["J"], mm["M"]
    B = synth.mixture_torch(n, J, seed=900)
    CB, aB, bB = bolt.fit_codebooks(B[:50_000].contiguous(), M, 8, synth.kmeans_init_rows(50_000, 900),
                                    Qtrain=B[torch.from_numpy(synth.train_query_rows(n, 900)).cuda()].contiguous(),
                                    metric=bolt.METRIC_DOT)
    codesB = bolt.encode(B, CB)
    A = torch.from_numpy(synth.iid(rows, J, 901)).cuda()
    out = torch.empty((rows, n), dtype=torch.float32, device="cuda")
    ms = _graph_ms(lambda s: bolt.approx_matmul(A, codesB, n, CB, aB, bB, out=out, stream=s), reps=5)
    lookups = rows * n * M
    peak = alu_peak.lookups_per_s()
    out_bytes = rows * n * 4
    del B, out
    torch.cuda.empty_cache()
    return {"workload": "matmul: A 4,096 x 512 fp32 x encoded B 100,000 x 512 (M=32) -> 4,096 x 100,000 fp32",
            "ms": round(ms, 4), "lookups": lookups,
            "alu_bound": {"achieved_Tlookup_s": round(lookups / (ms * 1e-3) / 1e12, 4),
                          "peak_Tlookup_s": round(peak / 1e12, 4), "frac": round(lookups / (ms * 1e-3) / peak, 4)},
            "hbm_bound": {"output_GB": round(out_bytes / 1e9, 3),
                          "achieved_GBps": round(out_bytes / (ms * 1e-3) / 1e9, 1), "peak_GBps": hbm_peak,
                          "frac": round(out_bytes / (ms * 1e-3) / 1e9 / hbm_peak, 4)}}


# dram__bytes_read.sum + dram__bytes_write.sum of one topk_kernel launch
# (ncu, one query, 8,000,000 vectors, cold caches: 64,133,888 + 11,264
# bytes, profiles/topk_kernel_mixture_8m.md) scaled by 50M / 8M; the traffic
# is the codes once, proportional to n.  None once the kernel changes.
TOPK_TRAFFIC_50M = (64_133_888 + 11_264) * 50 // 8


def roofline_topk_50m(launch_ms, n, M, hbm_peak, peak_kind, core_us):
    algo = n * M // 2  # bytes of codes one launch reads (Sec. 3.1: M/2 bytes per 4-bit code vector)
    achieved = algo / (launch_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "topk_kernel", "achieved": round(achieved, 1), "peak": hbm_peak,
            "unit": "GB/s", "frac": round(achieved / hbm_peak, 4), "traffic": TOPK_TRAFFIC_50M,
            "traffic_unit": "bytes per launch", "algorithmic_bytes": algo, "peak_kind": peak_kind,
            "launch_ms": round(launch_ms, 5),
            "timing": "one launch by itself: 20 one-query launches on one stream in a CUDA graph, events "
                      "around 10 replays",
            "lookup_core_floor": {"us_per_pass": round(core_us, 2),
                                  "frac_of_hbm": round(algo / (core_us * 1e-6) / 1e9 / hbm_peak, 4),
                                  "launch_vs_floor": round(core_us * 1e-3 / launch_ms, 4),
                                  "probe": "bolt_probe_lookup_core: the same blocks, tables and bulk-copy rings, "
                                           "sums reduced to their minimum only"}}


def run_bolt(args, world, rank, local):
    import torch

    from paper_1706_10283_gb300 import bolt, synth
    from paper_1706_10283_gb300.pipeline import SearchStep

    torch.cuda.set_device(local)
    bolt.lib()
    hbm_peak, peak_kind = peaks()
    cfg1 = workload(None)
    X, Q1, Xd, Qd, C, quant = prepare(cfg1, data_seed=rank)
    big = synth.CONFIGS["serve_50m"]
    n, J, M, k, nq = big["n"], big["J"], big["M"], 100, args.large_nq
    seed_base = 5000 + 100 * rank
    codes50 = build_50m(C, seed_base)
    row0, Xins = insert_batch(seed_base)
    Q50 = synth.mixture(nq, J, 1)
    step = SearchStep(n, J, M, nq, k, C, quant, streams=args.large_streams, codes=codes50, insert_row0=row0,
                      insert_rows=Xins.shape[0])
    step.set_inputs(Xins, torch.from_numpy(Q50).cuda())
    step.capture()

    # ---- device-resident timed region
    sampler = ClockSampler(local)
    for _ in range(args.warmup):
        step.replay()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step.replay(timed=True)
    ev1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier(world)
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    per_query = step.topk_ms_per_launch()
    for m in step.metrics:
        bolt.check_topk(step.idx[m])
    value = world * 2.0 * nq * n / (ms * 1e-3)

    # ---- end to end from pinned host buffers
    Xh = Xins.cpu().pin_memory()
    Qh = torch.from_numpy(Q50).pin_memory()
    oi = [torch.empty((nq, k), dtype=torch.int64).pin_memory() for _ in range(2)]
    od = [torch.empty((nq, k), dtype=torch.float32).pin_memory() for _ in range(2)]
    for _ in range(max(1, args.warmup)):
        step.run_from_host(Xh, Qh, oi, od)
    torch.cuda.synchronize()
    barrier(world)
    ev0.record()
    for _ in range(args.steps):
        step.run_from_host(Xh, Qh, oi, od)
    ev1.record()
    torch.cuda.synchronize()
    for t in oi:
        bolt.check_topk(t)
    ems = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    e2e = {"value": world * 2.0 * nq * n / (ems * 1e-3), "unit": UNIT, "ms_per_step": round(ems, 4),
           "h2d_bytes_per_step": step.h2d_bytes(), "d2h_bytes_per_step": step.d2h_bytes(),
           "api": "SearchStep.run_from_host (pinned host -> libbolt.so -> pinned host)"}

    # ---- roofline of the dominant kernel: one launch by itself, and the
    # bare lookup core over the same codes
    launch_ms = step.serial_topk_ms()
    core_us = bolt.probe_lookup_core(codes50, n, step.luts[bolt.METRIC_L2][0].contiguous(), reps=10)
    roof = roofline_topk_50m(launch_ms, n, M, hbm_peak, peak_kind, core_us)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": config_dict(args),
            "clocks": clocks, "e2e": e2e, "gpu_launches": args.steps * step.launches_per_step,
            "gpu_launches_per_step": step.launches_per_step, "roofline": roof,
            "topk_ms_per_query_in_step": round(per_query, 5),
            "code_GBps_in_step": round(2 * nq * n * M / 2 / (ms * 1e-3) / 1e9, 1)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import parallel

        codes_host = bolt.unpack_codes(codes50, n, M).cpu().numpy()
        Cn = C.cpu().numpy()
        Xins_h = Xh.numpy()
        v1, w1, d1 = oracle_step_sample(codes_host, Xins_h, Q50, Cn, quant, nq, k, threads=1, q_sample=1)
        nt = parallel.host_threads()
        vn, wn, dn = oracle_step_sample(codes_host, Xins_h, Q50, Cn, quant, nq, k, threads=nt, q_sample=4)
        line["cpu_baseline"] = {"value": vn, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": dn,
                                "cpu_seconds": round(wn, 2),
                                "single_thread": {"value": v1, "cores": 1, "sample": d1,
                                                  "cpu_seconds": round(w1, 2)}}
        del codes_host
    del step
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_aux:
        line["mixture_1m"] = one_million_step(args, X, Q1, Xd, Qd, C, quant, hbm_peak, peak_kind)
        line["small_iid_l2"] = small_iid_step()
        line["batch_64_on_50m"] = batch_64_on_50m(codes50, C, quant)
        line["scan_sums"] = scan_sums_report(codes50, C, quant, hbm_peak)
        line["accuracy_mixture_1m"] = accuracy_report(Xd, C, quant)
        del Xd
        line["serving"] = serving(codes50, C, quant)
        del codes50
        torch.cuda.empty_cache()
        line["encode_10m"] = encode_10m()
        line["batched_collections"] = batched_collections()
        line["approx_matmul"] = approx_matmul_standalone(hbm_peak)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_only(args):
    """Small profiling runs (for ncu): `launches` launches of one kernel after
    the workload's own setup; prints per-launch CUDA-event times."""
    import torch

    from paper_1706_10283_gb300 import bolt, synth

    torch.cuda.set_device(0)
    bolt.lib()
    if args.only == "accuracy":
        cfg = workload(8)
        X, Q, Xd, Qd, C, quant = prepare(cfg, 0)
        print(json.dumps(accuracy_report(Xd, C, quant)), flush=True)
        return
    if args.only == "large50m":
        cfg = workload(8)
        X, Q, Xd, Qd, C, quant = prepare(cfg, 0)
        del X, Xd
        codes50 = build_50m(C)
        n, M, k = 50_000_000, cfg["M"], 100
        a, b = quant[bolt.METRIC_L2]
        luts = bolt.build_luts(Qd[:8].contiguous(), C, bolt.METRIC_L2, a, b)
        ws = torch.empty(bolt.topk_workspace_bytes(n, M, 1, k), dtype=torch.uint8, device="cuda")

        def eight(s):
            for i in range(8):
                bolt.topk(codes50, n, M, luts[i:i + 1], k, bolt.METRIC_L2, workspace=ws, stream=s)

        print(json.dumps({"topk_kernel_50m_ms_per_launch": round(_graph_ms(eight, reps=3) / 8, 4),
                          "lookup_core_us": round(bolt.probe_lookup_core(codes50, n, luts[0].contiguous()), 2)}),
              flush=True)
        return
    if args.only == "serve":
        cfg = workload(8)
        X, Q, Xd, Qd, C, quant = prepare(cfg, 0)
        del X, Xd
        codes50 = build_50m(C)
        print(json.dumps(serving(codes50, C, quant)), flush=True)
        return
    if args.only == "batch":
        batch = collections_setup(args.collections)
        plan = bolt.BatchPlan([(c["codes"], c["n"], c["M"], c["luts"], c["sums"]) for c in batch])
        plan.autotune()
        print("tiles:", plan.tuning(), flush=True)
        fn = lambda: plan.run()  # noqa: E731
    elif args.only == "matmul":
        mm = synth.CONFIGS["matmul_4096x512_100k"]
        rows, n, J, M = mm["rows"], mm["n"], mm["J"], mm["M"]
        B = synth.mixture_torch(n, J, seed=900)
        CB = bolt.fit_codebooks(B[:50_000].contiguous(), M, 4, synth.kmeans_init_rows(50_000, 900))
        aB, bB, _ = bolt.fit_quantizer(B[:256].contiguous(), CB, bolt.METRIC_DOT)
        codesB = bolt.encode(B, CB)
        A = torch.from_numpy(synth.iid(rows, J, 901)).cuda()
        out = torch.empty((rows, n), dtype=torch.float32, device="cuda")
        fn = lambda: bolt.approx_matmul(A, codesB, n, CB, aB, bB, out=out)  # noqa: E731
    elif args.only in ("encode10m", "encode10m_tc"):
        cfg = synth.CONFIGS["encode_10m"]
        n, J, M = 2_000_000, cfg["J"], cfg["M"]  # 2 GB of fp32 input: > L2, small for ncu
        X = synth.mixture_torch(n, J, seed=0)
        C = bolt.fit_codebooks(X[:100_000].contiguous(), M, 4, synth.kmeans_init_rows(100_000, 0))
        codes = torch.empty(bolt.codes_bytes(n, M), dtype=torch.uint8, device="cuda")
        prec = bolt.PREC_BF16_RECHECK if args.only == "encode10m_tc" else bolt.PREC_FP32
        fn = lambda: bolt.encode(X, C, prec, out=codes)  # noqa: E731
    else:
        cfg = workload(8)
        X, Q, Xd, Qd, C, quant = prepare(cfg, 0)
        n, M, k = cfg["n"], cfg["M"], cfg["k"]
        nq = 1
        if args.only in ("topk50m", "topk8m_batch64"):
            n = 8_000_000  # 64 MB of codes: > L2/2 and well above one wave of CTAs
            Xd = synth.mixture_torch(n, cfg["J"], seed=5)
        if args.only == "topk8m_batch64":
            nq = 64
            Qd = synth.mixture_torch(nq, cfg["J"], seed=6)
        codes = bolt.encode(Xd, C)
        a, b = quant[bolt.METRIC_L2]
        luts = bolt.build_luts(Qd, C, bolt.METRIC_L2, a, b)
        ws = torch.empty(bolt.topk_workspace_bytes(n, M, nq, k), dtype=torch.uint8, device="cuda")
        fn = lambda: bolt.topk(codes, n, M, luts[:nq], k, bolt.METRIC_L2, workspace=ws)  # noqa: E731
    torch.cuda.synchronize()
    for i in range(args.launches):  # plain launches (what ncu captures)
        fn()
    torch.cuda.synchronize()
    if args.graph_reps:
        # device time per launch: `launches` calls captured in one graph
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            for i in range(args.launches):
                fn()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.graph_reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (args.graph_reps * args.launches)
        print("%s: %.4f ms per launch (%d graph-captured launches x %d replays)" %
              (args.only, ms, args.launches, args.graph_reps), flush=True)


def main():
    args = parse()
    if args.only:
        run_only(args)
        return
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_bolt(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
