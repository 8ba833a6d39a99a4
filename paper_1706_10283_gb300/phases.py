"""Per-CTA phase times of the fused top-k kernels (diagnostic).

Builds the diagnostic variant libbolt_stamps.so (-DBOLT_PHASE_STAMPS: for
query 0, thread 0 of every CTA of the top-k kernels records the global timer
at fixed points), loads it in place of libbolt.so and prints one JSON object:

  streaming_50m  topk_kernel over 50,000,000 mixture vectors (J = 128,
                 M = 16, k = 100), one query per launch, L2 and dot
  small_1m       topk_small_kernel over 1,000,000 mixture vectors

For every launch: microseconds from the first CTA's start to each phase,
as (min, median, max) over the CTAs, and the last CTA's merge phases.  The
stamped build differs from the library only by those timer reads.

    python -m paper_1706_10283_gb300.phases [--launches 3]
"""
import argparse
import ctypes as C
import json

import numpy as np

from . import bolt, synth
from . import build as _build

STREAM_PHASES = [(1, "first_threshold"), (2, "loop_end"), (3, "published")]
STREAM_LAST = [(3, "published"), (8, "counts_and_bound"), (9, "gathered"), (4, "end")]
SMALL_PHASES = [(1, "scan"), (2, "kth_bin"), (3, "kept"), (4, "sorted"), (5, "ticket")]
SMALL_LAST = [(5, "ticket"), (6, "loaded"), (7, "pool_bound"), (8, "checked"), (9, "gathered"), (10, "sorted"),
              (11, "end")]


def _read(fn):
    buf = np.zeros(1024 * 16, np.uint64)
    rc = fn(buf.ctypes.data_as(C.c_void_p), 1)
    if rc:
        raise bolt.BoltError(rc, "reading the stamps failed")
    return buf.reshape(1024, 16).astype(np.int64)


def _summary(s, phases, last_phases, end_slot, counts):
    G = int((s[:, 0] > 0).sum())
    s = s[:G]
    t0 = s[:, 0].min()
    last = int(np.argmax(s[:, end_slot]))
    rel = (s - t0) / 1e3
    out = {"ctas": G}
    for i, name in phases:
        out[name] = [round(float(np.percentile(rel[:, i], p)), 2) for p in (0, 50, 100)]
    out["last_cta"] = {name: round(float(rel[last, i]), 2) for i, name in last_phases}
    for i, name, how in counts:
        out[name] = round(float(s[:, i].mean()), 1) if how == "mean" else int(s[last, i])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--launches", type=int, default=3)
    args = ap.parse_args()
    import torch

    L = bolt.load_library(_build.build(stamps=True))
    for name in ("bolt_debug_stamps_topk", "bolt_debug_stamps_small"):
        getattr(L, name).argtypes = [C.c_void_p, C.c_int]
    torch.cuda.set_device(0)
    J, M, k = 128, 16, 100
    Xf = synth.mixture_torch(100_000, J, seed=0)
    Cb = bolt.fit_codebooks(Xf, M, 4, synth.kmeans_init_rows(100_000, 0))
    Qtr = Xf[torch.from_numpy(synth.train_query_rows(100_000, 0)).cuda()].contiguous()
    Q = torch.from_numpy(synth.mixture(16, J, 77)).cuda()
    luts = {}
    for metric in (bolt.METRIC_L2, bolt.METRIC_DOT):
        a, b, _ = bolt.fit_quantizer(Qtr, Cb, metric)
        luts[metric] = bolt.build_luts(Q, Cb, metric, a, b)
    del Xf, Qtr
    res = {}
    for n, key, reader, phases, last, end_slot, counts in (
            (50_000_000, "streaming_50m", L.bolt_debug_stamps_topk, STREAM_PHASES, STREAM_LAST, 4,
             [(5, "keys_published_mean", "mean"), (6, "merge_total", "last"), (7, "merge_survivors", "last")]),
            (1_000_000, "small_1m", L.bolt_debug_stamps_small, SMALL_PHASES, SMALL_LAST, 11,
             [(13, "ctas_fast_keep", "sum"), (14, "merge_fast", "last")])):
        codes = torch.empty(bolt.codes_bytes(n, M), dtype=torch.uint8, device="cuda")
        chunk = 1 << 21
        buf = torch.empty((min(n, chunk), J), dtype=torch.float32, device="cuda")
        for lo in range(0, n, chunk):
            hi = min(n, lo + chunk)
            X = synth.mixture_torch(hi - lo, J, seed=5000 + lo // chunk, out=buf[:hi - lo])
            bolt.encode(X, Cb, out=codes[lo // 256 * M * 128:lo // 256 * M * 128 + bolt.codes_bytes(hi - lo, M)])
        del buf
        ws = torch.empty(bolt.topk_workspace_bytes(n, M, 1, k), dtype=torch.uint8, device="cuda")
        runs = []
        for metric in (bolt.METRIC_L2, bolt.METRIC_DOT):
            for qi in range(args.launches):
                bolt.topk(codes, n, M, luts[metric][qi:qi + 1], k, metric, workspace=ws)  # warm
                torch.cuda.synchronize()
                _read(reader)  # clear
                bolt.topk(codes, n, M, luts[metric][qi:qi + 1], k, metric, workspace=ws)
                torch.cuda.synchronize()
                s = _read(reader)
                cs = [(i, nm, "mean") if how == "sum" else (i, nm, how) for i, nm, how in counts]
                out = _summary(s, phases, last, end_slot, cs)
                for i, nm, how in counts:
                    if how == "sum":
                        out[nm] = int(s[:out["ctas"], i].sum())
                runs.append(dict(metric=["l2", "dot"][metric], **out))
        res[key] = runs
        del codes, ws
        torch.cuda.empty_cache()
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
