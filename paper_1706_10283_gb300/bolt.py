"""Thin Python binding of libbolt.so (the C ABI in include/bolt.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (torch supplies device memory and the
current stream); functions with the same names as the C entry points (minus
the ``bolt_`` prefix) allocate outputs when none are given.  There is no CPU
fallback: if the library cannot be loaded, or no CUDA device is present,
calls raise ``BoltError``.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbolt.so")

OK, EINVAL, EUNSUPPORTED, ENOMEM, ECUDA, ETIMEOUT = range(6)
METRIC_L2, METRIC_DOT, METRIC_L1, METRIC_LP = 0, 1, 2, 3
PREC_FP32, PREC_BF16_RECHECK = 0, 1
K = 16
BLOCK = 256


class BoltError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bolt error %d: %s" % (code, msg))
        self.code = code


_lib = None

_SIGS = {
    "bolt_last_error": ([], C.c_char_p),
    "bolt_probe_int_lanes": ([C.POINTER(C.c_double)], C.c_int),
    "bolt_set_wait_limit_ns": ([C.c_uint64], C.c_int),
    "bolt_topk_u32_workspace_bytes": ([C.c_int64, C.c_int32, C.c_int64, C.c_int32], C.c_int64),
    "bolt_topk_u32": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p,
                       C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "bolt_probe_lookup_core": ([C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.POINTER(C.c_float), C.c_void_p],
                               C.c_int),
    "bolt_version": ([], C.c_char_p),
    "bolt_codes_bytes": ([C.c_int64, C.c_int32], C.c_int64),
    "bolt_pack_codes": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_unpack_codes": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_encode": ([C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                     C.c_void_p], C.c_int),
    "bolt_build_luts": ([C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_float,
                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_build_luts_lp": ([C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_float, C.c_float,
                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_scan_l2": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_scan_dot": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_scan_u32": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_dequantize_u32": ([C.c_void_p, C.c_int64, C.c_float, C.c_float, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_scan_float": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_topk_workspace_bytes": ([C.c_int64, C.c_int32, C.c_int64, C.c_int32], C.c_int64),
    "bolt_topk": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p,
                   C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "bolt_topk_noalloc": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                           C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_dequant_params": ([C.c_float, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_dequantize": ([C.c_void_p, C.c_int64, C.c_float, C.c_float, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_approx_matmul": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                            C.c_float, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_fit_codebooks": ([C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                            C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_fit_quantizer": ([C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_fit_quantizer_lp": ([C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_float, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_topk_merge": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_int32, C.c_int32,
                         C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_write_codes": ([C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "bolt_topk_filter": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64, C.c_int32,
                          C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "bolt_batch_plan_bytes": ([C.c_void_p, C.c_int32], C.c_int64),
    "bolt_batch_plan": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "bolt_scan_batched": ([C.c_void_p, C.c_void_p], C.c_int),
    "bolt_batch_autotune": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p], C.c_int),
}


class Collection(C.Structure):
    """struct bolt_collection (include/bolt.h)."""

    _fields_ = [("codes", C.c_void_p), ("luts", C.c_void_p), ("sums", C.c_void_p), ("n", C.c_int64),
                ("nq", C.c_int64), ("ld", C.c_int64), ("M", C.c_int32), ("qt_max", C.c_int32),
                ("units_per_warp", C.c_int32), ("sum_bits", C.c_int32)]


def _load(path):
    L = C.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


def lib():
    """Load libbolt.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        from . import build as _build

        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise BoltError(ECUDA, "libbolt.so is not built")
        _lib = _load(LIB_PATH)
    return _lib


def load_library(path):
    """Use the library at `path` (a build of the same sources, e.g. the
    diagnostic libbolt_stamps.so) instead of libbolt.so in this process;
    call before any other function of this module."""
    global _lib
    if _lib is not None:
        raise BoltError(EINVAL, "a library is already loaded in this process")
    _lib = _load(path)
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc):
    if rc != OK:
        raise BoltError(rc, lib().bolt_last_error().decode())


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise BoltError(ECUDA, "no CUDA device: the Bolt library has no CPU path")
    return torch


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise BoltError(EINVAL, "%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise BoltError(EINVAL, "%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise BoltError(EINVAL, "%s must be contiguous" % name)
    return t


def _host_f32(b):
    arr = np.ascontiguousarray(np.asarray(b, dtype=np.float32))
    return arr, arr.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ layout
def codes_bytes(n, M):
    return int(lib().bolt_codes_bytes(n, M))


def pack_codes(rowmajor, out=None, stream=None):
    torch = _torch()
    _dev(rowmajor, torch.uint8, "rowmajor")
    n, M = rowmajor.shape
    if out is None:
        out = torch.empty(codes_bytes(n, M), dtype=torch.uint8, device=rowmajor.device)
    _check(lib().bolt_pack_codes(_ptr(rowmajor), n, M, _ptr(out), _stream(stream)))
    return out


def unpack_codes(blocked, n, M, out=None, stream=None):
    torch = _torch()
    _dev(blocked, torch.uint8, "blocked")
    if out is None:
        out = torch.empty((n, M), dtype=torch.uint8, device=blocked.device)
    _check(lib().bolt_unpack_codes(_ptr(blocked), n, M, _ptr(out), _stream(stream)))
    return out


# ------------------------------------------------------------------ encode
def encode(X, centroids, precision=PREC_FP32, out=None, n_rechecked=None, stream=None):
    torch = _torch()
    _dev(X, torch.float32, "X")
    _dev(centroids, torch.float32, "centroids")
    n, J = X.shape
    M = centroids.shape[0]
    if out is None:
        out = torch.empty(codes_bytes(n, M), dtype=torch.uint8, device=X.device)
    _check(lib().bolt_encode(_ptr(X), n, J, M, _ptr(centroids), precision, _ptr(out), _ptr(n_rechecked),
                             _stream(stream)))
    return out


# ------------------------------------------------------------------ LUT
def build_luts(Q, centroids, metric, a, b, out=None, out_f32=False, stream=None):
    """Returns uint8 tables (nq, M, 16) [and fp32 tables if out_f32]."""
    torch = _torch()
    _dev(Q, torch.float32, "Q")
    _dev(centroids, torch.float32, "centroids")
    nq, J = Q.shape
    M = centroids.shape[0]
    if out is None:
        out = torch.empty((nq, M, K), dtype=torch.uint8, device=Q.device)
    f32 = torch.empty((nq, M, K), dtype=torch.float32, device=Q.device) if out_f32 else None
    bh, bp = _host_f32(b)
    _check(lib().bolt_build_luts(_ptr(Q), nq, J, M, _ptr(centroids), metric, float(a), bp, _ptr(out), _ptr(f32),
                                 _stream(stream)))
    return (out, f32) if out_f32 else out


def build_luts_lp(Q, centroids, p, a, b, out=None, out_f32=False, stream=None):
    """L_p tables (delta = |q - c|^p, real p > 0): uint8 (nq, M, 16) [and
    fp32 tables if out_f32]; rank their sums with METRIC_LP."""
    torch = _torch()
    _dev(Q, torch.float32, "Q")
    _dev(centroids, torch.float32, "centroids")
    nq, J = Q.shape
    M = centroids.shape[0]
    if out is None:
        out = torch.empty((nq, M, K), dtype=torch.uint8, device=Q.device)
    f32 = torch.empty((nq, M, K), dtype=torch.float32, device=Q.device) if out_f32 else None
    bh, bp = _host_f32(b)
    _check(lib().bolt_build_luts_lp(_ptr(Q), nq, J, M, _ptr(centroids), float(p), float(a), bp, _ptr(out),
                                    _ptr(f32), _stream(stream)))
    return (out, f32) if out_f32 else out


# ------------------------------------------------------------------ scan / top-k
def _scan(fn, codes, n, M, luts, out, stream):
    torch = _torch()
    _dev(codes, torch.uint8, "codes")
    _dev(luts, torch.uint8, "luts")
    nq = luts.shape[0]
    if out is None:
        out = torch.empty((nq, n), dtype=torch.uint16, device=luts.device)
    _check(fn(_ptr(codes), n, M, _ptr(luts), nq, _ptr(out), _stream(stream)))
    return out


def scan_l2(codes, n, M, luts, out=None, stream=None):
    return _scan(lib().bolt_scan_l2, codes, n, M, luts, out, stream)


def scan_dot(codes, n, M, luts, out=None, stream=None):
    return _scan(lib().bolt_scan_dot, codes, n, M, luts, out, stream)


def scan_u32(codes, n, M, luts, out=None, stream=None):
    """Exact sums for any M up to 4096: (nq, n) int32 tensor holding the
    uint32 sums (all below 2^20, so the values read the same)."""
    torch = _torch()
    _dev(codes, torch.uint8, "codes")
    _dev(luts, torch.uint8, "luts")
    nq = luts.shape[0]
    if out is None:
        out = torch.empty((nq, n), dtype=torch.int32, device=luts.device)
    _dev(out, torch.int32, "out")
    _check(lib().bolt_scan_u32(_ptr(codes), n, M, _ptr(luts), nq, _ptr(out), _stream(stream)))
    return out


def scan_float(codes, n, M, luts_f32, out=None, stream=None):
    """fp32 scan over fp32 tables ("Bolt No Quantize"): (nq, n) float32."""
    torch = _torch()
    _dev(codes, torch.uint8, "codes")
    _dev(luts_f32, torch.float32, "luts_f32")
    nq = luts_f32.shape[0]
    if out is None:
        out = torch.empty((nq, n), dtype=torch.float32, device=luts_f32.device)
    _check(lib().bolt_scan_float(_ptr(codes), n, M, _ptr(luts_f32), nq, _ptr(out), _stream(stream)))
    return out


def probe_int_lanes():
    """Integer-ALU lanes per clock per SM of the current GPU (prmt loop)."""
    v = C.c_double()
    _check(lib().bolt_probe_int_lanes(C.byref(v)))
    return v.value


def probe_lookup_core(codes, n, luts, reps=10, stream=None):
    """Microseconds per pass of the bare lookup core (M = 16) over n vectors
    with one query's tables luts (16, 16) uint8: the floor of a one-query
    fused scan + top-k."""
    torch = _torch()
    _dev(codes, torch.uint8, "codes")
    _dev(luts, torch.uint8, "luts")
    v = C.c_float()
    _check(lib().bolt_probe_lookup_core(_ptr(codes), n, _ptr(luts), reps, C.byref(v), _stream(stream)))
    return float(v.value)


def topk_workspace_bytes(n, M, nq, k):
    v = int(lib().bolt_topk_workspace_bytes(n, M, nq, k))
    if v < 0:
        raise BoltError(EINVAL, lib().bolt_last_error().decode())
    return v


TIMED_OUT = -2  # index of every entry of a row whose bounded device wait gave up


def check_topk(idx):
    """Raise BoltError(ETIMEOUT) if any row of a top-k index array (torch
    tensor or numpy array, (nq, k)) is marked as timed out (index -2 in
    column 0: a bounded wait on the GPU gave up and the row is invalid).
    A device tensor is read back, which waits for its stream."""
    if idx.shape[0] == 0 or idx.shape[1] == 0:
        return
    col = idx[:, 0]
    bad = col == TIMED_OUT
    nbad = int(bad.sum())
    if nbad:
        raise BoltError(ETIMEOUT, "%d of %d top-k rows timed out on the GPU (a bounded wait gave up; index -2)"
                        % (nbad, idx.shape[0]))


def topk(codes, n, M, luts, k, metric, out_sums=None, out_idx=None, workspace=None, stream=None, check=False):
    """(sums uint16 (nq, k), idx int64 (nq, k)), best first.  A row whose
    bounded device wait gave up holds index -2 everywhere; check=True waits
    for the result and raises BoltError(ETIMEOUT) for such rows (otherwise
    call check_topk on the result before using it)."""
    torch = _torch()
    _dev(codes, torch.uint8, "codes")
    _dev(luts, torch.uint8, "luts")
    nq = luts.shape[0]
    dev = luts.device
    if out_sums is None:
        out_sums = torch.empty((nq, k), dtype=torch.uint16, device=dev)
    if out_idx is None:
        out_idx = torch.empty((nq, k), dtype=torch.int64, device=dev)
    wbytes = workspace.numel() if workspace is not None else 0
    _check(lib().bolt_topk(_ptr(codes), n, M, _ptr(luts), nq, k, metric, _ptr(out_sums), _ptr(out_idx),
                           _ptr(workspace), wbytes, _stream(stream)))
    if check:
        check_topk(out_idx)
    return out_sums, out_idx


def topk_u32_workspace_bytes(n, M, nq, k):
    v = int(lib().bolt_topk_u32_workspace_bytes(n, M, nq, k))
    if v < 0:
        raise BoltError(EINVAL, lib().bolt_last_error().decode())
    return v


def topk_u32(codes, n, M, luts, k, metric, out_sums=None, out_idx=None, workspace=None, stream=None):
    """Top-k for up to 4096 codebooks: (sums (nq, k) int32 tensor holding the
    uint32 sums (all below 2^20), idx int64 (nq, k)), best first."""
    torch = _torch()
    _dev(codes, torch.uint8, "codes")
    _dev(luts, torch.uint8, "luts")
    nq = luts.shape[0]
    dev = luts.device
    if out_sums is None:
        out_sums = torch.empty((nq, k), dtype=torch.int32, device=dev)
    if out_idx is None:
        out_idx = torch.empty((nq, k), dtype=torch.int64, device=dev)
    wbytes = workspace.numel() if workspace is not None else 0
    _check(lib().bolt_topk_u32(_ptr(codes), n, M, _ptr(luts), nq, k, metric, _ptr(out_sums), _ptr(out_idx),
                               _ptr(workspace), wbytes, _stream(stream)))
    return out_sums, out_idx


def topk_merge(sums, idx, offsets, M, metric, out_sums=None, out_idx=None, stream=None):
    """Merge per-shard top-k lists: sums (nshard, nq, k) uint16, idx (nshard,
    nq, k) int64 local indices, offsets (nshard,) int64 device tensor of
    global row offsets.  Returns (sums, idx) of shape (nq, k)."""
    torch = _torch()
    _dev(sums, torch.uint16, "sums")
    _dev(idx, torch.int64, "idx")
    _dev(offsets, torch.int64, "offsets")
    nshard, nq, k = idx.shape
    if out_sums is None:
        out_sums = torch.empty((nq, k), dtype=torch.uint16, device=idx.device)
    if out_idx is None:
        out_idx = torch.empty((nq, k), dtype=torch.int64, device=idx.device)
    _check(lib().bolt_topk_merge(_ptr(sums), _ptr(idx), _ptr(offsets), nshard, nq, k, M, metric, _ptr(out_sums),
                                 _ptr(out_idx), _stream(stream)))
    return out_sums, out_idx


def write_codes(rowmajor, rows, blocked, n_cap, stream=None):
    """Write row-major codes (count, M) uint8 into rows (count,) int64 of a
    blocked code array with room for n_cap vectors."""
    torch = _torch()
    _dev(rowmajor, torch.uint8, "rowmajor")
    _dev(rows, torch.int64, "rows")
    _dev(blocked, torch.uint8, "blocked")
    count, M = rowmajor.shape
    _check(lib().bolt_write_codes(_ptr(rowmajor), count, M, _ptr(rows), _ptr(blocked), n_cap, _stream(stream)))


def topk_filter(sums, idx, dead_bits, n_bits, k_out, stream=None):
    """Keep the first k_out live entries of each top-k list (dead_bits: int32
    tensor viewed as a bitmap of dead rows)."""
    torch = _torch()
    _dev(sums, torch.uint16, "sums")
    _dev(idx, torch.int64, "idx")
    _dev(dead_bits, torch.int32, "dead_bits")
    nq, k_in = idx.shape
    out_s = torch.empty((nq, k_out), dtype=torch.uint16, device=idx.device)
    out_i = torch.empty((nq, k_out), dtype=torch.int64, device=idx.device)
    _check(lib().bolt_topk_filter(_ptr(sums), _ptr(idx), nq, k_in, _ptr(dead_bits), n_bits, k_out, _ptr(out_s),
                                  _ptr(out_i), _stream(stream)))
    return out_s, out_i


# ------------------------------------------------------------------ dequantize / matmul
def dequant_params(a, b):
    bh, bp = _host_f32(b)
    ia, bias = C.c_float(), C.c_float()
    _check(lib().bolt_dequant_params(float(a), bp, bh.shape[0], C.byref(ia), C.byref(bias)))
    return ia.value, bias.value


def dequantize(S, a, b, out=None, stream=None):
    torch = _torch()
    _dev(S, torch.uint16, "S")
    inv_a, bias = dequant_params(a, b)
    if out is None:
        out = torch.empty(S.shape, dtype=torch.float32, device=S.device)
    _check(lib().bolt_dequantize(_ptr(S), S.numel(), inv_a, bias, _ptr(out), _stream(stream)))
    return out


def dequantize_u32(S, a, b, out=None, stream=None):
    """Dequantize uint32 sums held in an int32 tensor (scan_u32's output)."""
    torch = _torch()
    _dev(S, torch.int32, "S")
    inv_a, bias = dequant_params(a, b)
    if out is None:
        out = torch.empty(S.shape, dtype=torch.float32, device=S.device)
    _check(lib().bolt_dequantize_u32(_ptr(S), S.numel(), inv_a, bias, _ptr(out), _stream(stream)))
    return out


def approx_matmul(A, codesB, n, centroids, a, b, out=None, stream=None):
    torch = _torch()
    _dev(A, torch.float32, "A")
    _dev(codesB, torch.uint8, "codesB")
    _dev(centroids, torch.float32, "centroids")
    rows, J = A.shape
    M = centroids.shape[0]
    if out is None:
        out = torch.empty((rows, n), dtype=torch.float32, device=A.device)
    bh, bp = _host_f32(b)
    _check(lib().bolt_approx_matmul(_ptr(A), rows, J, _ptr(codesB), n, M, _ptr(centroids), float(a), bp,
                                    _ptr(out), _stream(stream)))
    return out


# ------------------------------------------------------------------ fit
def fit_codebooks(X, M, iters, init_rows, Qtrain=None, metric=METRIC_L2, stream=None):
    """Returns centroids (M, 16, J/M) and, with Qtrain, (a, b)."""
    torch = _torch()
    _dev(X, torch.float32, "X")
    n, J = X.shape
    cent = torch.empty((M, K, J // M), dtype=torch.float32, device=X.device)
    rows = np.ascontiguousarray(init_rows, dtype=np.int64)
    a = C.c_float(0.0)
    b = np.zeros(M, np.float32)
    nqt = 0 if Qtrain is None else Qtrain.shape[0]
    if Qtrain is not None:
        _dev(Qtrain, torch.float32, "Qtrain")
    _check(lib().bolt_fit_codebooks(_ptr(X), n, J, M, iters, rows.ctypes.data_as(C.c_void_p), _ptr(Qtrain), nqt,
                                    metric, _ptr(cent), C.byref(a), b.ctypes.data_as(C.c_void_p),
                                    _stream(stream)))
    if Qtrain is None:
        return cent
    return cent, np.float32(a.value), b


def fit_quantizer(Qtrain, centroids, metric, stream=None):
    """Returns (a, b[M], alpha_index)."""
    torch = _torch()
    _dev(Qtrain, torch.float32, "Qtrain")
    _dev(centroids, torch.float32, "centroids")
    nqt, J = Qtrain.shape
    M = centroids.shape[0]
    a = C.c_float(0.0)
    b = np.zeros(M, np.float32)
    ai = C.c_int32(0)
    _check(lib().bolt_fit_quantizer(_ptr(Qtrain), nqt, J, M, _ptr(centroids), metric, C.byref(a),
                                    b.ctypes.data_as(C.c_void_p), C.byref(ai), _stream(stream)))
    return np.float32(a.value), b, int(ai.value)


def fit_quantizer_lp(Qtrain, centroids, p, stream=None):
    """The quantizer fit over L_p tables: (a, b[M], alpha_index)."""
    torch = _torch()
    _dev(Qtrain, torch.float32, "Qtrain")
    _dev(centroids, torch.float32, "centroids")
    nqt, J = Qtrain.shape
    M = centroids.shape[0]
    a = C.c_float(0.0)
    b = np.zeros(M, np.float32)
    ai = C.c_int32(0)
    _check(lib().bolt_fit_quantizer_lp(_ptr(Qtrain), nqt, J, M, _ptr(centroids), float(p), C.byref(a),
                                       b.ctypes.data_as(C.c_void_p), C.byref(ai), _stream(stream)))
    return np.float32(a.value), b, int(ai.value)


# ------------------------------------------------------------------ batched scan
def sums_ld(n):
    """Row stride (uint16 entries) of a batched-scan sums matrix: n rounded up to 8."""
    return (n + 7) // 8 * 8


class BatchPlan:
    """A device-resident task list over many collections (bolt_batch_plan).

    ``entries`` is a list of (codes, n, M, luts, sums) with torch CUDA
    tensors: codes blocked, luts (nq, M, 16) uint8, sums (nq, sums_ld(n))
    uint16, or int32 holding the uint32 sums (required for M > 256, up to
    4096 codebooks).  The plan keeps references to the tensors so their
    memory stays alive while the plan exists.
    """

    def __init__(self, entries, tuning=None, stream=None):
        torch = _torch()
        self._keep = []
        arr = (Collection * max(1, len(entries)))()
        for i, (codes, n, M, luts, sums) in enumerate(entries):
            _dev(codes, torch.uint8, "codes")
            _dev(luts, torch.uint8, "luts")
            wide = sums.dtype == torch.int32
            _dev(sums, torch.int32 if wide else torch.uint16, "sums")
            nq = luts.shape[0]
            ld = sums.shape[1] if sums.dim() == 2 else sums_ld(n)
            arr[i] = Collection(codes.data_ptr(), luts.data_ptr(), sums.data_ptr(), n, nq, ld, M, 0, 0,
                                32 if wide else 0)
            if tuning is not None:
                arr[i].qt_max, arr[i].units_per_warp = tuning[i]
            self._keep += [codes, luts, sums]
        self.ncoll = len(entries)
        self.colls = arr
        self.device = entries[0][0].device if entries else torch.device("cuda")
        self._upload(stream)

    def tuning(self):
        return [(self.colls[i].qt_max, self.colls[i].units_per_warp) for i in range(self.ncoll)]

    def _upload(self, stream):
        torch = _torch()
        nbytes = int(lib().bolt_batch_plan_bytes(C.cast(self.colls, C.c_void_p), self.ncoll))
        if nbytes < 0:
            raise BoltError(-nbytes, lib().bolt_last_error().decode())
        self.plan = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        _check(lib().bolt_batch_plan(C.cast(self.colls, C.c_void_p), self.ncoll, _ptr(self.plan), self.plan.numel(),
                                     _stream(stream)))

    def autotune(self, stream=None):
        """Time the candidates (bolt_batch_autotune), keep the fastest, re-plan.
        Returns the batch time (ms) with the chosen settings."""
        ms = C.c_float(0.0)
        _check(lib().bolt_batch_autotune(C.cast(self.colls, C.c_void_p), self.ncoll, _stream(stream), C.byref(ms)))
        self._upload(stream)
        return ms.value

    def run(self, stream=None):
        _check(lib().bolt_scan_batched(_ptr(self.plan), _stream(stream)))
