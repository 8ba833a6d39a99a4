"""Bolt CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct CPU restatement of Bolt (Blalock & Guttag,
KDD'17) used to check the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` legs may import this package; the product path
(``paper_1706_10283_gb300``) never does and shares no code with it.

All arithmetic lives in ``bolt_oracle.c`` (see its header for every reading
of the paper it takes); this module only marshals numpy arrays.

Parity status: every function is pinned by ``tests/test_oracle.py`` against
brute force, closed forms, library routines or hand-computed golden values.
The quantizer fit's selection rule (the grid alpha of least loss, ties to the
smaller alpha) is pinned against independently computed losses; the alpha it
picks on realistic data has no worked value in the paper to compare with.

``oracle.parallel`` runs the same functions on row ranges in host threads (the
timed CPU baseline); it adds no arithmetic of its own beyond taking the best k
of the per-range lists with ``topk``.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

METRIC_L2 = 0
METRIC_DOT = 1
METRIC_L1 = 2
METRIC_LP = 3  # |q - c|^p tables (lut_lp_f32 / lut_lp_f64), ranked ascending
K = 16
ALPHAS = (0.0, 0.001, 0.002, 0.005, 0.01, 0.02, 0.05, 0.1)

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64, i32, f32 = C.c_int64, C.c_int32, C.c_float
        sig = {
            "bo_encode_f32": [f32p, i64, i32, i32, f32p, u8p],
            "bo_encode_f64": [f32p, i64, i32, i32, f32p, u8p],
            "bo_decode": [u8p, i64, i32, i32, f32p, f32p],
            "bo_kmeans": [f32p, i64, i32, i32, i32, i64p, f32p, C.c_void_p],
            "bo_lut_f32": [f32p, i64, i32, i32, f32p, i32, f32p],
            "bo_lut_f64": [f32p, i64, i32, i32, f32p, i32, f64p],
            "bo_lut_lp_f32": [f32p, i64, i32, i32, f32p, C.c_float, f32p],
            "bo_lut_lp_f64": [f32p, i64, i32, i32, f32p, C.c_float, f64p],
            "bo_quantize": [f32p, i64, i32, f32, f32p, u8p],
            "bo_quant_params": [f32p, i64, i32, i32, C.POINTER(C.c_double), f64p],
            "bo_fit_quant": [f32p, i64, i32, C.POINTER(C.c_float), f32p, C.POINTER(C.c_int32), f64p],
            "bo_scan": [u8p, i64, i32, u8p, i64, u16p],
            "bo_scan_u32": [u8p, i64, i32, u8p, i64, u32p],
            "bo_dequant_u32": [u32p, i64, f32, f32, f32p],
            "bo_scan_float": [u8p, i64, i32, f32p, i64, f32p],
            "bo_topk": [u16p, i64, i64, i32, i32, u16p, i64p],
            "bo_topk_u32": [u32p, i64, i64, i32, i32, u32p, i64p],
            "bo_dequant_params": [f32, f32p, i32, C.POINTER(C.c_float), C.POINTER(C.c_float)],
            "bo_dequant": [u16p, i64, f32, f32, f32p],
            "bo_matmul": [f32p, i64, i32, u8p, i64, i32, f32p, f32, f32p, f32p],
        }
        for name, args in sig.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        del i32p
    return _lib


class OracleError(RuntimeError):
    pass


def _ok(rc, name):
    if rc != 0:
        raise OracleError("%s returned %d" % (name, rc))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def encode(X, C_, precision="f32"):
    """Row-major n x M codes (one 0..15 code per byte).  Sec. 3.1, h."""
    X, C_ = _f32(X), _f32(C_)
    n, J = X.shape
    M = C_.shape[0]
    codes = np.empty((n, M), np.uint8)
    fn = lib().bo_encode_f32 if precision == "f32" else lib().bo_encode_f64
    _ok(fn(X, n, J, M, C_, codes), "encode")
    return codes


def decode(codes, C_):
    """Reconstruction x_hat (Sec. 3.3 definition)."""
    codes, C_ = _u8(codes), _f32(C_)
    n, M = codes.shape
    s = C_.shape[2]
    out = np.empty((n, M * s), np.float32)
    _ok(lib().bo_decode(codes, n, M * s, M, C_, out), "decode")
    return out


def kmeans(X, M, iters, init_rows, return_objective=False):
    """Centroids M x 16 x s (fp32).  init_rows: 16 distinct row indices."""
    X = _f32(X)
    n, J = X.shape
    s = J // M
    C_ = np.empty((M, K, s), np.float32)
    rows = np.ascontiguousarray(init_rows, dtype=np.int64)
    assert rows.shape == (K,)
    obj = np.empty(iters + 1, np.float64)
    _ok(lib().bo_kmeans(X, n, J, M, iters, rows, C_, obj.ctypes.data), "kmeans")
    return (C_, obj) if return_objective else C_


def lut_f32(Q, C_, metric):
    """Float table D, nq x M x 16 (Sec. 3.1 query encoding)."""
    Q, C_ = _f32(Q), _f32(C_)
    nq, J = Q.shape
    M = C_.shape[0]
    D = np.empty((nq, M, K), np.float32)
    _ok(lib().bo_lut_f32(Q, nq, J, M, C_, metric, D), "lut_f32")
    return D


def lut_f64(Q, C_, metric):
    Q, C_ = _f32(Q), _f32(C_)
    nq, J = Q.shape
    M = C_.shape[0]
    D = np.empty((nq, M, K), np.float64)
    _ok(lib().bo_lut_f64(Q, nq, J, M, C_, metric, D), "lut_f64")
    return D


def lut_lp_f32(Q, C_, p):
    """L_p table (delta = |q - c|^p, real p > 0), fp32: C library powf per
    dim, fp32 adds in dim order."""
    Q, C_ = _f32(Q), _f32(C_)
    nq, J = Q.shape
    M = C_.shape[0]
    D = np.empty((nq, M, K), np.float32)
    _ok(lib().bo_lut_lp_f32(Q, nq, J, M, C_, float(p), D), "lut_lp_f32")
    return D


def lut_lp_f64(Q, C_, p):
    Q, C_ = _f32(Q), _f32(C_)
    nq, J = Q.shape
    M = C_.shape[0]
    D = np.empty((nq, M, K), np.float64)
    _ok(lib().bo_lut_lp_f64(Q, nq, J, M, C_, float(p), D), "lut_lp_f64")
    return D


def quantize(D, a, b):
    """uint8 tables beta_m(D) (Sec. 3.2)."""
    D = _f32(D)
    nq, M, _ = D.shape
    out = np.empty((nq, M, K), np.uint8)
    _ok(lib().bo_quantize(D, nq, M, float(a), _f32(b), out), "quantize")
    return out


def fit_quant(Dtrain):
    """Returns (a, b[M], alpha_index, losses[8]) fitted on training tables."""
    Dtrain = _f32(Dtrain)
    ntq, M, _ = Dtrain.shape
    a = C.c_float()
    b = np.empty(M, np.float32)
    ai = C.c_int32()
    losses = np.empty(8, np.float64)
    _ok(lib().bo_fit_quant(Dtrain, ntq, M, C.byref(a), b, C.byref(ai), losses), "fit_quant")
    return np.float32(a.value), b, int(ai.value), losses


def quant_params(Dtrain, alpha_idx):
    """fp64 (a, b[M]) for grid point alpha_idx, before any fp32 rounding."""
    Dtrain = _f32(Dtrain)
    ntq, M, _ = Dtrain.shape
    a = C.c_double()
    b = np.empty(M, np.float64)
    _ok(lib().bo_quant_params(Dtrain, ntq, M, int(alpha_idx), C.byref(a), b), "quant_params")
    return a.value, b


def scan(codes, luts):
    """Exact uint16 sums, nq x n."""
    codes, luts = _u8(codes), _u8(luts)
    n, M = codes.shape
    nq = luts.shape[0]
    assert luts.shape == (nq, M, K)
    out = np.empty((nq, n), np.uint16)
    _ok(lib().bo_scan(codes, n, M, luts, nq, out), "scan")
    return out


def scan_u32(codes, luts):
    """Exact uint32 sums, nq x n (any M up to 4096)."""
    codes, luts = _u8(codes), _u8(luts)
    n, M = codes.shape
    nq = luts.shape[0]
    assert luts.shape == (nq, M, K)
    out = np.empty((nq, n), np.uint32)
    _ok(lib().bo_scan_u32(codes, n, M, luts, nq, out), "scan_u32")
    return out


def dequant_u32(S, a, b):
    S = np.ascontiguousarray(S, dtype=np.uint32)
    inv_a, bias = dequant_params(a, b)
    out = np.empty(S.shape, np.float32)
    _ok(lib().bo_dequant_u32(S.reshape(-1), S.size, inv_a, bias, out.reshape(-1)), "dequant_u32")
    return out


def scan_float(codes, D):
    codes, D = _u8(codes), _f32(D)
    n, M = codes.shape
    nq = D.shape[0]
    out = np.empty((nq, n), np.float32)
    _ok(lib().bo_scan_float(codes, n, M, D, nq, out), "scan_float")
    return out


def topk(sums, k, metric):
    """(sums nq x k uint16, idx nq x k int64), sorted best first."""
    sums = np.ascontiguousarray(sums, dtype=np.uint16)
    nq, n = sums.shape
    os_ = np.empty((nq, k), np.uint16)
    oi = np.empty((nq, k), np.int64)
    _ok(lib().bo_topk(sums, n, nq, k, metric, os_, oi), "topk")
    return os_, oi


def topk_u32(sums, k, metric):
    """top-k over uint32 sums (more than 256 codebooks): (sums nq x k uint32,
    idx nq x k int64), best first, ties to the lower index."""
    sums = np.ascontiguousarray(sums, dtype=np.uint32)
    nq, n = sums.shape
    os_ = np.empty((nq, k), np.uint32)
    oi = np.empty((nq, k), np.int64)
    _ok(lib().bo_topk_u32(sums, n, nq, k, metric, os_, oi), "topk_u32")
    return os_, oi


def dequant_params(a, b):
    b = _f32(b)
    ia, bias = C.c_float(), C.c_float()
    _ok(lib().bo_dequant_params(float(a), b, b.shape[0], C.byref(ia), C.byref(bias)), "dequant_params")
    return np.float32(ia.value), np.float32(bias.value)


def dequant(S, a, b):
    S = np.ascontiguousarray(S, dtype=np.uint16)
    inv_a, bias = dequant_params(a, b)
    out = np.empty(S.shape, np.float32)
    _ok(lib().bo_dequant(S.reshape(-1), S.size, inv_a, bias, out.reshape(-1)), "dequant")
    return out


def matmul(A, codesB, C_, a, b):
    A, codesB, C_ = _f32(A), _u8(codesB), _f32(C_)
    rows, J = A.shape
    n, M = codesB.shape
    out = np.empty((rows, n), np.float32)
    _ok(lib().bo_matmul(A, rows, J, codesB, n, M, C_, float(a), _f32(b), out), "matmul")
    return out


def lib_path():
    return os.path.abspath(_build.LIB)
