"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the
oracle-side checks.

This module holds no Bolt arithmetic (no distances, no argmin, no tables):
it only draws vectors and the random choices the method consumes (k-means
seed rows, training-query rows), so that both sides receive identical
arrays.  The paper evaluates on Sift1M, Convnet1M, LabelMe22k and MNIST
(Sec. 4.1), which are not available here; these generators stand in for
them with the shapes of those workloads.

Recipes
-------
* ``iid(n, J, seed)``: i.i.d. N(0, 1) fp32 rows from ``numpy.random.default_rng(seed)``.
* ``mixture(n, J, seed)``: a 256-component Gaussian mixture with a decaying
  spectrum.  The mixture itself is fixed by seed 42: U is the Q factor of
  the QR decomposition of a J x J standard normal matrix (fp64; columns
  multiplied by the sign of R's diagonal), lambda_i = 1/i (i = 1..J),
  L = U diag(sqrt(lambda)), means mu_c = 2 L z_c with z_c ~ N(0, I).  A row
  draws a component c uniformly and returns mu_c + L z, z ~ N(0, I), cast
  to fp32.  ``seed`` (0 for database rows, 1 for queries) drives c and z.
* ``mixture_torch(n, J, seed, device)``: the same mixture drawn in chunks
  with torch's generator on the device, for databases of 10M+ rows (the
  values differ from the numpy draw; whichever array a test uses is handed
  to both sides).
* ``kmeans_init_rows(n, seed)``: 16 distinct row indices,
  ``default_rng(seed).choice(n, 16, replace=False)``.
* ``train_query_rows(n, seed, count=256)``: the rows of the database used as
  training queries for the lookup-table quantizer (Sec. 4.1 says a portion
  of the training database serves as queries),
  ``default_rng(seed + 1).choice(n, count, replace=False)``.
* ``collections(seed=3, count=64)``: the multi-collection batch: N log-uniform
  in [1e3, 2e6], J in {64, 128, 256}, M in {8, 16, 32}, 1..256 queries each.
* ``poisson_trace(seed, count, rate, ...)``: a serving trace: exponential
  inter-arrival times of mean 1/rate seconds, request sizes log-uniform in
  [1, max_q] queries (rounded down), metric L2 or dot with probability 1/2,
  k uniform in [k_lo, k_hi], a fraction ``matmul_frac`` of approximate-matmul
  requests; each request's queries are ``mixture(nq, J, 10_000 + i)`` rows.
"""
import math

import numpy as np

K = 16
MIX_COMPONENTS = 256
MIX_SEED = 42

_mix_cache = {}


def iid(n, J, seed):
    return np.random.default_rng(seed).standard_normal((n, J), dtype=np.float64).astype(np.float32)


def mixture_params(J):
    """(L [J x J] fp64, mu [256 x J] fp64) of the seed-42 mixture."""
    if J not in _mix_cache:
        rng = np.random.default_rng(MIX_SEED)
        G = rng.standard_normal((J, J))
        U, R = np.linalg.qr(G)
        U = U * np.sign(np.diag(R))[None, :]
        lam = 1.0 / np.arange(1, J + 1, dtype=np.float64)
        L = U * np.sqrt(lam)[None, :]
        Z = rng.standard_normal((MIX_COMPONENTS, J))
        mu = 2.0 * Z @ L.T
        _mix_cache[J] = (L, mu)
    return _mix_cache[J]


def mixture(n, J, seed, chunk=1 << 18):
    L, mu = mixture_params(J)
    rng = np.random.default_rng(seed)
    out = np.empty((n, J), np.float32)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        c = rng.integers(0, MIX_COMPONENTS, hi - lo)
        z = rng.standard_normal((hi - lo, J))
        out[lo:hi] = (mu[c] + z @ L.T).astype(np.float32)
    return out


def mixture_torch(n, J, seed, device="cuda", chunk=1 << 21, out=None):
    import torch

    L, mu = mixture_params(J)
    Lt = torch.tensor(L.T, dtype=torch.float32, device=device)
    mut = torch.tensor(mu, dtype=torch.float32, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    if out is None:
        out = torch.empty((n, J), dtype=torch.float32, device=device)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        c = torch.randint(0, MIX_COMPONENTS, (hi - lo,), generator=g, device=device)
        z = torch.randn((hi - lo, J), generator=g, device=device)
        torch.addmm(mut[c], z, Lt, out=out[lo:hi])
    return out


def kmeans_init_rows(n, seed):
    return np.random.default_rng(seed).choice(n, K, replace=False).astype(np.int64)


def train_query_rows(n, seed, count=256):
    return np.random.default_rng(seed + 1).choice(n, min(count, n), replace=False).astype(np.int64)


def collections(seed=3, count=64, n_lo=1e3, n_hi=2e6):
    """List of dicts {n, J, M, nq, data_seed, query_seed} for the batched
    multi-collection workload."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(math.floor(10 ** rng.uniform(math.log10(n_lo), math.log10(n_hi))))
        J = int(rng.choice([64, 128, 256]))
        M = int(rng.choice([8, 16, 32]))
        nq = int(rng.integers(1, 257))
        out.append(dict(n=n, J=J, M=M, nq=nq, data_seed=1000 + i, query_seed=2000 + i))
    return out


def poisson_trace(seed, count, rate, J, max_q=512, k_lo=10, k_hi=100, matmul_frac=0.0, J_mm=None, max_rows=512):
    """List of dicts {t_arrival, kind, nq, metric, k, Q} (t in seconds from 0)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        mm = matmul_frac > 0 and rng.uniform() < matmul_frac
        top = max_rows if mm else max_q
        nq = int(math.floor(2 ** rng.uniform(0, math.log2(top + 1))))
        nq = max(1, min(top, nq))
        metric = int(rng.integers(0, 2))
        k = int(rng.integers(k_lo, k_hi + 1))
        d = J_mm if mm else J
        out.append(dict(t_arrival=t, kind="matmul" if mm else "search", nq=nq, metric=metric, k=k,
                        Q=mixture(nq, d, 10_000 + i)))
    return out


# Named workloads (database size, dims, codebooks, queries, top-k).
CONFIGS = {
    "small_iid_l2": dict(n=10_000, J=32, M=8, nq=16, k=10, kind="iid", iters=16),
    "mixture_1m": dict(n=1_000_000, J=128, M=16, nq=1000, k=100, kind="mixture", iters=16),
    "encode_10m": dict(n=10_000_000, J=256, M=32, kind="mixture"),
    "serve_50m": dict(n=50_000_000, J=128, M=16, kind="mixture"),
    "matmul_4096x512_100k": dict(rows=4096, n=100_000, J=512, M=32),
}
