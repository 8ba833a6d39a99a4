"""Pins for the CPU oracle against facts that do not come from the oracle:
brute force, closed forms, library routines (scipy), invariants the paper
states (Sec. 3.1 subspace decomposition, Sec. 3.3 lemmas), hand-derived
values and the numbers the paper prints (tests/golden/paper_numbers.json).

Each test is chosen so that a plausible slip in bolt_oracle.c (a dropped
term, a wrong sign or index, a transposed operand, a wrong tie rule) fails.
"""
import json
import os

import numpy as np
import pytest
import scipy.cluster.vq as vq
from scipy.spatial.distance import cdist

import oracle
from paper_1706_10283_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def blobs(n, J, seed, spread=0.05, centers=16):
    """Well separated clusters: no near-ties in the argmin."""
    rng = np.random.default_rng(seed)
    cen = rng.standard_normal((centers, J)) * 4.0
    lab = rng.integers(0, centers, n)
    return (cen[lab] + spread * rng.standard_normal((n, J))).astype(np.float32)


def fp64_dists(X, C):
    """(n, M, 16) squared distances in fp64 by a library routine."""
    n, J = X.shape
    M, K, s = C.shape
    out = np.empty((n, M, K))
    for m in range(M):
        out[:, m, :] = cdist(X[:, m * s:(m + 1) * s].astype(np.float64), C[m].astype(np.float64), "sqeuclidean")
    return out


# ------------------------------------------------------------------ paper numbers
def test_paper_numbers_code_size():
    """Sec. 4.6 compression ratios follow from M/2 bytes per 4-bit code vector."""
    g = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))
    assert g["centroids_per_codebook"]["value"] == oracle.K == 16
    assert tuple(g["alpha_grid"]["value"]) == oracle.ALPHAS
    for key, nbytes in (("compression_ratios_8B", 8), ("compression_ratios_32B", 32)):
        for J, ratio in g[key]["value"].items():
            M = 2 * nbytes  # 4-bit codes: two codebooks per byte
            assert int(J) * 4 // nbytes == ratio
            # the oracle's code array holds M codes per vector
            X = blobs(3, int(J) - int(J) % M if int(J) % M else int(J), 0)
            if X.shape[1] % M == 0:
                C = np.zeros((M, 16, X.shape[1] // M), np.float32)
                assert oracle.encode(X, C).shape == (3, M)


# ------------------------------------------------------------------ encoder
def test_encode_matches_fp64_bruteforce():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((500, 24)).astype(np.float32)
    C = rng.standard_normal((4, 16, 6)).astype(np.float32)
    d = fp64_dists(X, C)
    ref = d.argmin(axis=2)
    srt = np.sort(d, axis=2)
    clear = (srt[:, :, 1] - srt[:, :, 0]) > 1e-4 * (1 + srt[:, :, 0])
    got32 = oracle.encode(X, C)
    got64 = oracle.encode(X, C, precision="f64")
    assert clear.mean() > 0.95
    np.testing.assert_array_equal(got32[clear], ref[clear])
    np.testing.assert_array_equal(got64[clear], ref[clear])


def test_encode_m1_is_scipy_vq():
    """With M = 1 the encoder is plain nearest-centroid assignment."""
    X = blobs(400, 8, 2)
    C = X[:16].reshape(1, 16, 8).copy() + np.float32(0.01)
    ref, _ = vq.vq(X.astype(np.float64), C[0].astype(np.float64))
    np.testing.assert_array_equal(oracle.encode(X, C)[:, 0], ref)


def test_encode_centroid_points_and_ties():
    rng = np.random.default_rng(3)
    C = rng.standard_normal((3, 16, 5)).astype(np.float32)
    want = rng.integers(0, 16, (40, 3))
    X = np.concatenate([C[m, want[:, m]] for m in range(3)], axis=1)
    np.testing.assert_array_equal(oracle.encode(X, C), want)
    # duplicated centroid: the lower index wins
    C2 = C.copy()
    C2[1, 11] = C2[1, 4]
    X2 = np.concatenate([C2[0, [0]], C2[1, [11]], C2[2, [7]]], axis=1)
    assert oracle.encode(X2, C2).tolist() == [[0, 4, 7]]
    # hand example: J = 2, M = 2, x = (0.4, -2) picks centroid 0 in m=0
    # (|0.4-0|^2 = .16 < |0.4-1|^2 = .36) and centroid 2 in m=1 (exact hit)
    C3 = np.zeros((2, 16, 1), np.float32) + 100
    C3[0, 0, 0], C3[0, 1, 0] = 0.0, 1.0
    C3[1, 2, 0], C3[1, 3, 0] = -2.0, -1.0
    assert oracle.encode(np.array([[0.4, -2.0]], np.float32), C3).tolist() == [[0, 2]]


def test_decode_is_centroid_lookup():
    """Sec. 3.3 reconstruction: x_hat^(m) = c_{h(x)_m}^(m)."""
    rng = np.random.default_rng(4)
    C = rng.standard_normal((4, 16, 3)).astype(np.float32)
    X = rng.standard_normal((50, 12)).astype(np.float32)
    codes = oracle.encode(X, C)
    xh = oracle.decode(codes, C)
    ref = np.concatenate([C[m][codes[:, m]] for m in range(4)], axis=1)
    np.testing.assert_array_equal(xh, ref)
    # and the code of the reconstruction is the code itself
    np.testing.assert_array_equal(oracle.encode(xh, C), codes)


# ------------------------------------------------------------------ k-means
def test_kmeans_m1_matches_scipy_kmeans2():
    X = blobs(2000, 6, 5, spread=0.3)
    rows = synth.kmeans_init_rows(len(X), 0)
    C, obj = oracle.kmeans(X, 1, 8, rows, return_objective=True)
    ref, _ = vq.kmeans2(X.astype(np.float64), X[rows].astype(np.float64), iter=8, minit="matrix",
                        missing="warn")
    np.testing.assert_allclose(C[0], ref, rtol=1e-6, atol=1e-6)


def test_kmeans_subspaces_are_independent():
    """Consecutive-dims partition (Sec. 3.1): M codebooks == M separate
    1-codebook fits on the column blocks, with the same seed rows."""
    X = synth.iid(3000, 12, 7)
    rows = synth.kmeans_init_rows(len(X), 7)
    C = oracle.kmeans(X, 3, 5, rows)
    for m in range(3):
        Cm = oracle.kmeans(np.ascontiguousarray(X[:, 4 * m:4 * m + 4]), 1, 5, rows)
        np.testing.assert_array_equal(C[m], Cm[0])


def test_kmeans_objective_nonincreasing():
    X = synth.mixture(4000, 16, 0)
    rows = synth.kmeans_init_rows(len(X), 0)
    _, obj = oracle.kmeans(X, 4, 10, rows, return_objective=True)
    assert np.all(np.diff(obj) <= 1e-6 * obj[:-1])
    assert obj[-1] < obj[0]


def test_kmeans_empty_cluster_keeps_centroid():
    # 17 rows: 16 seeds, two of them identical -> the duplicate cluster is
    # never chosen (ties go to the lower index) and must keep its seed.
    X = np.arange(16, dtype=np.float32).reshape(16, 1) * 10
    X = np.concatenate([X, X[:1]], 0)
    rows = np.arange(16)
    rows = rows.copy()
    rows[5] = 16  # row 16 duplicates row 0
    C = oracle.kmeans(X, 1, 3, rows)
    assert C[0, 5, 0] == 0.0  # seed value kept
    assert C[0, 0, 0] == 0.0


# ------------------------------------------------------------------ LUT g
@pytest.mark.parametrize("metric", [oracle.METRIC_L2, oracle.METRIC_DOT, oracle.METRIC_L1])
def test_lut_decomposition_equals_distance_to_reconstruction(metric):
    """Sec. 3.1: the sum over subspaces of the table entries picked by the
    codes equals the distance between q and the reconstruction x_hat."""
    rng = np.random.default_rng(8)
    C = rng.standard_normal((8, 16, 4)).astype(np.float32)
    X = rng.standard_normal((300, 32)).astype(np.float32)
    Q = rng.standard_normal((7, 32)).astype(np.float32)
    codes = oracle.encode(X, C)
    xh = oracle.decode(codes, C).astype(np.float64)
    D = oracle.lut_f64(Q, C, metric)
    got = D[:, np.arange(8)[None, :], codes].sum(axis=2)  # (nq, n)
    if metric == oracle.METRIC_L2:
        ref = cdist(Q.astype(np.float64), xh, "sqeuclidean")
    elif metric == oracle.METRIC_L1:
        ref = cdist(Q.astype(np.float64), xh, "cityblock")
    else:
        ref = Q.astype(np.float64) @ xh.T
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    D32 = oracle.lut_f32(Q, C, metric)
    scale = np.abs(Q).max() * np.abs(C).max() * 4 + (D if metric != oracle.METRIC_DOT else 0)
    assert np.all(np.abs(D32 - D) <= 1e-5 * np.maximum(1.0, np.abs(D)) * 4 + 1e-6 * scale)


def test_lut_matches_cdist_per_subspace():
    rng = np.random.default_rng(9)
    C = rng.standard_normal((4, 16, 8)).astype(np.float32)
    Q = rng.standard_normal((5, 32)).astype(np.float32)
    D = oracle.lut_f64(Q, C, oracle.METRIC_L2)
    Dd = oracle.lut_f64(Q, C, oracle.METRIC_DOT)
    D1 = oracle.lut_f64(Q, C, oracle.METRIC_L1)
    D1f = oracle.lut_f32(Q, C, oracle.METRIC_L1)
    for m in range(4):
        q = Q[:, 8 * m:8 * m + 8].astype(np.float64)
        np.testing.assert_allclose(D[:, m, :], cdist(q, C[m].astype(np.float64), "sqeuclidean"), rtol=1e-13)
        np.testing.assert_allclose(Dd[:, m, :], q @ C[m].astype(np.float64).T, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(D1[:, m, :], cdist(q, C[m].astype(np.float64), "cityblock"), rtol=1e-13)
        # fp32 entry: 8 fp32 subtractions and adds, each within half an ulp
        np.testing.assert_allclose(D1f[:, m, :], D1[:, m, :], rtol=8 * 2.0 ** -23)


def test_lut_exact_when_x_is_made_of_centroids():
    """x_hat = x when every subvector is a centroid: the table sum is the
    exact distance (up to the fp32 rounding of the table)."""
    rng = np.random.default_rng(10)
    C = (rng.integers(-8, 8, (4, 16, 2))).astype(np.float32)  # small integers: exact in fp32
    pick = rng.integers(0, 16, (20, 4))
    X = np.concatenate([C[m, pick[:, m]] for m in range(4)], axis=1)
    Q = rng.integers(-8, 8, (3, 8)).astype(np.float32)
    D = oracle.lut_f32(Q, C, oracle.METRIC_L2)
    got = D[:, np.arange(4)[None, :], pick].sum(axis=2)
    ref = ((Q[:, None, :].astype(np.float64) - X[None].astype(np.float64)) ** 2).sum(-1)
    np.testing.assert_array_equal(got, ref)  # integers: exact


# ------------------------------------------------------------------ beta_m
def test_quantize_hand_values():
    """beta(y) = clamp(floor(a (y - b)), 0, 255), hand-computed with a = 2,
    b = 1 (Sec. 3.2)."""
    ys = np.array([1.0, 1.75, 0.5, 128.0, 128.5, 200.0, np.nan, 1.4999999], np.float32)
    want = [0, 1, 0, 254, 255, 255, 0, 0]
    D = ys.reshape(1, 1, 8)
    D = np.concatenate([D, D], axis=2)  # 16 entries
    got = oracle.quantize(D, 2.0, np.array([1.0], np.float32))[0, 0, :8]
    assert got.tolist() == want


def test_quantize_lemma1_bound_and_monotone():
    """Lemma 1 (Sec. 3.3), read for floor rounding: inside [b, b + 255/a]
    the reconstruction error is below 1/a."""
    rng = np.random.default_rng(11)
    a, b = np.float32(3.7), np.float32(-2.25)
    y = np.sort(rng.uniform(-2.25, -2.25 + 255 / 3.7, 16 * 4096)).astype(np.float32)
    beta = oracle.quantize(y.reshape(-1, 1, 16), a, np.array([b], np.float32)).reshape(-1)
    yhat = beta.astype(np.float64) / np.float64(a) + np.float64(b)
    err = np.abs(yhat - y.astype(np.float64))
    assert err.max() < 1 / 3.7 * (1 + 1e-5)
    assert np.all(np.diff(beta.astype(np.int32)) >= 0)  # y sorted -> beta monotone
    assert beta.min() == 0 and beta.max() >= 254


# ------------------------------------------------------------------ quantizer fit
def test_fit_quant_two_point_tie_rule():
    """Entries only at 0 and 255: every alpha maps them exactly (a = 1,
    b = 0), all eight losses are 0 and the tie goes to alpha = 0."""
    vals = np.where(np.arange(4096) % 2 == 0, 0.0, 255.0).astype(np.float32)
    a, b, ai, losses = oracle.fit_quant(vals.reshape(256, 1, 16))
    assert ai == 0 and a == 1.0 and b[0] == 0.0 and np.all(losses == 0.0)


def test_quant_params_order_statistics_hand():
    """b = F^-1(alpha), a = 255 / (F^-1(1 - alpha) - b) (Sec. 3.2) with the
    lower-rank quantile: for one table holding 0..4095 (n = 4096),
    b = floor(alpha * 4095) and the upper quantile is floor((1-alpha)*4095)."""
    D = np.arange(4096, dtype=np.float32)[::-1].copy().reshape(256, 1, 16)
    want_lo = [0, 4, 8, 20, 40, 81, 204, 409]
    want_hi = [4095, 4090, 4086, 4074, 4054, 4013, 3890, 3685]
    for i in range(8):
        a, b = oracle.quant_params(D, i)
        assert b[0] == want_lo[i]
        assert a == 255.0 / (want_hi[i] - want_lo[i])


def test_quant_params_pooled_upper_quantile_hand():
    """Two tables: b_m is per table, a comes from the pooled offsets.
    Table 0 = 0..2047 (x2), table 1 = 1000 + 0..4095: offsets pool to
    {0..2047 twice} U {0..4095}; their max (alpha = 0) is 4095."""
    t0 = np.tile(np.arange(2048, dtype=np.float32), 2)
    t1 = 1000 + np.arange(4096, dtype=np.float32)
    D = np.stack([t0, t1], 1).reshape(256, 16, 2).transpose(0, 2, 1).copy()
    a, b = oracle.quant_params(D, 0)
    assert b.tolist() == [0.0, 1000.0] and a == 255.0 / 4095.0


def test_fit_quant_scale_equivariance():
    """Scaling every entry by 4 scales b by 4, a by 1/4, keeps alpha."""
    rng = np.random.default_rng(19)
    D = rng.gamma(2.0, 3.0, (256, 3, 16)).astype(np.float32)
    a, b, ai, _ = oracle.fit_quant(D)
    a4, b4, ai4, _ = oracle.fit_quant(D * np.float32(4))
    assert ai4 == ai and np.all(b4 == 4 * b) and np.isclose(a4 * 4, a, rtol=1e-7)


def test_fit_quant_shared_a_and_per_table_b():
    """Two tables that differ by a constant shift get b's differing by that
    shift and the same reconstruction error (the shared a sees offset
    entries, Sec. 3.2 last paragraph)."""
    rng = np.random.default_rng(12)
    base = rng.gamma(2.0, 3.0, (300, 1, 16)).astype(np.float32)
    D = np.concatenate([base, base + np.float32(64.0)], axis=1)
    a, b, ai, losses = oracle.fit_quant(D)
    assert b[1] - b[0] == np.float32(64.0)
    aa, bb, _, _ = oracle.fit_quant(base)
    assert aa == a and bb[0] == b[0]


def test_fit_quant_loss_matches_quantize_path():
    """The fit's fp64 loss for its chosen alpha agrees with the error of
    the fp32 quantize path using the returned (a, b)."""
    rng = np.random.default_rng(13)
    D = (rng.standard_normal((256, 4, 16)) ** 2 * 5).astype(np.float32)
    a, b, ai, losses = oracle.fit_quant(D)
    beta = oracle.quantize(D, a, b).astype(np.float64)
    yhat = beta / np.float64(a) + b.astype(np.float64)[None, :, None]
    mse = np.mean((yhat - D.astype(np.float64)) ** 2)
    np.testing.assert_allclose(mse, losses[ai], rtol=2e-3)


def _grid_losses_numpy(D):
    """Mean squared reconstruction error (Sec. 3.2, E[(y_hat - y)^2]) for
    every alpha of the grid, computed here in numpy from each grid point's
    fp64 (a, b_m): beta = clamp(floor(a (y - b_m)), 0, 255), y_hat = beta / a
    + b_m, averaged over every training entry of every table."""
    y = D.astype(np.float64)
    out = []
    for i in range(8):
        a, b = oracle.quant_params(D, i)
        beta = np.clip(np.floor(a * (y - b[None, :, None])), 0.0, 255.0)
        out.append(np.mean((beta / a + b[None, :, None] - y) ** 2))
    return np.array(out)


def _alpha_case(kind):
    """Training tables on which the best alpha lies inside the grid.  Bulk
    entries uniform on [0, 1) plus one entry at 2.0: with 131,072 entries
    the outlier's clamping costs less than the coarser steps it forces at
    alpha = 0, while large alphas clamp too much of the bulk."""
    n = 131072
    rng = np.random.default_rng(7)
    if kind == "interior":
        v = rng.uniform(0, 1, n).astype(np.float32)
        v[0] = 2.0
        rng.shuffle(v)
        return v.reshape(n // 16, 1, 16)
    if kind == "tie":
        # 1.5% of the entries exactly 0 and 1.5% exactly 1: alpha in
        # {.001, .002, .005, .01} picks the same quantile values (0 and 1),
        # so those four grid points have identical parameters and losses
        p = int(0.015 * n)
        v = np.concatenate([np.zeros(p), np.ones(p), rng.uniform(0, 1, n - 2 * p - 1), [2.0]]).astype(np.float32)
        rng.shuffle(v)
        return v.reshape(n // 16, 1, 16)
    # four tables offset by 0, 10, 20, 30 (the shared a sees y - b_m pooled)
    v = rng.uniform(0, 1, (n // 16, 4, 16)).astype(np.float32) + np.float32([0, 10, 20, 30])[None, :, None]
    v[5, 2, 3] = 22.0
    return v


@pytest.mark.parametrize("kind", ["interior", "tie", "pooled"])
def test_fit_quant_selects_grid_argmin(kind):
    """The fit returns the alpha with the smallest loss (Sec. 3.2: alpha is
    chosen to minimize E[(y_hat - y)^2] over the grid), ties to the smaller
    alpha, and the a, b of that grid point rounded to fp32.  The losses are
    recomputed independently in numpy.  The cases put the minimum inside the
    grid (not at its first or last point) and, for "tie", on four grid points
    at once, so a reversed comparison, ties going to the larger alpha or
    returning the last alpha all fail."""
    D = _alpha_case(kind)
    want = _grid_losses_numpy(D)
    a, b, ai, losses = oracle.fit_quant(D)
    np.testing.assert_allclose(losses, want, rtol=1e-9)
    best = np.flatnonzero(want == want.min())
    assert 0 < best[0] < 7, "case must put the minimum inside the grid"
    if kind == "tie":
        assert best.tolist() == [1, 2, 3, 4]
    else:
        # a margin far above the 1e-9 agreement, so rounding cannot move the argmin
        assert len(best) == 1 and want.min() < (1 - 1e-6) * np.partition(want, 1)[1]
    assert ai == best[0]
    a64, b64 = oracle.quant_params(D, ai)
    assert a == np.float32(a64) and np.array_equal(b, b64.astype(np.float32))


# ------------------------------------------------------------------ scan
def test_scan_bruteforce_exact():
    rng = np.random.default_rng(14)
    for n, M, nq in ((0, 4, 2), (1, 1, 1), (777, 16, 3), (100, 256, 2)):
        codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
        luts = rng.integers(0, 256, (nq, M, 16)).astype(np.uint8)
        got = oracle.scan(codes, luts)
        ref = np.zeros((nq, n), np.int64)
        for m in range(M):
            ref += luts[:, m, :][:, codes[:, m]].astype(np.int64)
        np.testing.assert_array_equal(got, ref)
    # maximum: M = 256 tables of 255 -> 65280 fits in uint16
    luts = np.full((1, 256, 16), 255, np.uint8)
    assert oracle.scan(np.zeros((2, 256), np.uint8), luts).tolist() == [[65280, 65280]]


def test_scan_float_is_bolt_no_quantize_sum():
    rng = np.random.default_rng(15)
    codes = rng.integers(0, 16, (50, 4)).astype(np.uint8)
    D = rng.standard_normal((2, 4, 16)).astype(np.float32)
    got = oracle.scan_float(codes, D)
    ref = sum(D[:, m, :][:, codes[:, m]].astype(np.float64) for m in range(4))
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-6)


# ------------------------------------------------------------------ top-k
@pytest.mark.parametrize("metric", [oracle.METRIC_L2, oracle.METRIC_DOT, oracle.METRIC_L1])
def test_topk_matches_lexsort(metric):
    rng = np.random.default_rng(16)
    sums = rng.integers(0, 40, (3, 5000)).astype(np.uint16)  # many ties
    k = 37
    got_s, got_i = oracle.topk(sums, k, metric)
    for q in range(3):
        idx = np.arange(5000)
        key = -sums[q].astype(np.int64) if metric == oracle.METRIC_DOT else sums[q].astype(np.int64)
        order = np.lexsort((idx, key))[:k]
        np.testing.assert_array_equal(got_i[q], order)
        np.testing.assert_array_equal(got_s[q], sums[q][order])


@pytest.mark.parametrize("metric", [oracle.METRIC_L2, oracle.METRIC_DOT, oracle.METRIC_L1])
def test_topk_u32_matches_lexsort(metric):
    """The uint32-sum top-k (more than 256 codebooks) against numpy lexsort,
    with sums past the uint16 range and long tie runs; ties to the lower
    index, L2 / L1 ascending, dot descending."""
    rng = np.random.default_rng(18)
    sums = (rng.integers(0, 50, (3, 7000)) * 7919 + 60_000).astype(np.uint32)  # values up to ~450,000
    for k in (1, 100, 1024):
        got_s, got_i = oracle.topk_u32(sums, k, metric)
        for q in range(3):
            key = -sums[q].astype(np.int64) if metric == oracle.METRIC_DOT else sums[q].astype(np.int64)
            order = np.lexsort((np.arange(7000), key))[:k]
            np.testing.assert_array_equal(got_i[q], order)
            np.testing.assert_array_equal(got_s[q], sums[q][order])
    s, i = oracle.topk_u32(np.array([[70_000, 3, 70_000]], np.uint32), 5, oracle.METRIC_DOT)
    assert i.tolist() == [[0, 2, 1, -1, -1]] and s.tolist() == [[70_000, 70_000, 3, 0, 0]]


def test_topk_pads_when_k_exceeds_n():
    s, i = oracle.topk(np.array([[5, 3, 5]], np.uint16), 5, oracle.METRIC_L2)
    assert i.tolist() == [[1, 0, 2, -1, -1]] and s.tolist() == [[3, 5, 5, 0, 0]]
    s, i = oracle.topk(np.array([[5, 3, 5]], np.uint16), 2, oracle.METRIC_DOT)
    assert i.tolist() == [[0, 2]]


# ------------------------------------------------------------------ dequantize / matmul
def test_dequant_is_sum_of_table_reconstructions():
    """S/a + sum_m b_m == sum_m (beta_m/a + b_m) (Sec. 3.2 bias remark)."""
    rng = np.random.default_rng(17)
    a = np.float32(0.73)
    b = rng.standard_normal(8).astype(np.float32)
    beta = rng.integers(0, 256, (100, 8))
    S = beta.sum(1).astype(np.uint16)
    got = oracle.dequant(S, a, b)
    ref = (beta / np.float64(a) + b.astype(np.float64)).sum(1)
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-4)
    ia, bias = oracle.dequant_params(a, b)
    assert ia == np.float32(1 / np.float64(a))


def test_matmul_bound_and_composition():
    """Approximate A B^T (Sec. 4.4) stays within M/a of A x_hat^T when no
    table entry is clipped (Lemma 1 per table), and equals the composition
    of the oracle's own stages."""
    rng = np.random.default_rng(18)
    J, M = 32, 8
    B = synth.mixture(600, J, 0)
    C = oracle.kmeans(B, M, 4, synth.kmeans_init_rows(600, 0))
    codes = oracle.encode(B, C)
    A = rng.standard_normal((20, J)).astype(np.float32)
    D = oracle.lut_f32(A, C, oracle.METRIC_DOT)
    # alpha = 0 fit on the same rows: nothing is clipped
    a, b, ai, _ = oracle.fit_quant(D)
    if ai != 0:
        pytest.skip("fit chose clipping")
    out = oracle.matmul(A, codes, C, a, b)
    xh = oracle.decode(codes, C).astype(np.float64)
    exact = A.astype(np.float64) @ xh.T
    assert np.max(np.abs(out - exact)) <= M / a * (1 + 1e-4) + 1e-3
    S = oracle.scan(codes, oracle.quantize(D, a, b))
    np.testing.assert_array_equal(out, oracle.dequant(S, a, b))


# ------------------------------------------------------------------ lemmas 3 and 4
def test_lemmas_3_and_4_hold_for_reconstruction():
    X = synth.mixture(2000, 32, 0)
    Q = synth.mixture(50, 32, 1)
    C = oracle.kmeans(X, 8, 6, synth.kmeans_init_rows(2000, 0))
    xh = oracle.decode(oracle.encode(X, C), C).astype(np.float64)
    Xd, Qd = X.astype(np.float64), Q.astype(np.float64)
    r = np.linalg.norm(Xd - xh, axis=1)
    lhs3 = np.abs(Qd @ Xd.T - Qd @ xh.T)
    assert np.all(lhs3 <= np.linalg.norm(Qd, axis=1)[:, None] * r[None, :] + 1e-9)
    lhs4 = np.abs(cdist(Qd, Xd) - cdist(Qd, xh))
    assert np.all(lhs4 <= r[None, :] + 1e-9)


# ------------------------------------------------------------------ more than 256 codebooks (uint32 sums)
def test_scan_u32_closed_forms_beyond_uint16():
    """All-255 tables give 255 M exactly (past 65,535 from M = 258 on); tables
    whose entry is the code itself give the row sum of the codes (a library
    reduction); M = 1 picks one table entry."""
    rng = np.random.default_rng(61)
    for M in (257, 258, 300, 1024, 4096):
        codes = rng.integers(0, 16, (37, M)).astype(np.uint8)
        full = np.full((2, M, 16), 255, np.uint8)
        np.testing.assert_array_equal(oracle.scan_u32(codes, full), np.full((2, 37), 255 * M, np.uint32))
        ident = np.tile(np.arange(16, dtype=np.uint8), (1, M, 1))
        np.testing.assert_array_equal(oracle.scan_u32(codes, ident)[0], codes.astype(np.int64).sum(axis=1))
    luts = rng.integers(0, 256, (3, 1, 16)).astype(np.uint8)
    codes = rng.integers(0, 16, (50, 1)).astype(np.uint8)
    np.testing.assert_array_equal(oracle.scan_u32(codes, luts), luts[:, 0, codes[:, 0]])


def test_scan_u32_splits_into_uint16_scans():
    """The sum over M = 700 codebooks is the sum of the scans over any split
    of the codebooks (additivity of the sum over m); for M <= 256 it equals the
    uint16 scan."""
    rng = np.random.default_rng(62)
    M, n = 700, 301
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    luts = rng.integers(0, 256, (4, M, 16)).astype(np.uint8)
    parts = [(0, 256), (256, 512), (512, 700)]
    want = sum(oracle.scan(codes[:, a:b], luts[:, a:b]).astype(np.int64) for a, b in parts)
    np.testing.assert_array_equal(oracle.scan_u32(codes, luts), want)
    np.testing.assert_array_equal(oracle.scan_u32(codes[:, :200], luts[:, :200]),
                                  oracle.scan(codes[:, :200], luts[:, :200]))
    # brute force on a tiny case
    c, l = codes[:3, :300], luts[:1, :300]
    bf = [int(sum(int(l[0, m, c[i, m]]) for m in range(300))) for i in range(3)]
    assert oracle.scan_u32(c, l)[0].tolist() == bf


def test_dequant_u32_matches_uint16_and_closed_form():
    rng = np.random.default_rng(63)
    b = rng.standard_normal(400).astype(np.float32)
    S16 = rng.integers(0, 65536, 1000).astype(np.uint16)
    np.testing.assert_array_equal(oracle.dequant_u32(S16.astype(np.uint32), 3.5, b), oracle.dequant(S16, 3.5, b))
    S = np.array([0, 65536, 100_000, 255 * 4096], np.uint32)
    zero = np.zeros(4096, np.float32)
    np.testing.assert_array_equal(oracle.dequant_u32(S, 1.0, zero), S.astype(np.float32))


def test_encode_and_tables_beyond_256_codebooks():
    """M = 512, s = 2: points built from centroids encode to their indices;
    each table entry equals the fp64 distance by a library routine (within
    fp32 rounding) and the sum of the L2 table entries picked by a vector's
    own codes is the squared distance to its reconstruction (Sec. 3.1
    decomposition)."""
    rng = np.random.default_rng(64)
    M, s = 512, 2
    C = rng.standard_normal((M, 16, s)).astype(np.float32)
    want = rng.integers(0, 16, (20, M))
    X = np.concatenate([C[m, want[:, m]] for m in range(M)], axis=1)
    np.testing.assert_array_equal(oracle.encode(X, C), want)
    Q = rng.standard_normal((3, M * s)).astype(np.float32)
    D = oracle.lut_f32(Q, C, oracle.METRIC_L2)
    ref = np.stack([cdist(Q[:, m * s:(m + 1) * s].astype(np.float64), C[m].astype(np.float64), "sqeuclidean")
                    for m in range(M)], axis=1)
    np.testing.assert_allclose(D, ref, rtol=1e-5, atol=1e-6)
    picked = D[:, np.arange(M)[None, :], want[:5]].sum(axis=2)  # (3, 5)
    dist = ((Q[:, None, :].astype(np.float64) - X[None, :5].astype(np.float64)) ** 2).sum(axis=2)
    np.testing.assert_allclose(picked, dist, rtol=1e-5)
    a, bq = 2.0, np.zeros(M, np.float32)
    L = oracle.quantize(D, a, bq)
    assert L.shape == (3, M, 16)
    np.testing.assert_array_equal(L, np.clip(np.floor(D * np.float32(a)), 0, 255).astype(np.uint8))


@pytest.mark.parametrize("metric", [oracle.METRIC_L2, oracle.METRIC_DOT, oracle.METRIC_L1])
def test_parallel_driver_equals_single_scan(metric):
    """The threaded driver of the timed CPU baseline returns exactly the
    oracle's single-threaded top-k, ties included (tables with 4 values make
    long tie runs that cross range boundaries)."""
    from oracle import parallel

    rng = np.random.default_rng(30 + metric)
    codes = rng.integers(0, 16, (100_003, 8)).astype(np.uint8)
    luts = rng.integers(0, 4, (3, 8, 16)).astype(np.uint8)
    want = oracle.topk(oracle.scan(codes, luts), 100, metric)
    for threads in (1, 3, 7):
        got = parallel.scan_topk(codes, luts, 100, metric, threads=threads)
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])


def test_parallel_encode_equals_encode():
    from oracle import parallel

    rng = np.random.default_rng(31)
    X = rng.standard_normal((10_007, 16)).astype(np.float32)
    C = rng.standard_normal((4, 16, 4)).astype(np.float32)
    np.testing.assert_array_equal(parallel.encode(X, C, threads=3, chunk=1000), oracle.encode(X, C))


# ------------------------------------------------------------------ L_p tables
def test_lp_tables_reduce_to_l1_and_l2():
    """p = 1 is the L1 table (powf(t, 1) = t exactly); p = 2 in fp64 is the
    L2 table up to the last bit of a term (pow(t, 2) against t * t)."""
    rng = np.random.default_rng(40)
    Q = rng.standard_normal((5, 24)).astype(np.float32)
    C = rng.standard_normal((6, 16, 4)).astype(np.float32)
    np.testing.assert_array_equal(oracle.lut_lp_f32(Q, C, 1.0), oracle.lut_f32(Q, C, oracle.METRIC_L1))
    np.testing.assert_allclose(oracle.lut_lp_f64(Q, C, 2.0), oracle.lut_f64(Q, C, oracle.METRIC_L2), rtol=1e-14)


def test_lp_tables_closed_forms():
    """One differing coordinate d gives |d|^p exactly for exact powers
    (2^3 = 8, 4^0.5 = 2, 0.25^1.5 = 0.125, 3^0 is excluded: p > 0), and a
    query on a centroid gives 0; the entries of the other centroids follow
    the subspace's own dims only."""
    s = 4
    C = np.zeros((2, 16, s), np.float32)
    for k in range(16):
        C[:, k, :] = k  # centroid k of both subspaces: all coordinates k
    for d, p, want in ((2.0, 3.0, 8.0), (4.0, 0.5, 2.0), (0.25, 1.5, 0.125)):
        q = np.zeros((1, 2 * s), np.float32)
        q[0, 1] = d  # subspace 0: one coordinate d away from centroid 0
        D = oracle.lut_lp_f64(q, C, p)
        assert D[0, 0, 0] == want
        assert D[0, 1, 0] == 0.0  # subspace 1: the query is on centroid 0
        # centroid 5 in subspace 1: four coordinates 5 away
        assert D[0, 1, 5] == pytest.approx(4 * 5.0 ** p, rel=1e-15)
        assert oracle.lut_lp_f32(q, C, p)[0, 0, 0] == np.float32(want)


@pytest.mark.parametrize("p", [0.5, 1.5, 3.0])
def test_lp_tables_homogeneous_and_fp32_close(p):
    """Scaling query and centroids by 2 scales every entry by 2^p (fp64,
    up to rounding), and the fp32 table is within 1e-5 of the fp64 one."""
    rng = np.random.default_rng(41)
    Q = rng.standard_normal((4, 32)).astype(np.float32)
    C = rng.standard_normal((8, 16, 4)).astype(np.float32)
    D = oracle.lut_lp_f64(Q, C, p)
    D2 = oracle.lut_lp_f64(2 * Q, 2 * C, p)
    np.testing.assert_allclose(D2, D * 2.0 ** p, rtol=1e-12)
    np.testing.assert_allclose(oracle.lut_lp_f32(Q, C, p), D, rtol=1e-5, atol=1e-6)
    with pytest.raises(oracle.OracleError):
        oracle.lut_lp_f32(Q, C, 0.0)


def test_lp_metric_ranks_ascending():
    """Top-k of L_p sums ranks ascending with ties to the lower index, the
    same order as L1."""
    rng = np.random.default_rng(42)
    S = rng.integers(0, 50, (3, 2000)).astype(np.uint16)
    a = oracle.topk(S, 37, oracle.METRIC_LP)
    b = oracle.topk(S, 37, oracle.METRIC_L1)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert (np.diff(a[0].astype(int), axis=1) >= 0).all()
