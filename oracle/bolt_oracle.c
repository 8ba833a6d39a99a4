/*
 * Bolt CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of the Bolt method (Blalock &
 * Guttag, "Bolt: Accelerated Data Mining with Fast Vector Compression",
 * KDD'17), written to check the CUDA library against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never does.  It shares no code, header, table or constant with
 * the CUDA sources.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (see oracle/build.py), so
 * every floating-point operation below is one IEEE operation in the order it
 * is written.  fmaf()/fma() are the only fused operations and are spelled out.
 *
 * Notation follows the paper: J dims, M codebooks (subspaces), K = 16
 * centroids per codebook, s = J/M dims per subspace, N database vectors.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *  - Subspace m owns the consecutive dims [m*s, (m+1)*s) (Sec. 3.1: "typically
 *    ... J/M consecutive indices"); J must be a multiple of M.
 *  - Encoder distance for one (x, m, k) is accumulated in fp32 in dim order as
 *    acc = fmaf(t, t, acc), t = x_j - c_j, starting from 0.  Argmin ties go to
 *    the lowest centroid index.
 *  - LUT entry (Sec. 3.1, the matrix D): L2 uses the same fmaf order as the
 *    encoder; dot uses acc = fmaf(q_j, c_j, acc) in dim order.
 *  - Quantizer (Sec. 3.2): beta_m(y) = clamp(floor(a*(y - b_m)), 0, 255) with
 *    t = (y - b_m) then t * a as two separately rounded fp32 operations; NaN
 *    maps to 0.  Reconstruction y_hat = beta/a + b_m.
 *  - Quantizer fit (Sec. 3.2): b_m = lower-rank empirical alpha-quantile of
 *    table m's training entries; a = 255 / (pooled (1-alpha)-quantile of
 *    y - b_m over all tables) (a = 1 if that quantile is <= 0); alpha from
 *    the paper's grid by minimum mean squared reconstruction error, computed
 *    in fp64, ties to the smaller alpha; a and b_m are then rounded to fp32.
 *  - Scan (Sec. 3.1, approximate distance as a sum of M table entries): exact
 *    integer sum, stored as uint16 (255*M <= 65535 for M <= 256); for more
 *    codebooks (up to BO_MAX_M) the same sum stored as uint32 (bo_scan_u32).
 *  - Top-k: L2 ascending sum, dot descending sum, ties to the lower index;
 *    k > N pads with index -1 and sum 0.
 *  - Dequantize (Sec. 3.2, the biases sum to one known offset): out =
 *    (float)S * inv_a + B as two fp32 roundings, inv_a = (float)(1/(double)a),
 *    B = (float)(sum_m (double)b_m).
 *  - k-means (Sec. 3.1 background, PQ codebooks): Lloyd iterations with the
 *    assignment above; means accumulated in fp64 in row order, divided in
 *    fp64 and rounded to fp32; an empty cluster keeps its centroid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BO_K 16
#define BO_OK 0
#define BO_EINVAL 1
#define BO_EUNSUPPORTED 2
#define BO_ENOMEM 3

/* L1: delta = |q_j - x_j| (the L_p family of Sec. 1.1 with p = 1; f(r) = r
 * is monotone, so nearest neighbours rank by the sum itself, ascending).
 * L_p: delta = |q_j - x_j|^p for a real p > 0 (the same family; f(r) =
 * r^(1/p) is monotone, so the ranking is again by the sum, ascending); its
 * tables come from bo_lut_lp_f32 / bo_lut_lp_f64. */
enum { BO_METRIC_L2 = 0, BO_METRIC_DOT = 1, BO_METRIC_L1 = 2, BO_METRIC_LP = 3 };

/* Largest codebook count; uint16 sums (bo_scan, bo_topk) hold M <= 256. */
#define BO_MAX_M 4096

static int check_shape(int64_t n, int32_t J, int32_t M) {
    if (n < 0 || J <= 0 || M <= 0) return BO_EINVAL;
    if (J % M != 0) return BO_EUNSUPPORTED;
    if (M > BO_MAX_M) return BO_EUNSUPPORTED;
    return BO_OK;
}

/* ---------------------------------------------------------------- encode h
 * Sec. 3.1, the PQ encoding function h: i_m = argmin_i d(c_i^(m), x^(m)),
 * with K = 16 centroids per codebook (Sec. 3.2, change 1).
 * codes: row-major n x M, one code (0..15) per byte. */
int bo_encode_f32(const float *X, int64_t n, int32_t J, int32_t M,
                  const float *C, uint8_t *codes) {
    int rc = check_shape(n, J, M);
    if (rc) return rc;
    const int s = J / M;
    for (int64_t i = 0; i < n; i++) {
        const float *x = X + i * (int64_t)J;
        for (int m = 0; m < M; m++) {
            float best = INFINITY;
            int best_k = 0;
            for (int k = 0; k < BO_K; k++) {
                const float *c = C + ((int64_t)m * BO_K + k) * s;
                float acc = 0.0f;
                for (int j = 0; j < s; j++) {
                    float t = x[m * s + j] - c[j];
                    acc = fmaf(t, t, acc);
                }
                if (acc < best) { /* strict: ties keep the lower index */
                    best = acc;
                    best_k = k;
                }
            }
            codes[i * M + m] = (uint8_t)best_k;
        }
    }
    return BO_OK;
}

/* Same argmin with every quantity in fp64: used for distortion and the
 * mismatch rate of the fp32 encoders against exact-ish arithmetic. */
int bo_encode_f64(const float *X, int64_t n, int32_t J, int32_t M,
                  const float *C, uint8_t *codes) {
    int rc = check_shape(n, J, M);
    if (rc) return rc;
    const int s = J / M;
    for (int64_t i = 0; i < n; i++) {
        const float *x = X + i * (int64_t)J;
        for (int m = 0; m < M; m++) {
            double best = INFINITY;
            int best_k = 0;
            for (int k = 0; k < BO_K; k++) {
                const float *c = C + ((int64_t)m * BO_K + k) * s;
                double acc = 0.0;
                for (int j = 0; j < s; j++) {
                    double t = (double)x[m * s + j] - (double)c[j];
                    acc = acc + t * t;
                }
                if (acc < best) {
                    best = acc;
                    best_k = k;
                }
            }
            codes[i * M + m] = (uint8_t)best_k;
        }
    }
    return BO_OK;
}

/* Definition "Reconstruction" (Sec. 3.3): x_hat replaces each subvector by
 * its chosen centroid. */
int bo_decode(const uint8_t *codes, int64_t n, int32_t J, int32_t M,
              const float *C, float *Xhat) {
    int rc = check_shape(n, J, M);
    if (rc) return rc;
    const int s = J / M;
    for (int64_t i = 0; i < n; i++)
        for (int m = 0; m < M; m++) {
            int k = codes[i * M + m];
            if (k >= BO_K) return BO_EINVAL;
            const float *c = C + ((int64_t)m * BO_K + k) * s;
            for (int j = 0; j < s; j++) Xhat[i * J + m * s + j] = c[j];
        }
    return BO_OK;
}

/* fp64 squared reconstruction error summed over all rows and subspaces. */
static double objective(const float *X, int64_t n, int32_t J, int32_t M,
                        const float *C, const uint8_t *codes) {
    const int s = J / M;
    double tot = 0.0;
    for (int64_t i = 0; i < n; i++)
        for (int m = 0; m < M; m++) {
            const float *c = C + ((int64_t)m * BO_K + codes[i * M + m]) * s;
            for (int j = 0; j < s; j++) {
                double t = (double)X[i * J + m * s + j] - (double)c[j];
                tot = tot + t * t;
            }
        }
    return tot;
}

/* ---------------------------------------------------------------- k-means
 * Sec. 3.1 background: codebooks are learned by k-means, O(KNJT).
 * init_rows: the 16 database rows whose subvectors seed every codebook.
 * objective_out (nullable, iters+1 values): objective of the assignment to
 * the centroids of iteration t, t = 0..iters. */
int bo_kmeans(const float *X, int64_t n, int32_t J, int32_t M, int32_t iters,
              const int64_t *init_rows, float *C, double *objective_out) {
    int rc = check_shape(n, J, M);
    if (rc) return rc;
    if (n <= 0 || iters < 0) return BO_EINVAL;
    const int s = J / M;
    for (int k = 0; k < BO_K; k++) {
        if (init_rows[k] < 0 || init_rows[k] >= n) return BO_EINVAL;
        for (int m = 0; m < M; m++)
            for (int j = 0; j < s; j++)
                C[((int64_t)m * BO_K + k) * s + j] = X[init_rows[k] * J + m * s + j];
    }
    uint8_t *codes = (uint8_t *)malloc((size_t)n * M);
    double *sum = (double *)malloc(sizeof(double) * (size_t)M * BO_K * s);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)M * BO_K);
    if (!codes || !sum || !cnt) {
        free(codes); free(sum); free(cnt);
        return BO_ENOMEM;
    }
    for (int it = 0; it <= iters; it++) {
        bo_encode_f32(X, n, J, M, C, codes);
        if (objective_out) objective_out[it] = objective(X, n, J, M, C, codes);
        if (it == iters) break;
        memset(sum, 0, sizeof(double) * (size_t)M * BO_K * s);
        memset(cnt, 0, sizeof(int64_t) * (size_t)M * BO_K);
        for (int64_t i = 0; i < n; i++)
            for (int m = 0; m < M; m++) {
                int k = codes[i * M + m];
                cnt[m * BO_K + k] += 1;
                for (int j = 0; j < s; j++)
                    sum[((int64_t)m * BO_K + k) * s + j] += (double)X[i * J + m * s + j];
            }
        for (int m = 0; m < M; m++)
            for (int k = 0; k < BO_K; k++) {
                int64_t c = cnt[m * BO_K + k];
                if (c == 0) continue; /* empty cluster keeps its centroid */
                for (int j = 0; j < s; j++) {
                    int64_t o = ((int64_t)m * BO_K + k) * s + j;
                    C[o] = (float)(sum[o] / (double)c);
                }
            }
    }
    free(codes); free(sum); free(cnt);
    return BO_OK;
}

/* ---------------------------------------------------------------- LUT g
 * Sec. 3.1, query encoding: D_im = delta(q^(m), c_i^(m)); delta is the
 * squared difference summed over the subspace (L2) or the product summed
 * (dot), Sec. 1.1's distance form.  D layout: [q][m][k] (16 contiguous
 * entries per (query, codebook)). */
int bo_lut_f32(const float *Q, int64_t nq, int32_t J, int32_t M, const float *C,
               int32_t metric, float *D) {
    int rc = check_shape(nq, J, M);
    if (rc) return rc;
    if (metric != BO_METRIC_L2 && metric != BO_METRIC_DOT && metric != BO_METRIC_L1) return BO_EINVAL;
    const int s = J / M;
    for (int64_t q = 0; q < nq; q++)
        for (int m = 0; m < M; m++)
            for (int k = 0; k < BO_K; k++) {
                const float *c = C + ((int64_t)m * BO_K + k) * s;
                const float *x = Q + q * J + m * s;
                float acc = 0.0f;
                if (metric == BO_METRIC_L2) {
                    for (int j = 0; j < s; j++) {
                        float t = x[j] - c[j];
                        acc = fmaf(t, t, acc);
                    }
                } else if (metric == BO_METRIC_L1) {
                    for (int j = 0; j < s; j++) acc = acc + fabsf(x[j] - c[j]);
                } else {
                    for (int j = 0; j < s; j++) acc = fmaf(x[j], c[j], acc);
                }
                D[(q * M + m) * BO_K + k] = acc;
            }
    return BO_OK;
}

/* The same table in fp64 (reference for the float-LUT tolerance). */
int bo_lut_f64(const float *Q, int64_t nq, int32_t J, int32_t M, const float *C,
               int32_t metric, double *D) {
    int rc = check_shape(nq, J, M);
    if (rc) return rc;
    if (metric != BO_METRIC_L2 && metric != BO_METRIC_DOT && metric != BO_METRIC_L1) return BO_EINVAL;
    const int s = J / M;
    for (int64_t q = 0; q < nq; q++)
        for (int m = 0; m < M; m++)
            for (int k = 0; k < BO_K; k++) {
                const float *c = C + ((int64_t)m * BO_K + k) * s;
                const float *x = Q + q * J + m * s;
                double acc = 0.0;
                for (int j = 0; j < s; j++) {
                    if (metric == BO_METRIC_L2) {
                        double t = (double)x[j] - (double)c[j];
                        acc = acc + t * t;
                    } else if (metric == BO_METRIC_L1) {
                        acc = acc + fabs((double)x[j] - (double)c[j]);
                    } else {
                        acc = acc + (double)x[j] * (double)c[j];
                    }
                }
                D[(q * M + m) * BO_K + k] = acc;
            }
    return BO_OK;
}

/* L_p tables (Sec. 1.1 family, delta = |q_j - c_j|^p, real p > 0): the
 * entries summed over the subspace's dims in order from the first, each
 * |q_j - c_j|^p from the C library's powf with fp32 adds; the fp64 form
 * (pow, fp64 adds) is the reference for the float tolerance.  A GPU's
 * powf may differ from this one in the last bits, so its tables are
 * compared within a tolerance and its bytes by quantizing its own floats. */
int bo_lut_lp_f32(const float *Q, int64_t nq, int32_t J, int32_t M, const float *C, float p, float *D) {
    int rc = check_shape(nq, J, M);
    if (rc) return rc;
    if (!(p > 0.0f) || !(p < INFINITY)) return BO_EINVAL;
    const int s = J / M;
    for (int64_t q = 0; q < nq; q++)
        for (int m = 0; m < M; m++)
            for (int k = 0; k < BO_K; k++) {
                const float *c = C + ((int64_t)m * BO_K + k) * s;
                const float *x = Q + q * J + m * s;
                float acc = 0.0f;
                for (int j = 0; j < s; j++) acc = acc + powf(fabsf(x[j] - c[j]), p);
                D[(q * M + m) * BO_K + k] = acc;
            }
    return BO_OK;
}

int bo_lut_lp_f64(const float *Q, int64_t nq, int32_t J, int32_t M, const float *C, float p, double *D) {
    int rc = check_shape(nq, J, M);
    if (rc) return rc;
    if (!(p > 0.0f) || !(p < INFINITY)) return BO_EINVAL;
    const int s = J / M;
    for (int64_t q = 0; q < nq; q++)
        for (int m = 0; m < M; m++)
            for (int k = 0; k < BO_K; k++) {
                const float *c = C + ((int64_t)m * BO_K + k) * s;
                const float *x = Q + q * J + m * s;
                double acc = 0.0;
                for (int j = 0; j < s; j++) acc = acc + pow(fabs((double)x[j] - (double)c[j]), (double)p);
                D[(q * M + m) * BO_K + k] = acc;
            }
    return BO_OK;
}

/* ---------------------------------------------------------------- beta_m
 * Sec. 3.2: beta_m(y) = max(0, min(255, floor(a (y - b_m)))). */
static uint8_t quantize_one(float y, float a, float b) {
    float t = y - b;
    t = t * a;
    if (!(t >= 0.0f)) return 0; /* negative or NaN */
    if (t >= 255.0f) return 255;
    return (uint8_t)floorf(t);
}

int bo_quantize(const float *D, int64_t nq, int32_t M, float a, const float *b,
                uint8_t *luts) {
    if (nq < 0 || M <= 0 || M > BO_MAX_M) return BO_EINVAL;
    for (int64_t q = 0; q < nq; q++)
        for (int m = 0; m < M; m++)
            for (int k = 0; k < BO_K; k++) {
                int64_t o = (q * M + m) * BO_K + k;
                luts[o] = quantize_one(D[o], a, b[m]);
            }
    return BO_OK;
}

/* ---------------------------------------------------------------- fit a, b
 * Sec. 3.2: b = F^-1(alpha), a = 255 / (F^-1(1-alpha) - b), alpha chosen from
 * {0, .001, .002, .005, .01, .02, .05, .1} by the mean squared error of the
 * reconstruction; per-table b_m, one shared a from the pooled distribution
 * (reading stated in the file header). */
static const double kAlphas[8] = {0.0, 0.001, 0.002, 0.005, 0.01, 0.02, 0.05, 0.1};

static int cmp_double(const void *pa, const void *pb) {
    double x = *(const double *)pa, y = *(const double *)pb;
    return (x > y) - (x < y);
}

/* table m's entries in ascending order: sorted[m*nm + r], nm = 16*ntq */
static double *sorted_tables(const float *Dtrain, int64_t ntq, int32_t M) {
    const int64_t nm = ntq * BO_K;
    double *sorted = (double *)malloc(sizeof(double) * (size_t)(nm * M));
    if (!sorted) return NULL;
    for (int m = 0; m < M; m++) {
        for (int64_t q = 0; q < ntq; q++)
            for (int k = 0; k < BO_K; k++)
                sorted[m * nm + q * BO_K + k] = (double)Dtrain[(q * M + m) * BO_K + k];
        qsort(sorted + m * nm, (size_t)nm, sizeof(double), cmp_double);
    }
    return sorted;
}

/* fp64 (a, b_m) for one alpha: b_m = F_m^-1(alpha) (lower-rank empirical
 * quantile), a = 255 / F_pool^-1(1 - alpha) of the offsets y - b_m. */
static int params_for_alpha(const double *sorted, int64_t nm, int32_t M, double alpha,
                            double *a_out, double *b_out) {
    const int64_t np = nm * M;
    double *pooled = (double *)malloc(sizeof(double) * (size_t)np);
    if (!pooled) return BO_ENOMEM;
    const int64_t lo = (int64_t)floor(alpha * (double)(nm - 1));
    for (int m = 0; m < M; m++) b_out[m] = sorted[m * nm + lo];
    for (int m = 0; m < M; m++)
        for (int64_t r = 0; r < nm; r++) pooled[m * nm + r] = sorted[m * nm + r] - b_out[m];
    qsort(pooled, (size_t)np, sizeof(double), cmp_double);
    const int64_t hi = (int64_t)floor((1.0 - alpha) * (double)(np - 1));
    const double upper = pooled[hi];
    *a_out = upper > 0.0 ? 255.0 / upper : 1.0;
    free(pooled);
    return BO_OK;
}

/* fp64 parameters for grid point alpha_idx (0..7). */
int bo_quant_params(const float *Dtrain, int64_t ntq, int32_t M, int32_t alpha_idx,
                    double *a_out, double *b_out) {
    if (ntq <= 0 || M <= 0 || M > BO_MAX_M || alpha_idx < 0 || alpha_idx > 7) return BO_EINVAL;
    double *sorted = sorted_tables(Dtrain, ntq, M);
    if (!sorted) return BO_ENOMEM;
    int rc = params_for_alpha(sorted, ntq * BO_K, M, kAlphas[alpha_idx], a_out, b_out);
    free(sorted);
    return rc;
}

/* Dtrain: ntq x M x 16 fp32 table entries of the training queries.
 * loss_out (nullable): the 8 losses of the grid; alpha_idx_out (nullable). */
int bo_fit_quant(const float *Dtrain, int64_t ntq, int32_t M, float *a_out,
                 float *b_out, int32_t *alpha_idx_out, double *loss_out) {
    if (ntq <= 0 || M <= 0 || M > BO_MAX_M) return BO_EINVAL;
    const int64_t nm = ntq * BO_K;     /* entries per table */
    const int64_t np = nm * M;         /* pooled entries */
    double *sorted = sorted_tables(Dtrain, ntq, M);
    double *bm = (double *)malloc(sizeof(double) * (size_t)M);
    double *best_b = (double *)malloc(sizeof(double) * (size_t)M);
    if (!sorted || !bm || !best_b) {
        free(sorted); free(bm); free(best_b);
        return BO_ENOMEM;
    }
    double best_loss = INFINITY, best_a = 1.0;
    int best_idx = 0;
    for (int ai = 0; ai < 8; ai++) {
        double a;
        if (params_for_alpha(sorted, nm, M, kAlphas[ai], &a, bm)) {
            free(sorted); free(bm); free(best_b);
            return BO_ENOMEM;
        }
        double loss = 0.0;
        for (int m = 0; m < M; m++)
            for (int64_t r = 0; r < nm; r++) {
                double y = sorted[m * nm + r];
                double t = floor(a * (y - bm[m]));
                double beta = t < 0.0 ? 0.0 : (t > 255.0 ? 255.0 : t);
                double yhat = beta / a + bm[m];
                loss = loss + (yhat - y) * (yhat - y);
            }
        loss = loss / (double)np;
        if (loss_out) loss_out[ai] = loss;
        if (loss < best_loss) { /* strict: ties keep the smaller alpha */
            best_loss = loss;
            best_a = a;
            best_idx = ai;
            memcpy(best_b, bm, sizeof(double) * (size_t)M);
        }
    }
    *a_out = (float)best_a;
    for (int m = 0; m < M; m++) b_out[m] = (float)best_b[m];
    if (alpha_idx_out) *alpha_idx_out = best_idx;
    free(sorted); free(bm); free(best_b);
    return BO_OK;
}

/* ---------------------------------------------------------------- scan
 * Sec. 3.1, the approximate distance sum_m D[h(x)_m, m] with Bolt's 8-bit
 * tables (Sec. 3.2): an exact integer sum.  codes: row-major n x M; luts:
 * [q][m][16] bytes; sums: [q][n]. */
int bo_scan(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts,
            int64_t nq, uint16_t *sums) {
    if (n < 0 || nq < 0 || M <= 0 || M > 256) return BO_EINVAL;
    for (int64_t q = 0; q < nq; q++)
        for (int64_t i = 0; i < n; i++) {
            uint32_t acc = 0;
            for (int m = 0; m < M; m++) {
                int k = codes[i * M + m];
                if (k >= BO_K) return BO_EINVAL;
                acc += luts[(q * M + m) * BO_K + k];
            }
            sums[q * n + i] = (uint16_t)acc;
        }
    return BO_OK;
}

/* The same exact sum for any M up to BO_MAX_M, stored as uint32
 * (255 * 4096 < 2^20). */
int bo_scan_u32(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts,
                int64_t nq, uint32_t *sums) {
    if (n < 0 || nq < 0 || M <= 0 || M > BO_MAX_M) return BO_EINVAL;
    for (int64_t q = 0; q < nq; q++)
        for (int64_t i = 0; i < n; i++) {
            uint32_t acc = 0;
            for (int m = 0; m < M; m++) {
                int k = codes[i * M + m];
                if (k >= BO_K) return BO_EINVAL;
                acc += luts[(q * M + m) * BO_K + k];
            }
            sums[q * n + i] = acc;
        }
    return BO_OK;
}

/* "Bolt No Quantize" (Sec. 4.2): the same sum over unquantized fp32 tables,
 * accumulated in codebook order. */
int bo_scan_float(const uint8_t *codes, int64_t n, int32_t M, const float *D,
                  int64_t nq, float *out) {
    if (n < 0 || nq < 0 || M <= 0 || M > 256) return BO_EINVAL;
    for (int64_t q = 0; q < nq; q++)
        for (int64_t i = 0; i < n; i++) {
            float acc = 0.0f;
            for (int m = 0; m < M; m++) acc = acc + D[(q * M + m) * BO_K + codes[i * M + m]];
            out[q * n + i] = acc;
        }
    return BO_OK;
}

/* ---------------------------------------------------------------- top-k
 * Nearest neighbours (smallest L2) / maximum inner product (largest dot),
 * Sec. 1.2 and Sec. 4.5.  Keeps a sorted list of the k best seen so far. */
static int better(int32_t metric, uint16_t s1, int64_t i1, uint16_t s2, int64_t i2) {
    if (s1 != s2) return metric == BO_METRIC_DOT ? s1 > s2 : s1 < s2;
    return i1 < i2;
}

int bo_topk(const uint16_t *sums, int64_t n, int64_t nq, int32_t k, int32_t metric,
            uint16_t *out_sums, int64_t *out_idx) {
    if (n < 0 || nq < 0 || k <= 0) return BO_EINVAL;
    if (metric != BO_METRIC_L2 && metric != BO_METRIC_DOT && metric != BO_METRIC_L1 && metric != BO_METRIC_LP)
        return BO_EINVAL;
    for (int64_t q = 0; q < nq; q++) {
        uint16_t *bs = out_sums + q * k;
        int64_t *bi = out_idx + q * k;
        int cnt = 0;
        for (int64_t i = 0; i < n; i++) {
            uint16_t s = sums[q * n + i];
            if (cnt == k && !better(metric, s, i, bs[k - 1], bi[k - 1])) continue;
            int pos = cnt < k ? cnt : k - 1;
            while (pos > 0 && better(metric, s, i, bs[pos - 1], bi[pos - 1])) {
                bs[pos] = bs[pos - 1];
                bi[pos] = bi[pos - 1];
                pos--;
            }
            bs[pos] = s;
            bi[pos] = i;
            if (cnt < k) cnt++;
        }
        for (int r = cnt; r < k; r++) {
            bs[r] = 0;
            bi[r] = -1;
        }
    }
    return BO_OK;
}

/* The same selection over the uint32 sums of more than 256 codebooks
 * (bo_scan_u32): the order (L2 and L1 ascending, dot descending) and the tie
 * rule (lower index first) are those of bo_topk. */
static int better_u32(int32_t metric, uint32_t s1, int64_t i1, uint32_t s2, int64_t i2) {
    if (s1 != s2) return metric == BO_METRIC_DOT ? s1 > s2 : s1 < s2;
    return i1 < i2;
}

int bo_topk_u32(const uint32_t *sums, int64_t n, int64_t nq, int32_t k, int32_t metric,
                uint32_t *out_sums, int64_t *out_idx) {
    if (n < 0 || nq < 0 || k <= 0) return BO_EINVAL;
    if (metric != BO_METRIC_L2 && metric != BO_METRIC_DOT && metric != BO_METRIC_L1 && metric != BO_METRIC_LP)
        return BO_EINVAL;
    for (int64_t q = 0; q < nq; q++) {
        uint32_t *bs = out_sums + q * k;
        int64_t *bi = out_idx + q * k;
        int cnt = 0;
        for (int64_t i = 0; i < n; i++) {
            uint32_t s = sums[q * n + i];
            if (cnt == k && !better_u32(metric, s, i, bs[k - 1], bi[k - 1])) continue;
            int pos = cnt < k ? cnt : k - 1;
            while (pos > 0 && better_u32(metric, s, i, bs[pos - 1], bi[pos - 1])) {
                bs[pos] = bs[pos - 1];
                bi[pos] = bi[pos - 1];
                pos--;
            }
            bs[pos] = s;
            bi[pos] = i;
            if (cnt < k) cnt++;
        }
        for (int r = cnt; r < k; r++) {
            bs[r] = 0;
            bi[r] = -1;
        }
    }
    return BO_OK;
}

/* ---------------------------------------------------------------- dequantize
 * Sec. 3.2: sum of per-table reconstructions beta_m/a + b_m = S/a + sum_m b_m;
 * the bias sum_m b_m is the "one overall bias" known after training. */
int bo_dequant_params(float a, const float *b, int32_t M, float *inv_a, float *bias) {
    if (M <= 0 || !(a > 0.0f)) return BO_EINVAL;
    double tot = 0.0;
    for (int m = 0; m < M; m++) tot = tot + (double)b[m];
    *inv_a = (float)(1.0 / (double)a);
    *bias = (float)tot;
    return BO_OK;
}

int bo_dequant(const uint16_t *S, int64_t count, float inv_a, float bias, float *out) {
    if (count < 0) return BO_EINVAL;
    for (int64_t i = 0; i < count; i++) {
        float t = (float)S[i] * inv_a;
        out[i] = t + bias;
    }
    return BO_OK;
}

/* uint32 sums (M > 256): the same two roundings; S < 2^24 is exact in fp32. */
int bo_dequant_u32(const uint32_t *S, int64_t count, float inv_a, float bias, float *out) {
    if (count < 0) return BO_EINVAL;
    for (int64_t i = 0; i < count; i++) {
        float t = (float)S[i] * inv_a;
        out[i] = t + bias;
    }
    return BO_OK;
}

/* ---------------------------------------------------------------- matmul
 * Sec. 4.4: rows of A are queries (dot tables), B is the encoded database;
 * out[i][n] = dequantized approximate A_i . B_n, a nested loop of scans. */
int bo_matmul(const float *A, int64_t rows, int32_t J, const uint8_t *codesB,
              int64_t n, int32_t M, const float *C, float a, const float *b,
              float *out) {
    int rc = check_shape(rows, J, M);
    if (rc) return rc;
    float inv_a, bias;
    rc = bo_dequant_params(a, b, M, &inv_a, &bias);
    if (rc) return rc;
    float *D = (float *)malloc(sizeof(float) * (size_t)M * BO_K);
    uint8_t *lut = (uint8_t *)malloc((size_t)M * BO_K);
    uint16_t *S = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)(n > 0 ? n : 1));
    if (!D || !lut || !S) {
        free(D); free(lut); free(S);
        return BO_ENOMEM;
    }
    for (int64_t i = 0; i < rows; i++) {
        bo_lut_f32(A + i * J, 1, J, M, C, BO_METRIC_DOT, D);
        bo_quantize(D, 1, M, a, b, lut);
        rc = bo_scan(codesB, n, M, lut, 1, S);
        if (rc) break;
        bo_dequant(S, n, inv_a, bias, out + i * n);
    }
    free(D); free(lut); free(S);
    return rc;
}
