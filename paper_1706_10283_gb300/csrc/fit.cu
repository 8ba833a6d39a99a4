// Offline phase (Sec. 1.3): k-means codebooks (Sec. 3.1 background, PQ
// learns each codebook by k-means) and the lookup-table quantizer (Sec. 3.2,
// b = F^-1(alpha), a = 255 / (F^-1(1 - alpha) - b), alpha by grid search).
// FP64 is used only here: for the centroid means and the quantizer fit.
#include <math.h>

#include <vector>

#include "encode.cuh"
#include "lut.cuh"

namespace bolt {

constexpr int kChunkRows = 2048;  // fixed row chunk of the deterministic mean reduction

// ------------------------------------------------------------------ k-means
// Partial fp64 sums of one fixed chunk of rows.  Thread t owns column
// c = c0 + t (m = c / s, dim j = c % s) and adds the rows of the chunk in row
// order into its 16 per-centroid sums, so the result does not depend on
// scheduling.  The 16 sums (and, for j = 0, the 16 counts) live in shared
// memory slots of that thread, indexed by the row's code: one fp64 add per
// value.
__global__ void kmeans_partial_kernel(const float *__restrict__ X, int64_t n, int32_t J, int32_t M,
                                      const uint32_t *__restrict__ codes, double *__restrict__ psum,
                                      uint32_t *__restrict__ pcnt) {
    extern __shared__ double kms[];
    const int T = blockDim.x, t = threadIdx.x;
    double *sacc = kms;                                          // [kK][T]
    uint32_t *scnt = reinterpret_cast<uint32_t *>(kms + kK * T);  // [kK][T]
    const int s = J / M;
    const int64_t chunk = blockIdx.x;
    const int64_t r0 = chunk * kChunkRows;
    const int64_t r1 = min(n, r0 + kChunkRows);
    for (int c0 = 0; c0 < J; c0 += T) {
        const int c = c0 + t;
        if (c >= J) break;
        const int m = c / s, j = c % s;
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            sacc[k * T + t] = 0.0;
            scnt[k * T + t] = 0u;
        }
        for (int64_t v = r0; v < r1; ++v) {
            const int64_t b = v / kBlockVecs;
            const int r = (int)(v % kBlockVecs);
            const uint32_t word = codes[(b * M + m) * kRowWords + r / 8];
            const int code = (word >> (4 * (r % 8))) & 15;
            sacc[code * T + t] += (double)X[v * J + c];
            if (j == 0) scnt[code * T + t] += 1u;
        }
        double *dst = psum + chunk * (int64_t)J * kK;
#pragma unroll
        for (int k = 0; k < kK; ++k) dst[((int64_t)m * kK + k) * s + j] = sacc[k * T + t];
        if (j == 0) {
#pragma unroll
            for (int k = 0; k < kK; ++k) pcnt[chunk * (int64_t)M * kK + m * kK + k] = scnt[k * T + t];
        }
    }
}

// Sum the chunks in chunk order, divide in fp64, round to fp32; an empty
// cluster keeps its centroid.
__global__ void kmeans_update_kernel(const double *__restrict__ psum, const uint32_t *__restrict__ pcnt,
                                     int64_t nchunks, int32_t J, int32_t M, float *__restrict__ C) {
    const int s = J / M;
    const int64_t total = (int64_t)J * kK;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t mk = e / s;  // m * 16 + k
        double sum = 0.0;
        uint64_t cnt = 0;
        for (int64_t ch = 0; ch < nchunks; ++ch) {
            sum += psum[ch * total + e];
            cnt += pcnt[ch * (int64_t)M * kK + mk];
        }
        if (cnt > 0) C[e] = (float)(sum / (double)cnt);
    }
}

__global__ void kmeans_init_kernel(const float *__restrict__ X, int32_t J, int32_t M, const int64_t *rows,
                                   float *__restrict__ C) {
    const int s = J / M;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < J * kK; e += gridDim.x * blockDim.x) {
        const int j = e % s, k = (e / s) % kK, m = e / (s * kK);
        C[e] = X[rows[k] * J + m * s + j];
    }
}

// ------------------------------------------------------------------ quantizer fit
__constant__ double kAlphas[8] = {0.0, 0.001, 0.002, 0.005, 0.01, 0.02, 0.05, 0.1};

// Order-preserving map of a double to an unsigned 64-bit key.
__device__ __forceinline__ uint64_t dkey(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dval(uint64_t k) {
    const uint64_t b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)b);
}

constexpr int kFitThreads = 1024;

// rank-th smallest (0-based) of {value(i) : i < count} by 8 byte-wise
// histogram passes over the order-preserving keys.  `value` is evaluated on
// the fly.  All threads of the block must call it.
template <typename F>
__device__ uint64_t block_select(F value, int64_t count, int64_t rank, uint32_t *hist, uint64_t *shared_res) {
    uint64_t prefix = 0;
    int64_t kk = rank + 1;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint64_t hmask = shift == 56 ? 0ull : (~0ull << (shift + 8));
        for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
            const uint64_t key = dkey(value(i));
            if ((key & hmask) == (prefix & hmask)) atomicAdd(&hist[(key >> shift) & 255], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t c = 0;
            for (int d = 0; d < 256; ++d) {
                if (c + hist[d] >= kk) {
                    shared_res[0] = prefix | ((uint64_t)d << shift);
                    shared_res[1] = (uint64_t)c;
                    break;
                }
                c += hist[d];
            }
        }
        __syncthreads();
        prefix = shared_res[0];
        kk -= (int64_t)shared_res[1];
        __syncthreads();
    }
    return prefix;
}

// One CTA per grid point alpha.  D: fp32 tables [nqt][M][16].  Outputs per
// alpha: out_a[ai], out_b[ai*M + m], out_loss[ai] (all fp64).
__global__ void __launch_bounds__(kFitThreads) fit_quant_kernel(const float *__restrict__ D, int64_t nqt, int32_t M,
                                                                double *__restrict__ out_a, double *__restrict__ out_b,
                                                                double *__restrict__ out_loss) {
    __shared__ uint32_t hist[256];
    __shared__ uint64_t res[2];
    __shared__ double bm[256];
    __shared__ double red[kFitThreads / 32];
    const int ai = blockIdx.x;
    const double alpha = kAlphas[ai];
    const int64_t nm = nqt * kK;
    const int64_t np = nm * M;
    const int64_t lo = (int64_t)floor(alpha * (double)(nm - 1));
    for (int m = 0; m < M; ++m) {
        auto val = [&](int64_t i) -> double {
            const int64_t q = i / kK, k = i % kK;
            return (double)D[(q * M + m) * kK + k];
        };
        const uint64_t key = block_select(val, nm, lo, hist, res);
        if (threadIdx.x == 0) bm[m] = dval(key);
        __syncthreads();
    }
    const int64_t hi = (int64_t)floor((1.0 - alpha) * (double)(np - 1));
    auto off = [&](int64_t i) -> double {
        const int m = (int)((i / kK) % M);
        return (double)D[i] - bm[m];
    };
    const double upper = dval(block_select(off, np, hi, hist, res));
    const double a = upper > 0.0 ? 255.0 / upper : 1.0;
    double loss = 0.0;
    for (int64_t i = threadIdx.x; i < np; i += blockDim.x) {
        const int m = (int)((i / kK) % M);
        const double y = (double)D[i];
        const double t = floor(a * (y - bm[m]));
        const double beta = t < 0.0 ? 0.0 : (t > 255.0 ? 255.0 : t);
        const double yhat = beta / a + bm[m];
        loss += (yhat - y) * (yhat - y);
    }
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kFitThreads / 32; ++w) tot += red[w];
        out_loss[ai] = tot / (double)np;
        out_a[ai] = a;
        for (int m = 0; m < M; ++m) out_b[ai * M + m] = bm[m];
    }
}

// ------------------------------------------------------------------ host drivers
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

static int fit_quantizer_impl(const float *Qtrain, int64_t nqt, int32_t J, int32_t M, const float *C, int32_t metric,
                              float *a_host, float *b_host, int32_t *alpha_idx_host, cudaStream_t s,
                              float p = 1.0f) {
    DevBuf dD, dOut;
    const size_t nD = (size_t)nqt * M * kK;
    BOLT_CUDA(cudaMalloc(&dD.p, nD * (sizeof(float) + 1)));
    BOLT_CUDA(cudaMalloc(&dOut.p, sizeof(double) * (8 + 8 + 8 * (size_t)M)));
    float *D = static_cast<float *>(dD.p);
    uint8_t *scratch_luts = reinterpret_cast<uint8_t *>(D + nD);
    QuantParams qp;
    qp.a = 1.0f;
    for (int m = 0; m < 256; ++m) qp.b[m] = 0.0f;
    int rc = launch_build_luts(Qtrain, nqt, J, M, C, metric, qp, scratch_luts, D, s, nullptr, p);
    if (rc) return rc;
    double *out_a = static_cast<double *>(dOut.p);
    double *out_loss = out_a + 8;
    double *out_b = out_loss + 8;
    fit_quant_kernel<<<8, kFitThreads, 0, s>>>(D, nqt, M, out_a, out_b, out_loss);
    rc = check_launch("fit_quant_kernel");
    if (rc) return rc;
    std::vector<double> h(8 + 8 + 8 * (size_t)M);
    BOLT_CUDA(cudaMemcpyAsync(h.data(), dOut.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    BOLT_CUDA(cudaStreamSynchronize(s));
    int best = 0;
    for (int i = 1; i < 8; ++i)
        if (h[8 + i] < h[8 + best]) best = i;  // strict: ties keep the smaller alpha
    *a_host = (float)h[best];
    for (int m = 0; m < M; ++m) b_host[m] = (float)h[16 + (size_t)best * M + m];
    if (alpha_idx_host) *alpha_idx_host = best;
    return BOLT_OK;
}

static int kmeans_impl(const float *X, int64_t n, int32_t J, int32_t M, int32_t iters, const int64_t *init_rows_host,
                       float *C, cudaStream_t s) {
    for (int k = 0; k < kK; ++k)
        BOLT_REQUIRE(init_rows_host[k] >= 0 && init_rows_host[k] < n, BOLT_EINVAL, "init row %lld out of range",
                     (long long)init_rows_host[k]);
    const int64_t nchunks = (n + kChunkRows - 1) / kChunkRows;
    DevBuf dRows, dCodes, dSum, dCnt;
    BOLT_CUDA(cudaMalloc(&dRows.p, sizeof(int64_t) * kK));
    BOLT_CUDA(cudaMalloc(&dCodes.p, (size_t)bolt_codes_bytes(n, M)));
    BOLT_CUDA(cudaMalloc(&dSum.p, sizeof(double) * (size_t)nchunks * J * kK));
    BOLT_CUDA(cudaMalloc(&dCnt.p, sizeof(uint32_t) * (size_t)nchunks * M * kK));
    BOLT_CUDA(cudaMemcpyAsync(dRows.p, init_rows_host, sizeof(int64_t) * kK, cudaMemcpyHostToDevice, s));
    kmeans_init_kernel<<<(J * kK + 255) / 256, 256, 0, s>>>(X, J, M, static_cast<int64_t *>(dRows.p), C);
    int rc = check_launch("kmeans_init_kernel");
    if (rc) return rc;
    uint8_t *codes = static_cast<uint8_t *>(dCodes.p);
    for (int it = 0; it < iters; ++it) {
        rc = launch_encode_fp32(X, n, J, M, C, codes, s);
        if (rc) return rc;
        const int threads = J < 256 ? ((J + 31) / 32) * 32 : 256;
        const size_t smem = (size_t)threads * kK * (sizeof(double) + sizeof(uint32_t));
        kmeans_partial_kernel<<<(unsigned)nchunks, threads, smem, s>>>(X, n, J, M, reinterpret_cast<uint32_t *>(codes),
                                                                   static_cast<double *>(dSum.p),
                                                                   static_cast<uint32_t *>(dCnt.p));
        rc = check_launch("kmeans_partial_kernel");
        if (rc) return rc;
        kmeans_update_kernel<<<(J * kK + 255) / 256, 256, 0, s>>>(static_cast<double *>(dSum.p),
                                                                  static_cast<uint32_t *>(dCnt.p), nchunks, J, M, C);
        rc = check_launch("kmeans_update_kernel");
        if (rc) return rc;
    }
    BOLT_CUDA(cudaStreamSynchronize(s));
    return BOLT_OK;
}

}  // namespace bolt

extern "C" {

int bolt_fit_quantizer(const float *Qtrain, int64_t nqt, int32_t J, int32_t M, const float *centroids, int32_t metric,
                       float *a_host, float *b_host, int32_t *alpha_idx_host, void *stream) {
    bolt::clear_error();
    int rc = bolt::check_jm(J, M);
    if (rc) return rc;
    BOLT_REQUIRE(nqt >= 1, BOLT_EINVAL, "need at least one training query");
    BOLT_REQUIRE(metric == BOLT_METRIC_L2 || metric == BOLT_METRIC_DOT || metric == BOLT_METRIC_L1, BOLT_EINVAL,
                 "bad metric %d", metric);
    BOLT_REQUIRE(Qtrain && centroids && a_host && b_host, BOLT_EINVAL, "null pointer");
    return bolt::fit_quantizer_impl(Qtrain, nqt, J, M, centroids, metric, a_host, b_host, alpha_idx_host,
                                    (cudaStream_t)stream);
}

int bolt_fit_quantizer_lp(const float *Qtrain, int64_t nqt, int32_t J, int32_t M, const float *centroids, float p,
                          float *a_host, float *b_host, int32_t *alpha_idx_host, void *stream) {
    bolt::clear_error();
    int rc = bolt::check_jm(J, M);
    if (rc) return rc;
    BOLT_REQUIRE(nqt >= 1, BOLT_EINVAL, "need at least one training query");
    BOLT_REQUIRE(p > 0.0f && p < INFINITY, BOLT_EINVAL, "exponent p=%g must be positive and finite", (double)p);
    BOLT_REQUIRE(Qtrain && centroids && a_host && b_host, BOLT_EINVAL, "null pointer");
    return bolt::fit_quantizer_impl(Qtrain, nqt, J, M, centroids, BOLT_METRIC_LP, a_host, b_host, alpha_idx_host,
                                    (cudaStream_t)stream, p);
}

int bolt_fit_codebooks(const float *X, int64_t n, int32_t J, int32_t M, int32_t iters, const int64_t *init_rows_host,
                       const float *Qtrain, int64_t nqt, int32_t metric, float *centroids, float *a_host,
                       float *b_host, void *stream) {
    bolt::clear_error();
    int rc = bolt::check_jm(J, M);
    if (rc) return rc;
    rc = bolt::check_nm(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(n >= 1 && iters >= 0, BOLT_EINVAL, "need n >= 1 and iters >= 0");
    BOLT_REQUIRE(X && centroids && init_rows_host, BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(X, 16) && bolt::aligned(centroids, 16), BOLT_EINVAL, "X and centroids 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    rc = bolt::kmeans_impl(X, n, J, M, iters, init_rows_host, centroids, s);
    if (rc || Qtrain == nullptr) return rc;
    return bolt_fit_quantizer(Qtrain, nqt, J, M, centroids, metric, a_host, b_host, nullptr, stream);
}

}  // extern "C"
