// Query encoding g (Sec. 3.1, D_im = delta(q^(m), c_i^(m))) and Bolt's
// learned 8-bit quantization of the table (Sec. 3.2, beta_m).
#include "lut.cuh"

namespace bolt {

// Canonical fp32 table entry.  L2: acc = fma(t, t, acc), t = q_j - c_j;
// dot: acc = fma(q_j, c_j, acc); L1: acc = acc + |q_j - c_j|; L_p: acc = acc +
// powf(|q_j - c_j|, p); dims in order, starting from 0.
__device__ __forceinline__ float lut_entry(const float *__restrict__ q, const float *__restrict__ c, int s,
                                           int metric, float p) {
    float acc = 0.0f;
    if (metric == BOLT_METRIC_LP) {
        for (int j = 0; j < s; ++j) acc = __fadd_rn(acc, powf(fabsf(__fsub_rn(q[j], c[j])), p));
    } else if (metric == BOLT_METRIC_L2) {
        for (int j = 0; j < s; ++j) {
            const float t = __fsub_rn(q[j], c[j]);
            acc = __fmaf_rn(t, t, acc);
        }
    } else if (metric == BOLT_METRIC_L1) {
        for (int j = 0; j < s; ++j) acc = __fadd_rn(acc, fabsf(__fsub_rn(q[j], c[j])));
    } else {
        for (int j = 0; j < s; ++j) acc = __fmaf_rn(q[j], c[j], acc);
    }
    return acc;
}

// beta_m(y) = clamp(floor(a (y - b_m)), 0, 255): (y - b_m) and the product by
// a are separately rounded fp32 operations; NaN maps to 0.
__device__ __forceinline__ uint8_t quantize_entry(float y, float a, float b) {
    float t = __fsub_rn(y, b);
    t = __fmul_rn(t, a);
    if (!(t >= 0.0f)) return 0;
    if (t >= 255.0f) return 255;
    return (uint8_t)floorf(t);
}

// b_dev (nullable): the offsets b_m in device memory, for M > 256; else qp.b.
__global__ void build_luts_kernel(const float *__restrict__ Q, int64_t nq, int32_t J, int32_t M,
                                  const float *__restrict__ C, int32_t metric, QuantParams qp,
                                  const float *__restrict__ b_dev, uint8_t *__restrict__ luts,
                                  float *__restrict__ luts_f32, float p) {
    const int s = J / M;
    const int64_t total = nq * M * kK;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t % kK);
        const int m = (int)((t / kK) % M);
        const int64_t q = t / ((int64_t)kK * M);
        const float y = lut_entry(Q + q * J + m * s, C + ((int64_t)m * kK + k) * s, s, metric, p);
        if (luts_f32) luts_f32[t] = y;
        luts[t] = quantize_entry(y, qp.a, b_dev ? b_dev[m] : qp.b[m]);
    }
}

int launch_build_luts(const float *Q, int64_t nq, int32_t J, int32_t M, const float *C, int32_t metric,
                      const QuantParams &qp, uint8_t *luts, float *luts_f32, cudaStream_t stream,
                      const float *b_dev, float p) {
    const int64_t total = nq * M * kK;
    if (total == 0) return BOLT_OK;
    int64_t grid = (total + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 32;
    if (cap > 0 && grid > cap) grid = cap;
    build_luts_kernel<<<(int)grid, 256, 0, stream>>>(Q, nq, J, M, C, metric, qp, b_dev, luts, luts_f32, p);
    return check_launch("build_luts_kernel");
}

int make_quant_params(float a, const float *b_host, int32_t M, QuantParams *qp) {
    BOLT_REQUIRE(b_host, BOLT_EINVAL, "b_host is null");
    BOLT_REQUIRE(M >= 1 && M <= 256, BOLT_EUNSUPPORTED, "M=%d out of range", M);
    qp->a = a;
    for (int m = 0; m < 256; ++m) qp->b[m] = m < M ? b_host[m] : 0.0f;
    return BOLT_OK;
}

}  // namespace bolt

static int build_luts_any(const float *Q, int64_t nq, int32_t J, int32_t M, const float *centroids, int32_t metric,
                          float p, float a, const float *b_host, uint8_t *luts, float *luts_f32, void *stream) {
    int rc = bolt::check_jm_wide(J, M);
    if (rc) return rc;
    BOLT_REQUIRE(nq >= 0, BOLT_EINVAL, "nq=%lld < 0", (long long)nq);
    BOLT_REQUIRE(nq == 0 || (Q && centroids && luts), BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(b_host, BOLT_EINVAL, "b_host is null");
    cudaStream_t s = (cudaStream_t)stream;
    if (M <= 256) {
        bolt::QuantParams qp;
        rc = bolt::make_quant_params(a, b_host, M, &qp);
        if (rc) return rc;
        return bolt::launch_build_luts(Q, nq, J, M, centroids, metric, qp, luts, luts_f32, s, nullptr, p);
    }
    // More offsets than fit in the kernel's parameters: a stream-ordered
    // device copy, freed after the launch.
    if (nq == 0) return BOLT_OK;
    bolt::QuantParams qp;
    qp.a = a;
    for (int m = 0; m < 256; ++m) qp.b[m] = 0.0f;
    float *b_dev = nullptr;
    BOLT_CUDA(cudaMallocAsync(&b_dev, (size_t)M * sizeof(float), s));
    cudaError_t e = cudaMemcpyAsync(b_dev, b_host, (size_t)M * sizeof(float), cudaMemcpyHostToDevice, s);
    rc = e == cudaSuccess ? bolt::launch_build_luts(Q, nq, J, M, centroids, metric, qp, luts, luts_f32, s, b_dev, p)
                          : BOLT_ECUDA;
    cudaFreeAsync(b_dev, s);
    BOLT_REQUIRE(e == cudaSuccess, BOLT_ECUDA, "bolt_build_luts: %s", cudaGetErrorString(e));
    return rc;
}

extern "C" int bolt_build_luts(const float *Q, int64_t nq, int32_t J, int32_t M, const float *centroids,
                               int32_t metric, float a, const float *b_host, uint8_t *luts, float *luts_f32,
                               void *stream) {
    bolt::clear_error();
    BOLT_REQUIRE(metric == BOLT_METRIC_L2 || metric == BOLT_METRIC_DOT || metric == BOLT_METRIC_L1, BOLT_EINVAL,
                 "bad metric %d (L_p tables: bolt_build_luts_lp)", metric);
    return build_luts_any(Q, nq, J, M, centroids, metric, 1.0f, a, b_host, luts, luts_f32, stream);
}

extern "C" int bolt_build_luts_lp(const float *Q, int64_t nq, int32_t J, int32_t M, const float *centroids, float p,
                                  float a, const float *b_host, uint8_t *luts, float *luts_f32, void *stream) {
    bolt::clear_error();
    BOLT_REQUIRE(p > 0.0f && p < INFINITY, BOLT_EINVAL, "exponent p=%g must be positive and finite", (double)p);
    return build_luts_any(Q, nq, J, M, centroids, BOLT_METRIC_LP, p, a, b_host, luts, luts_f32, stream);
}
