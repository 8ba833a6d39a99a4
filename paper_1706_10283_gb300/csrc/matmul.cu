// Dequantization (Sec. 3.2: the per-table reconstructions beta_m/a + b_m
// sum to S/a + sum_m b_m) and the approximate matrix product of Sec. 4.4
// (rows of A are queries with dot tables; the encoded B is the database).
#include "lut.cuh"
#include "scan_tiles.cuh"

namespace bolt {

__device__ __forceinline__ float dequant_one(uint32_t S, float inv_a, float bias) {
    return __fadd_rn(__fmul_rn((float)S, inv_a), bias);
}

template <typename ST>
__global__ void dequantize_kernel(const ST *__restrict__ S, int64_t count, float inv_a, float bias,
                                  float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = dequant_one(S[i], inv_a, bias);
}

template <typename ST>
static int launch_dequantize(const ST *S, int64_t count, float inv_a, float bias, float *out, cudaStream_t s) {
    BOLT_REQUIRE(count >= 0, BOLT_EINVAL, "count < 0");
    if (count == 0) return BOLT_OK;
    BOLT_REQUIRE(S && out, BOLT_EINVAL, "null pointer");
    int64_t grid = (count + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (cap > 0 && grid > cap) grid = cap;
    dequantize_kernel<ST><<<(int)grid, 256, 0, s>>>(S, count, inv_a, bias, out);
    return check_launch("dequantize_kernel");
}

}  // namespace bolt

extern "C" {

int bolt_dequantize(const uint16_t *S, int64_t count, float inv_a, float bias, float *out, void *stream) {
    bolt::clear_error();
    return bolt::launch_dequantize(S, count, inv_a, bias, out, (cudaStream_t)stream);
}

int bolt_dequantize_u32(const uint32_t *S, int64_t count, float inv_a, float bias, float *out, void *stream) {
    bolt::clear_error();
    return bolt::launch_dequantize(S, count, inv_a, bias, out, (cudaStream_t)stream);
}

int bolt_approx_matmul(const float *A, int64_t rows, int32_t J, const uint8_t *codesB, int64_t n, int32_t M,
                       const float *centroids, float a, const float *b_host, float *out, void *stream) {
    bolt::clear_error();
    int rc = bolt::check_jm(J, M);
    if (rc) return rc;
    rc = bolt::check_nm(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(rows >= 0, BOLT_EINVAL, "rows < 0");
    BOLT_REQUIRE(rows <= 65535LL * 8, BOLT_EUNSUPPORTED, "rows=%lld too large per call", (long long)rows);
    if (rows == 0 || n == 0) return BOLT_OK;
    BOLT_REQUIRE(A && codesB && centroids && out, BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(codesB, 16), BOLT_EINVAL, "codes must be 16-byte aligned");
    float inv_a, bias;
    rc = bolt_dequant_params(a, b_host, M, &inv_a, &bias);
    if (rc) return rc;
    bolt::QuantParams qp;
    rc = bolt::make_quant_params(a, b_host, M, &qp);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *luts = nullptr;
    BOLT_CUDA(cudaMallocAsync((void **)&luts, (size_t)rows * M * bolt::kK, s));
    rc = bolt::launch_build_luts(A, rows, J, M, centroids, BOLT_METRIC_DOT, qp, luts, nullptr, s);
    if (rc == BOLT_OK) {
        // tiles of 8 rows of A: each code word prepared once for 8 tables
        rc = bolt::launch_tile_scan<8>(codesB, n, M, luts, rows, bolt::TileOutDequant{out, inv_a, bias}, s,
                                       "approx_matmul (tile_scan_kernel)");
    }
    cudaError_t e = cudaFreeAsync(luts, s);
    if (rc == BOLT_OK && e != cudaSuccess) {
        bolt::set_error("cudaFreeAsync: %s", cudaGetErrorString(e));
        rc = BOLT_ECUDA;
    }
    return rc;
}

}  // extern "C"
