// Dequantization (Sec. 3.2: the per-table reconstructions beta_m/a + b_m
// sum to S/a + sum_m b_m) and the approximate matrix product of Sec. 4.4
// (rows of A are queries with dot tables; the encoded B is the database).
#include "lut.cuh"
#include "scan_core.cuh"

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

// A CTA owns QB rows of A (their tables in shared memory) and strides over
// code blocks, one block per warp: each code word is prepared once and looked
// up in the QB tables.
template <int QB>
__global__ void __launch_bounds__(256) approx_matmul_kernel(const uint32_t *__restrict__ codes, int64_t n,
                                                            int32_t M, const uint8_t *__restrict__ luts,
                                                            int64_t rows, float inv_a, float bias,
                                                            float *__restrict__ out) {
    extern __shared__ uint4 lut_s[];  // [QB][M]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t row0 = (int64_t)blockIdx.y * QB;
    const int nr = (int)min((int64_t)QB, rows - row0);
    const uint4 *lut_g = reinterpret_cast<const uint4 *>(luts);
    for (int i = threadIdx.x; i < QB * M; i += blockDim.x) {
        const int qq = i / M;
        lut_s[i] = qq < nr ? lut_g[(row0 + qq) * M + (i % M)] : make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    const int64_t nb = num_blocks(n);
    for (int64_t b = (int64_t)blockIdx.x * 8 + warp; b < nb; b += (int64_t)gridDim.x * 8) {
        Acc8 acc[QB];
#pragma unroll
        for (int qq = 0; qq < QB; ++qq) acc[qq].zero();
        const uint32_t *row = codes + b * M * kRowWords + lane;
        for (int m = 0; m < M; ++m) {
            const WordSel sel = prep_word(__ldg(row + (int64_t)m * kRowWords));
#pragma unroll
            for (int qq = 0; qq < QB; ++qq) acc[qq].add(sel, lut_s[qq * M + m]);
        }
        const int64_t v0 = b * kBlockVecs + 8 * lane;
#pragma unroll
        for (int qq = 0; qq < QB; ++qq) {
            if (qq >= nr) break;
            uint32_t e_lo, o_lo, e_hi, o_hi;
            acc[qq].finish(e_lo, o_lo, e_hi, o_hi);
            const uint4 pk = pack_sums(e_lo, o_lo, e_hi, o_hi);
            const uint32_t w4[4] = {pk.x, pk.y, pk.z, pk.w};
            float f[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) f[i] = dequant_one((w4[i >> 1] >> (16 * (i & 1))) & 0xFFFFu, inv_a, bias);
            float *dst = out + (row0 + qq) * n + v0;
            if (v0 + 8 <= n && aligned(dst, 16)) {
                reinterpret_cast<float4 *>(dst)[0] = make_float4(f[0], f[1], f[2], f[3]);
                reinterpret_cast<float4 *>(dst)[1] = make_float4(f[4], f[5], f[6], f[7]);
            } else {
                for (int i = 0; i < 8 && v0 + i < n; ++i) dst[i] = f[i];
            }
        }
    }
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
        constexpr int QB = 8;
        const size_t smem = (size_t)QB * M * 16;
        rc = bolt::ensure_smem((const void *)bolt::approx_matmul_kernel<QB>, smem);
        if (rc == BOLT_OK) {
            const int64_t nb = bolt::num_blocks(n);
            const int64_t row_tiles = (rows + QB - 1) / QB;
            int64_t gx = (nb + 7) / 8;
            const int64_t want = (int64_t)bolt::device_sm_count() * 4;
            // enough CTAs to fill the GPU, fewer when row tiles already do
            int64_t gx_cap = want / (row_tiles > 0 ? row_tiles : 1);
            if (gx_cap < 1) gx_cap = 1;
            if (gx > gx_cap) gx = gx_cap;
            dim3 grid((unsigned)gx, (unsigned)row_tiles);
            bolt::approx_matmul_kernel<QB><<<grid, 256, smem, s>>>(reinterpret_cast<const uint32_t *>(codesB), n,
                                                                    M, luts, rows, inv_a, bias, out);
            rc = bolt::check_launch("approx_matmul_kernel");
        }
    }
    cudaError_t e = cudaFreeAsync(luts, s);
    if (rc == BOLT_OK && e != cudaSuccess) {
        bolt::set_error("cudaFreeAsync: %s", cudaGetErrorString(e));
        rc = BOLT_ECUDA;
    }
    return rc;
}

}  // extern "C"
