// Encoder h (Sec. 3.1: i_m = argmin_i d(c_i^(m), x^(m)); K = 16, Sec. 3.2),
// canonical fp32 form: for each (x, m, k) acc = fma(t, t, acc) over the
// subspace's dims in order, t = x_j - c_j; the smallest acc wins, ties to
// the lower k.  Output in the blocked code layout.
#include "encode.cuh"

namespace bolt {

// One CTA of 256 threads per 256-vector block (thread t <-> vector t of the
// block).  Centroids are staged in shared memory transposed to [m][j][k] so
// the 16 centroid values of one dim are one broadcast 64-byte read.
__global__ void __launch_bounds__(256) encode_fp32_kernel(const float *__restrict__ X, int64_t n, int32_t J,
                                                          int32_t M, const float *__restrict__ C,
                                                          uint32_t *__restrict__ codes) {
    extern __shared__ __align__(16) float cs[];  // [M][s][16]
    const int s = J / M;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < J * kK; i += blockDim.x) {
        // i indexes the source layout [m][k][j]
        const int j = i % s;
        const int k = (i / s) % kK;
        const int m = i / (s * kK);
        cs[((size_t)m * s + j) * kK + k] = C[i];
    }
    __syncthreads();
    const int64_t nb = num_blocks(n);
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t v = b * kBlockVecs + tid;
        const bool valid = v < n;
        const float *x = X + (valid ? v : 0) * (int64_t)J;
        for (int m = 0; m < M; ++m) {
            float acc[kK];
#pragma unroll
            for (int k = 0; k < kK; ++k) acc[k] = 0.0f;
            const float4 *cm = reinterpret_cast<const float4 *>(cs + (size_t)m * s * kK);
            for (int j = 0; j < s; ++j) {
                const float xj = valid ? __ldg(x + m * s + j) : 0.0f;
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    const float4 c4 = cm[j * 4 + k4];
                    float t;
                    t = __fsub_rn(xj, c4.x);
                    acc[4 * k4 + 0] = __fmaf_rn(t, t, acc[4 * k4 + 0]);
                    t = __fsub_rn(xj, c4.y);
                    acc[4 * k4 + 1] = __fmaf_rn(t, t, acc[4 * k4 + 1]);
                    t = __fsub_rn(xj, c4.z);
                    acc[4 * k4 + 2] = __fmaf_rn(t, t, acc[4 * k4 + 2]);
                    t = __fsub_rn(xj, c4.w);
                    acc[4 * k4 + 3] = __fmaf_rn(t, t, acc[4 * k4 + 3]);
                }
            }
            float best = acc[0];
            uint32_t code = 0;
#pragma unroll
            for (int k = 1; k < kK; ++k) {
                if (acc[k] < best) {  // strict: ties keep the lower index
                    best = acc[k];
                    code = (uint32_t)k;
                }
            }
            // NaN distances never compare below: code stays 0 as on the host.
            if (!valid) code = 0;
            uint32_t word = code << (4 * (lane & 7));
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
            if ((lane & 7) == 0) codes[(b * M + m) * kRowWords + (tid >> 3)] = word;
        }
    }
}

int launch_encode_fp32(const float *X, int64_t n, int32_t J, int32_t M, const float *C, uint8_t *codes,
                       cudaStream_t stream) {
    const int64_t nb = num_blocks(n);
    if (nb == 0) return BOLT_OK;
    const size_t smem = (size_t)J * kK * sizeof(float);
    BOLT_REQUIRE(smem <= 200 * 1024, BOLT_EUNSUPPORTED, "J=%d too large for the fp32 encoder", J);
    int rc = ensure_smem((const void *)encode_fp32_kernel, smem);
    if (rc) return rc;
    int64_t grid = nb;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (cap > 0 && grid > cap) grid = cap;
    encode_fp32_kernel<<<(int)grid, 256, smem, stream>>>(X, n, J, M, C, reinterpret_cast<uint32_t *>(codes));
    return check_launch("encode_fp32_kernel");
}

}  // namespace bolt

extern "C" int bolt_encode(const float *X, int64_t n, int32_t J, int32_t M, const float *centroids,
                           int32_t precision, uint8_t *codes, int64_t *n_rechecked, void *stream) {
    bolt::clear_error();
    int rc = bolt::check_jm(J, M);
    if (rc) return rc;
    rc = bolt::check_nm(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(precision == BOLT_PREC_FP32 || precision == BOLT_PREC_BF16_RECHECK, BOLT_EINVAL,
                 "bad precision %d", precision);
    cudaStream_t s = (cudaStream_t)stream;
    if (n_rechecked) BOLT_CUDA(cudaMemsetAsync(n_rechecked, 0, sizeof(int64_t), s));
    if (n == 0) return BOLT_OK;
    BOLT_REQUIRE(X && centroids && codes, BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(X, 16) && bolt::aligned(codes, 16) && bolt::aligned(centroids, 16), BOLT_EINVAL,
                 "X, centroids and codes must be 16-byte aligned");
    if (precision == BOLT_PREC_BF16_RECHECK && bolt::encode_tc_supported(J, M))
        return bolt::launch_encode_tc(X, n, J, M, centroids, codes, n_rechecked, s);
    return bolt::launch_encode_fp32(X, n, J, M, centroids, codes, s);
}
