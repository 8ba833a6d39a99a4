// Bolt scan d^ (Sec. 3.1, sum of the table entries the codes pick; Sec. 3.2
// 8-bit tables and vectorized lookups) and the fused exact top-k used for
// nearest-neighbour and maximum-inner-product search.
#include "scan_core.cuh"
#include "topk.cuh"

namespace bolt {

// ------------------------------------------------------------------ plain sums
// One warp per (query, 256-vector block); lane w owns word w of every row.
__global__ void __launch_bounds__(256) scan_sums_kernel(const uint32_t *__restrict__ codes, int64_t n, int32_t M,
                                                        const uint8_t *__restrict__ luts, int64_t nq,
                                                        uint16_t *__restrict__ sums) {
    const int lane = threadIdx.x & 31;
    const int64_t nb = num_blocks(n);
    const int64_t items = nb * nq;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < items; item += nwarps) {
        const int64_t q = item / nb;
        const int64_t b = item % nb;
        const uint4 *lut = reinterpret_cast<const uint4 *>(luts + q * M * kK);
        const uint32_t *row = codes + b * M * kRowWords + lane;
        Acc8 acc;
        acc.zero();
#pragma unroll 4
        for (int m = 0; m < M; ++m) {
            const uint32_t W = __ldg(row + (int64_t)m * kRowWords);
            acc.add(prep_word(W), __ldg(lut + m));
        }
        uint32_t e_lo, o_lo, e_hi, o_hi;
        acc.finish(e_lo, o_lo, e_hi, o_hi);
        const uint4 packed = pack_sums(e_lo, o_lo, e_hi, o_hi);
        const int64_t v0 = b * kBlockVecs + 8 * lane;
        uint16_t *dst = sums + q * n + v0;
        if (v0 + 8 <= n && aligned(dst, 16)) {
            *reinterpret_cast<uint4 *>(dst) = packed;
        } else {
            const uint32_t w[4] = {packed.x, packed.y, packed.z, packed.w};
            for (int i = 0; i < 8 && v0 + i < n; ++i) dst[i] = (uint16_t)(w[i >> 1] >> (16 * (i & 1)));
        }
    }
}

static int launch_scan_sums(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq,
                            uint16_t *sums, cudaStream_t stream) {
    if (n == 0 || nq == 0) return BOLT_OK;
    const int64_t items = num_blocks(n) * nq;
    int64_t grid = (items + 7) / 8;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (cap > 0 && grid > cap) grid = cap;
    scan_sums_kernel<<<(int)grid, 256, 0, stream>>>(reinterpret_cast<const uint32_t *>(codes), n, M, luts, nq, sums);
    return check_launch("scan_sums_kernel");
}

static int check_scan_args(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq,
                           const void *out) {
    int rc = check_nm(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(nq >= 0, BOLT_EINVAL, "nq=%lld < 0", (long long)nq);
    if (n == 0 || nq == 0) return BOLT_OK;
    BOLT_REQUIRE(codes && luts && out, BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(aligned(codes, 16) && aligned(luts, 16), BOLT_EINVAL, "codes and luts must be 16-byte aligned");
    return BOLT_OK;
}

}  // namespace bolt

extern "C" {

int bolt_scan_l2(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, uint16_t *sums,
                 void *stream) {
    bolt::clear_error();
    int rc = bolt::check_scan_args(codes, n, M, luts, nq, sums);
    if (rc) return rc;
    return bolt::launch_scan_sums(codes, n, M, luts, nq, sums, (cudaStream_t)stream);
}

int bolt_scan_dot(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, uint16_t *sums,
                  void *stream) {
    bolt::clear_error();
    int rc = bolt::check_scan_args(codes, n, M, luts, nq, sums);
    if (rc) return rc;
    return bolt::launch_scan_sums(codes, n, M, luts, nq, sums, (cudaStream_t)stream);
}

}  // extern "C"
