// Blocked code layout (the vectorized-lookup layout of Sec. 3.2, "encodings
// stored in blocks of at least V elements"): conversions to and from
// row-major one-code-per-byte form.
#include "common.cuh"

namespace bolt {

__global__ void pack_kernel(const uint8_t *__restrict__ rowmajor, int64_t n, int32_t M,
                            uint32_t *__restrict__ blocked, int64_t total_words) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total_words;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / ((int64_t)M * kRowWords);
        const int32_t m = (int32_t)((t / kRowWords) % M);
        const int32_t w = (int32_t)(t % kRowWords);
        const int64_t v0 = b * kBlockVecs + 8 * w;
        uint32_t word = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t v = v0 + i;
            if (v < n) word |= (uint32_t)(rowmajor[v * M + m] & 15u) << (4 * i);
        }
        blocked[t] = word;
    }
}

__global__ void unpack_kernel(const uint32_t *__restrict__ blocked, int64_t n, int32_t M,
                              uint8_t *__restrict__ rowmajor) {
    const int64_t total = n * M;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = t / M;
        const int32_t m = (int32_t)(t % M);
        const int64_t b = v / kBlockVecs;
        const int32_t r = (int32_t)(v % kBlockVecs);
        const uint32_t word = blocked[(b * M + m) * kRowWords + r / 8];
        rowmajor[t] = (uint8_t)((word >> (4 * (r % 8))) & 15u);
    }
}

static int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    int64_t cap = (int64_t)device_sm_count() * 16;
    if (cap <= 0) cap = 1024;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace bolt

extern "C" {

int bolt_pack_codes(const uint8_t *rowmajor, int64_t n, int32_t M, uint8_t *blocked, void *stream) {
    bolt::clear_error();
    int rc = bolt::check_nm_wide(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(blocked && (rowmajor || n == 0), BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(blocked, 16), BOLT_EINVAL, "blocked codes must be 16-byte aligned");
    const int64_t words = bolt::num_blocks(n) * M * bolt::kRowWords;
    if (words == 0) return BOLT_OK;
    bolt::pack_kernel<<<bolt::grid_for(words, 256), 256, 0, (cudaStream_t)stream>>>(
        rowmajor, n, M, reinterpret_cast<uint32_t *>(blocked), words);
    return bolt::check_launch("pack_kernel");
}

int bolt_unpack_codes(const uint8_t *blocked, int64_t n, int32_t M, uint8_t *rowmajor, void *stream) {
    bolt::clear_error();
    int rc = bolt::check_nm_wide(n, M);
    if (rc) return rc;
    BOLT_REQUIRE((blocked && rowmajor) || n == 0, BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(blocked, 16), BOLT_EINVAL, "blocked codes must be 16-byte aligned");
    if (n == 0) return BOLT_OK;
    bolt::unpack_kernel<<<bolt::grid_for(n * M, 256), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const uint32_t *>(blocked), n, M, rowmajor);
    return bolt::check_launch("unpack_kernel");
}

}  // extern "C"
