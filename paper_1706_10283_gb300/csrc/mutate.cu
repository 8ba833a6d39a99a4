// Online changes to an encoded database (the paper's setting has vectors
// arrive and change while the database is in use, Sec. 1.3): writing the
// codes of new or changed vectors into given rows of the blocked layout, and
// dropping deleted vectors (a bitmap of dead rows) from top-k lists.
#include "common.cuh"

namespace bolt {

// One thread per (vector, codebook): clear the row's nibble, then set it.
// Vectors that share a 32-bit word may be written by different threads, so
// both steps are atomic on the word.
__global__ void write_codes_kernel(const uint8_t *__restrict__ rowmajor, int64_t count, int32_t M,
                                   const int64_t *__restrict__ rows, uint32_t *__restrict__ blocked, int64_t n_cap,
                                   uint32_t *__restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * M) return;
    const int64_t i = t / M;
    const int m = (int)(t - i * M);
    const int64_t r = rows[i];
    const uint32_t code = rowmajor[i * M + m];
    if (r < 0 || r >= n_cap || code > 15u) {  // rejected: recorded, nothing written
        atomicOr(bad, 1u);
        return;
    }
    const int64_t b = r / kBlockVecs;
    const int w = (int)((r % kBlockVecs) >> 3);
    const int sh = 4 * (int)(r & 7);
    uint32_t *word = blocked + (b * M + m) * kRowWords + w;
    atomicAnd(word, ~(15u << sh));
    atomicOr(word, code << sh);
}

// One warp per query: the first k_out entries of the list whose index is
// not dead, in list order; padding (index -1, sum 0) after them.  A list
// with a failure marker (index -2) stays marked.
__global__ void topk_filter_kernel(const uint16_t *__restrict__ in_sums, const int64_t *__restrict__ in_idx,
                                   int64_t nq, int32_t k_in, const uint32_t *__restrict__ dead, int64_t n_bits,
                                   int32_t k_out, uint16_t *__restrict__ out_sums, int64_t *__restrict__ out_idx) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    const int64_t *ii = in_idx + q * k_in;
    const uint16_t *ss = in_sums + q * k_in;
    bool failed = false;
    for (int j = lane; j < k_in; j += 32) failed |= ii[j] == -2;
    failed = __any_sync(0xFFFFFFFFu, failed);
    int taken = 0;
    for (int j0 = 0; j0 < k_in && taken < k_out; j0 += 32) {
        const int j = j0 + lane;
        int64_t id = j < k_in ? ii[j] : -1;
        const bool live = id >= 0 && !(id < n_bits && ((dead[id >> 5] >> (id & 31)) & 1u));
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, live);
        const int pos = taken + __popc(bal & ((1u << lane) - 1u));
        if (live && pos < k_out) {
            out_idx[q * k_out + pos] = failed ? -2 : id;
            out_sums[q * k_out + pos] = ss[j];
        }
        taken += __popc(bal);
    }
    for (int r = min(taken, k_out) + lane; r < k_out; r += 32) {
        out_idx[q * k_out + r] = failed ? -2 : -1;
        out_sums[q * k_out + r] = 0;
    }
}

}  // namespace bolt

extern "C" {

int bolt_write_codes(const uint8_t *rowmajor, int64_t count, int32_t M, const int64_t *rows, uint8_t *blocked,
                     int64_t n_cap, void *stream) {
    bolt::clear_error();
    int rc = bolt::check_nm(n_cap, M);
    if (rc) return rc;
    BOLT_REQUIRE(count >= 0, BOLT_EINVAL, "count=%lld < 0", (long long)count);
    if (count == 0) return BOLT_OK;
    BOLT_REQUIRE(rowmajor && rows && blocked, BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(blocked, 16), BOLT_EINVAL, "blocked codes must be 16-byte aligned");
    // rows are device data: the kernel checks each against [0, n_cap) and
    // writes nothing for a bad one; the call then reports the error
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *bad = nullptr;
    BOLT_CUDA(cudaMallocAsync(&bad, 4, s));
    BOLT_CUDA(cudaMemsetAsync(bad, 0, 4, s));
    const int64_t threads = count * M;
    const int64_t grid = (threads + 255) / 256;
    BOLT_REQUIRE(grid < (int64_t)1 << 31, BOLT_EINVAL, "too many codes in one call");
    bolt::write_codes_kernel<<<(unsigned)grid, 256, 0, s>>>(rowmajor, count, M, rows,
                                                              reinterpret_cast<uint32_t *>(blocked), n_cap, bad);
    rc = bolt::check_launch("write_codes_kernel");
    uint32_t h = 0;
    cudaError_t e1 = cudaMemcpyAsync(&h, bad, 4, cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFreeAsync(bad, s);
    if (rc) return rc;
    BOLT_REQUIRE(e1 == cudaSuccess && e2 == cudaSuccess, BOLT_ECUDA, "bolt_write_codes: %s",
                 cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    BOLT_REQUIRE(h == 0, BOLT_EINVAL, "bolt_write_codes: a row index was outside [0, n_cap) or a code "
                                      "exceeded 15 (those entries were not written)");
    return BOLT_OK;
}

int bolt_topk_filter(const uint16_t *in_sums, const int64_t *in_idx, int64_t nq, int32_t k_in,
                     const uint32_t *dead_bits, int64_t n_bits, int32_t k_out, uint16_t *out_sums,
                     int64_t *out_idx, void *stream) {
    bolt::clear_error();
    BOLT_REQUIRE(nq >= 0 && k_in >= 1 && k_out >= 1 && k_out <= k_in && n_bits >= 0, BOLT_EINVAL,
                 "bad sizes nq=%lld k_in=%d k_out=%d", (long long)nq, k_in, k_out);
    if (nq == 0) return BOLT_OK;
    BOLT_REQUIRE(in_sums && in_idx && out_sums && out_idx && (dead_bits || n_bits == 0), BOLT_EINVAL,
                 "null pointer");
    const int64_t threads = nq * 32;
    bolt::topk_filter_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        in_sums, in_idx, nq, k_in, dead_bits, n_bits, k_out, out_sums, out_idx);
    return bolt::check_launch("topk_filter_kernel");
}

}  // extern "C"
