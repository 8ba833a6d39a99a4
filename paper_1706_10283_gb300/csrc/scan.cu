// Bolt scan d^ (Sec. 3.1, sum of the table entries the codes pick; Sec. 3.2
// 8-bit tables and vectorized lookups) and the fused exact top-k used for
// nearest-neighbour and maximum-inner-product search.
#include "scan_tiles.cuh"
#include "topk.cuh"

namespace bolt {

// ------------------------------------------------------------------ plain sums
// One warp per (query, 256-vector block) (grid-stride); lane w owns word w of
// every row.  Used for one query and for small scans.
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

// Several queries: tiles of up to 8 queries (each code word prepared once per
// tile), the (tile, block) tasks split evenly over one wave of CTAs
// (scan_tiles.cuh).
static int launch_scan_sums(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq,
                            uint16_t *sums, cudaStream_t stream) {
    if (n == 0 || nq == 0) return BOLT_OK;
    const int qb = nq >= 8 ? 8 : nq >= 4 ? 4 : nq >= 2 ? 2 : 1;
    const int64_t tile_tasks = (nq + qb - 1) / qb * num_blocks(n);
    // one query, or too few tile tasks to give every SM one (with short
    // codebook loops): one warp per (query, block) spreads the work wider
    if (nq == 1 || (tile_tasks < device_sm_count() && M <= 32)) {
        const int64_t items = num_blocks(n) * nq;
        int64_t grid = (items + 7) / 8;
        const int64_t cap = (int64_t)device_sm_count() * 8;
        if (cap > 0 && grid > cap) grid = cap;
        scan_sums_kernel<<<(int)grid, 256, 0, stream>>>(reinterpret_cast<const uint32_t *>(codes), n, M, luts, nq,
                                                        sums);
        return check_launch("scan_sums_kernel");
    }
    const TileOutSums16 out{sums};
    const char *what = "scan sums (tile_scan_kernel)";
    if (qb == 8) return launch_tile_scan<8>(codes, n, M, luts, nq, out, stream, what);
    if (qb == 4) return launch_tile_scan<4>(codes, n, M, luts, nq, out, stream, what);
    return launch_tile_scan<2>(codes, n, M, luts, nq, out, stream, what);
}

// ------------------------------------------------------------------ uint32 sums
// Any M up to kMaxWideM: the codebooks in chunks of 256, each chunk's sums
// exact in the uint16 form of the lookup core, added into 32-bit sums.
__global__ void __launch_bounds__(256) scan_u32_kernel(const uint32_t *__restrict__ codes, int64_t n, int32_t M,
                                                       const uint8_t *__restrict__ luts, int64_t nq,
                                                       uint32_t *__restrict__ sums) {
    const int lane = threadIdx.x & 31;
    const int64_t nb = num_blocks(n);
    const int64_t items = nb * nq;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < items; item += nwarps) {
        const int64_t q = item / nb;
        const int64_t b = item % nb;
        const uint4 *lut = reinterpret_cast<const uint4 *>(luts + q * M * kK);
        const uint32_t *row = codes + b * M * kRowWords + lane;
        uint32_t tot[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int m0 = 0; m0 < M; m0 += 256) {
            const int m1 = min(M, m0 + 256);
            Acc8 acc;
            acc.zero();
#pragma unroll 4
            for (int m = m0; m < m1; ++m) {
                const uint32_t W = __ldg(row + (int64_t)m * kRowWords);
                acc.add(prep_word(W), __ldg(lut + m));
            }
            uint32_t e_lo, o_lo, e_hi, o_hi;
            acc.finish(e_lo, o_lo, e_hi, o_hi);
            // e = S0 | S2 << 16, o = S1 | S3 << 16 (vectors 0..3), hi: 4..7
            tot[0] += e_lo & 0xFFFFu;
            tot[1] += o_lo & 0xFFFFu;
            tot[2] += e_lo >> 16;
            tot[3] += o_lo >> 16;
            tot[4] += e_hi & 0xFFFFu;
            tot[5] += o_hi & 0xFFFFu;
            tot[6] += e_hi >> 16;
            tot[7] += o_hi >> 16;
        }
        const int64_t v0 = b * kBlockVecs + 8 * lane;
        uint32_t *dst = sums + q * n + v0;
        if (v0 + 8 <= n && aligned(dst, 16)) {
            reinterpret_cast<uint4 *>(dst)[0] = make_uint4(tot[0], tot[1], tot[2], tot[3]);
            reinterpret_cast<uint4 *>(dst)[1] = make_uint4(tot[4], tot[5], tot[6], tot[7]);
        } else {
            for (int i = 0; i < 8 && v0 + i < n; ++i) dst[i] = tot[i];
        }
    }
}

// ------------------------------------------------------------------ float tables
// "Bolt No Quantize" (Sec. 4.2 ablation): the same scan over the fp32 tables
// D, summed in codebook order from 0 with one fp32 add per codebook.  One CTA
// per (query, range of blocks); the query's M x 16 table sits in shared
// memory, each lane looks up its 8 vectors' entries per code word.
constexpr int kFloatThreads = 256;

__global__ void __launch_bounds__(kFloatThreads) scan_float_kernel(const uint32_t *__restrict__ codes, int64_t n,
                                                                  int32_t M, const float *__restrict__ D,
                                                                  float *__restrict__ out, int64_t blocks_per_cta) {
    extern __shared__ float dtab[];  // [M][16]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q = blockIdx.y;
    for (int i = tid; i < M * kK; i += kFloatThreads) dtab[i] = __ldg(D + q * M * kK + i);
    __syncthreads();
    const int64_t nb = num_blocks(n);
    const int64_t b0 = (int64_t)blockIdx.x * blocks_per_cta;
    const int64_t b1 = min(nb, b0 + blocks_per_cta);
    for (int64_t b = b0 + warp; b < b1; b += kFloatThreads / 32) {
        const uint32_t *row = codes + b * M * kRowWords + lane;
        float acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = 0.0f;
#pragma unroll 4
        for (int m = 0; m < M; ++m) {
            const uint32_t W = __ldg(row + (int64_t)m * kRowWords);
            const float *t = dtab + m * kK;
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = __fadd_rn(acc[i], t[(W >> (4 * i)) & 15u]);
        }
        const int64_t v0 = b * kBlockVecs + 8 * lane;
        float *dst = out + q * n + v0;
        if (v0 + 8 <= n && aligned(dst, 16)) {
            reinterpret_cast<float4 *>(dst)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            reinterpret_cast<float4 *>(dst)[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        } else {
            for (int i = 0; i < 8 && v0 + i < n; ++i) dst[i] = acc[i];
        }
    }
}

int launch_scan_u32(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, uint32_t *sums,
                    cudaStream_t stream) {
    const int64_t items = num_blocks(n) * nq;
    int64_t grid = (items + 7) / 8;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (cap > 0 && grid > cap) grid = cap;
    scan_u32_kernel<<<(int)grid, 256, 0, stream>>>(reinterpret_cast<const uint32_t *>(codes), n, M, luts, nq, sums);
    return check_launch("scan_u32_kernel");
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

int bolt_scan_u32(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, uint32_t *sums,
                  void *stream) {
    bolt::clear_error();
    int rc = bolt::check_nm_wide(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(nq >= 0, BOLT_EINVAL, "nq=%lld < 0", (long long)nq);
    if (n == 0 || nq == 0) return BOLT_OK;
    BOLT_REQUIRE(codes && luts && sums, BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(codes, 16) && bolt::aligned(luts, 16), BOLT_EINVAL,
                 "codes and luts must be 16-byte aligned");
    return bolt::launch_scan_u32(codes, n, M, luts, nq, sums, (cudaStream_t)stream);
}

int bolt_scan_float(const uint8_t *codes, int64_t n, int32_t M, const float *luts_f32, int64_t nq, float *out,
                    void *stream) {
    bolt::clear_error();
    int rc = bolt::check_nm(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(nq >= 0, BOLT_EINVAL, "nq=%lld < 0", (long long)nq);
    if (n == 0 || nq == 0) return BOLT_OK;
    BOLT_REQUIRE(codes && luts_f32 && out, BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(codes, 16) && bolt::aligned(luts_f32, 4), BOLT_EINVAL,
                 "codes must be 16-byte aligned");
    BOLT_REQUIRE(nq <= 65535, BOLT_EUNSUPPORTED, "nq=%lld > 65535 per call", (long long)nq);
    const int64_t nb = bolt::num_blocks(n);
    int64_t gx = (int64_t)(bolt::device_sm_count() > 0 ? bolt::device_sm_count() : 1) * 4;
    gx = (gx + nq - 1) / nq;
    if (gx > nb) gx = nb;
    if (gx < 1) gx = 1;
    const int64_t bpc = (nb + gx - 1) / gx;
    gx = (nb + bpc - 1) / bpc;
    const size_t smem = (size_t)M * bolt::kK * 4;
    rc = bolt::ensure_smem((const void *)bolt::scan_float_kernel, smem);
    if (rc) return rc;
    bolt::scan_float_kernel<<<dim3((unsigned)gx, (unsigned)nq), bolt::kFloatThreads, smem, (cudaStream_t)stream>>>(
        reinterpret_cast<const uint32_t *>(codes), n, M, luts_f32, out, bpc);
    return bolt::check_launch("scan_float_kernel");
}

}  // extern "C"
