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

// Tasks are (row tile of QB rows of A, code block) pairs in row-tile-major
// order.  Every CTA owns an equal, contiguous share of them, so one wave of
// CTAs does the whole product with the same work per CTA; a share holds at
// most one row tile's worth of tasks (the grid has at least as many CTAs as
// there are row tiles), so it spans at most two row tiles, whose tables the
// CTA stages in shared memory.  The CTA's warps take the share's tasks in
// turn.  For a task, each code word of the block is prepared once and looked
// up in the QB tables of the tile; code words are loaded PF codebooks ahead.
template <int QB>
__global__ void __launch_bounds__(256) approx_matmul_kernel(const uint32_t *__restrict__ codes, int64_t n,
                                                            int32_t M, const uint8_t *__restrict__ luts,
                                                            int64_t rows, float inv_a, float bias,
                                                            float *__restrict__ out, int64_t ntasks) {
    extern __shared__ uint4 lut_s[];  // [2][QB][M]: the share's first and second row tile
    constexpr int PF = 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nb = num_blocks(n);
    const int64_t t0 = (int64_t)blockIdx.x * ntasks / gridDim.x;
    const int64_t t1 = (int64_t)(blockIdx.x + 1) * ntasks / gridDim.x;
    if (t0 >= t1) return;
    const int64_t rt0 = t0 / nb;
    const int ntile = (int)((t1 - 1) / nb - rt0 + 1);  // 1 or 2
    const uint4 *lut_g = reinterpret_cast<const uint4 *>(luts);
    for (int i = threadIdx.x; i < ntile * QB * M; i += blockDim.x) {
        const int qm = i % (QB * M);
        const int64_t row = (rt0 + i / (QB * M)) * QB + qm / M;
        lut_s[i] = row < rows ? lut_g[row * M + qm % M] : make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    int64_t t = t0 + warp;
    if (t >= t1) return;
    int64_t rt = t / nb, b = t - rt * nb;
    for (; t < t1; t += 8) {
        const uint4 *lt = lut_s + (rt - rt0) * QB * M;
        const int64_t row0 = rt * QB;
        const int nr = (int)min((int64_t)QB, rows - row0);
        Acc8 acc[QB];
#pragma unroll
        for (int qq = 0; qq < QB; ++qq) acc[qq].zero();
        const uint32_t *wrow = codes + b * M * kRowWords + lane;
        uint32_t wv[PF];
#pragma unroll
        for (int j = 0; j < PF; ++j) wv[j] = j < M ? __ldg(wrow + (int64_t)j * kRowWords) : 0u;
        for (int m0 = 0; m0 < M; m0 += PF) {
            uint32_t nx[PF];
#pragma unroll
            for (int j = 0; j < PF; ++j)
                nx[j] = m0 + PF + j < M ? __ldg(wrow + (int64_t)(m0 + PF + j) * kRowWords) : 0u;
#pragma unroll
            for (int j = 0; j < PF; ++j) {
                if (m0 + j < M) {
                    const WordSel sel = prep_word(wv[j]);
#pragma unroll
                    for (int qq = 0; qq < QB; ++qq) acc[qq].add(sel, lt[qq * M + m0 + j]);
                }
            }
#pragma unroll
            for (int j = 0; j < PF; ++j) wv[j] = nx[j];
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
        b += 8;
        while (b >= nb) {
            b -= nb;
            ++rt;
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
        const size_t smem = 2 * (size_t)QB * M * 16;
        auto kern = bolt::approx_matmul_kernel<QB>;
        rc = bolt::ensure_smem((const void *)kern, smem);
        if (rc == BOLT_OK) {
            const int64_t nb = bolt::num_blocks(n);
            const int64_t row_tiles = (rows + QB - 1) / QB;
            const int64_t ntasks = row_tiles * nb;
            // one wave: a multiple of the resident CTAs, at least one CTA per row
            // tile (so a share spans at most two tiles), at most one per task
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem) != cudaSuccess || per_sm < 1)
                per_sm = 1;
            const int64_t slots = (int64_t)bolt::device_sm_count() * per_sm;
            int64_t grid = slots > 0 ? slots * ((row_tiles + slots - 1) / slots) : row_tiles;
            if (grid < row_tiles) grid = row_tiles;
            if (grid > ntasks) grid = ntasks;
            kern<<<(unsigned)grid, 256, smem, s>>>(reinterpret_cast<const uint32_t *>(codesB), n, M, luts, rows,
                                                   inv_a, bias, out, ntasks);
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
