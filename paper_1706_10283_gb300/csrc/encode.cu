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

// ------------------------------------------------------------------ staged fp32 encoder
// Tiles of 32 rows are copied row by row (1-D bulk copies, 16-byte aligned
// rows) into shared memory with a row stride of an odd number of 16-byte
// units, so the 32 lanes of a warp (lane = row) read their subvectors with
// conflict-free 16-byte loads.  Warp w handles codebooks w, w + 8, ...; the 16
// centroid values of one dim are one broadcast read of the transposed
// centroid copy.  Two centroids are evaluated per packed fp32x2 instruction:
// each half is the same IEEE round-to-nearest operation as the scalar
// canonical order, so the codes are unchanged.
constexpr int kEncRows = 32;
constexpr int kEncThreads = 256;

__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}

int enc_row_stride(int J) {  // floats per shared-memory row
    int units = J / 4 + 1;
    if ((units & 1) == 0) ++units;
    return units * 4;
}

// 16 canonical distances of one subvector, two centroids per fp32x2 op.
// SC > 0: compile-time subspace size (a multiple of 4; 16-byte loads, full
// unroll); SC = 0: runtime size s.
template <int SC>
__device__ __forceinline__ void subspace_dists(const float *xr, const float4 *cm, int s, uint64_t (&acc)[8]) {
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) acc[k2] = 0ull;
    auto step = [&](float xj, int j) {
        const uint64_t x2 = f2_pack(xj, xj);
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
            const float4 c4 = cm[j * 4 + k4];
            uint64_t t2 = f2_sub(x2, f2_pack(c4.x, c4.y));
            acc[2 * k4] = f2_fma(t2, t2, acc[2 * k4]);
            t2 = f2_sub(x2, f2_pack(c4.z, c4.w));
            acc[2 * k4 + 1] = f2_fma(t2, t2, acc[2 * k4 + 1]);
        }
    };
    if (SC > 0) {
#pragma unroll
        for (int j4 = 0; j4 < SC / 4; ++j4) {
            const float4 x4 = reinterpret_cast<const float4 *>(xr)[j4];
            step(x4.x, 4 * j4 + 0);
            step(x4.y, 4 * j4 + 1);
            step(x4.z, 4 * j4 + 2);
            step(x4.w, 4 * j4 + 3);
        }
    } else {
        for (int j = 0; j < s; ++j) step(xr[j], j);
    }
}

template <int SC>
__global__ void __launch_bounds__(kEncThreads) encode_staged_kernel(const float *__restrict__ X, int64_t n, int32_t J,
                                                                    int32_t M, const float *__restrict__ C,
                                                                    uint32_t *__restrict__ codes, int row_stride) {
    extern __shared__ __align__(128) uint8_t esmem[];
    const int s = SC > 0 ? SC : J / M;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *cs = reinterpret_cast<float *>(esmem);                       // [M][s][16]
    float *xbuf = cs + (size_t)J * kK;                                   // 2 x [32][row_stride]
    uint64_t *bars = reinterpret_cast<uint64_t *>(xbuf + 2 * kEncRows * (size_t)row_stride);
    for (int i = tid; i < J * kK; i += kEncThreads) {
        const int j = i % s, k = (i / s) % kK, m = i / (s * kK);
        cs[((size_t)m * s + j) * kK + k] = C[i];
    }
    if (tid < 2) mbar_init(&bars[tid], 1);
    fence_mbar_init();
    __syncthreads();

    const int64_t ntiles = (n + kEncRows - 1) / kEncRows;
    const uint32_t row_bytes = (uint32_t)J * 4u;
    auto issue = [&](int64_t t, int buf) {  // warp 0: one bulk copy per valid row
        const int64_t r0 = t * kEncRows;
        const int rows = (int)min((int64_t)kEncRows, n - r0);
        if (lane == 0) mbar_arrive_expect_tx(&bars[buf], (uint32_t)rows * row_bytes);
        __syncwarp();
        if (lane < rows)
            bulk_g2s(xbuf + ((size_t)buf * kEncRows + lane) * row_stride, X + (r0 + lane) * J, row_bytes, &bars[buf]);
    };
    int64_t t = blockIdx.x;
    if (warp == 0) {
        if (t < ntiles) issue(t, 0);
        if (t + gridDim.x < ntiles) issue(t + gridDim.x, 1);
    }
    uint32_t parbits = 0u;  // bit b: parity of buffer b's next completion
    for (int buf = 0; t < ntiles; t += gridDim.x, buf ^= 1) {
        const bool ok = mbar_wait_bounded(&bars[buf], (parbits >> buf) & 1u, 1000000000ull);
        parbits ^= 1u << buf;
        const int64_t r0 = t * kEncRows;
        const bool valid = r0 + lane < n;
        const float *xr = xbuf + ((size_t)buf * kEncRows + lane) * row_stride;
        for (int m = warp; m < M; m += kEncThreads / 32) {
            uint64_t acc[8];
            subspace_dists<SC>(xr + m * s, reinterpret_cast<const float4 *>(cs + (size_t)m * s * kK), s, acc);
            float best = __uint_as_float((uint32_t)acc[0]);
            uint32_t code = 0;
#pragma unroll
            for (int k = 1; k < kK; ++k) {
                const float d = __uint_as_float((uint32_t)(acc[k >> 1] >> (32 * (k & 1))));
                if (d < best) {  // strict: ties keep the lower index
                    best = d;
                    code = (uint32_t)k;
                }
            }
            if (!valid || !ok) code = 0;
            uint32_t word = code << (4 * (lane & 7));
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
            if ((lane & 7) == 0) {
                const int64_t v = r0 + lane;  // first of 8 vectors; r0 is a multiple of 32
                codes[((v >> 8) * M + m) * kRowWords + ((v & 255) >> 3)] = word;
            }
        }
        if (t == ntiles - 1) {
            // words of the last block past the last tile hold padding vectors: code 0
            const int64_t v_end = r0 + kEncRows;
            const int w_end = (int)((v_end & 255) >> 3);
            if (w_end != 0)
                for (int m = warp; m < M; m += kEncThreads / 32)
                    for (int w = w_end + lane; w < kRowWords; w += 32)
                        codes[(((v_end - 1) >> 8) * M + m) * kRowWords + w] = 0u;
        }
        __syncthreads();  // every warp is done with this buffer
        if (warp == 0 && t + 2 * (int64_t)gridDim.x < ntiles) issue(t + 2 * (int64_t)gridDim.x, buf);
    }
}

// Two rows per lane (subspace sizes 4, 8, 16): every broadcast centroid load
// serves both rows' packed updates, and the two rows' accumulators are
// independent chains.  64-row tiles, 512 threads (warp w takes subspaces w,
// w + 16, ...; lane l rows l and l + 32 of the tile).
constexpr int kEnc2Rows = 64;
constexpr int kEnc2Threads = 512;

template <int SC>
__device__ __forceinline__ void subspace_dists2(const float *xa, const float *xb, const float4 *cm,
                                                uint64_t (&acc_a)[8], uint64_t (&acc_b)[8]) {
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) acc_a[k2] = acc_b[k2] = 0ull;
#pragma unroll
    for (int j4 = 0; j4 < SC / 4; ++j4) {
        const float4 a4 = reinterpret_cast<const float4 *>(xa)[j4];
        const float4 b4 = reinterpret_cast<const float4 *>(xb)[j4];
        const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = 4 * j4 + jj;
            const uint64_t xa2 = f2_pack(av[jj], av[jj]), xb2 = f2_pack(bv[jj], bv[jj]);
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
                const float4 c4 = cm[j * 4 + k4];
                const uint64_t c01 = f2_pack(c4.x, c4.y), c23 = f2_pack(c4.z, c4.w);
                uint64_t t = f2_sub(xa2, c01);
                acc_a[2 * k4] = f2_fma(t, t, acc_a[2 * k4]);
                t = f2_sub(xa2, c23);
                acc_a[2 * k4 + 1] = f2_fma(t, t, acc_a[2 * k4 + 1]);
                t = f2_sub(xb2, c01);
                acc_b[2 * k4] = f2_fma(t, t, acc_b[2 * k4]);
                t = f2_sub(xb2, c23);
                acc_b[2 * k4 + 1] = f2_fma(t, t, acc_b[2 * k4 + 1]);
            }
        }
    }
}

__device__ __forceinline__ uint32_t argmin16(const uint64_t (&acc)[8]) {
    float best = __uint_as_float((uint32_t)acc[0]);
    uint32_t code = 0;
#pragma unroll
    for (int k = 1; k < kK; ++k) {
        const float d = __uint_as_float((uint32_t)(acc[k >> 1] >> (32 * (k & 1))));
        if (d < best) {  // strict: ties keep the lower index
            best = d;
            code = (uint32_t)k;
        }
    }
    return code;
}

template <int SC>
__global__ void __launch_bounds__(kEnc2Threads, 1) encode_staged2_kernel(const float *__restrict__ X, int64_t n,
                                                                      int32_t J, int32_t M,
                                                                      const float *__restrict__ C,
                                                                      uint32_t *__restrict__ codes, int row_stride) {
    extern __shared__ __align__(128) uint8_t esmem[];
    constexpr int s = SC;
    constexpr int W = kEnc2Threads / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *cs = reinterpret_cast<float *>(esmem);                       // [M][s][16]
    float *xbuf = cs + (size_t)J * kK;                                   // 2 x [64][row_stride]
    uint64_t *bars = reinterpret_cast<uint64_t *>(xbuf + 2 * kEnc2Rows * (size_t)row_stride);
    for (int i = tid; i < J * kK; i += kEnc2Threads) {
        const int j = i % s, k = (i / s) % kK, m = i / (s * kK);
        cs[((size_t)m * s + j) * kK + k] = C[i];
    }
    if (tid < 2) mbar_init(&bars[tid], 1);
    fence_mbar_init();
    __syncthreads();

    const int64_t ntiles = (n + kEnc2Rows - 1) / kEnc2Rows;
    const uint32_t row_bytes = (uint32_t)J * 4u;
    auto issue = [&](int64_t t, int buf) {  // warp 0: one bulk copy per valid row
        const int64_t r0 = t * kEnc2Rows;
        const int rows = (int)min((int64_t)kEnc2Rows, n - r0);
        if (lane == 0) mbar_arrive_expect_tx(&bars[buf], (uint32_t)rows * row_bytes);
        __syncwarp();
        for (int r = lane; r < rows; r += 32)
            bulk_g2s(xbuf + ((size_t)buf * kEnc2Rows + r) * row_stride, X + (r0 + r) * J, row_bytes, &bars[buf]);
    };
    int64_t t = blockIdx.x;
    if (warp == 0) {
        if (t < ntiles) issue(t, 0);
        if (t + gridDim.x < ntiles) issue(t + gridDim.x, 1);
    }
    uint32_t parbits = 0u;  // bit b: parity of buffer b's next completion
    for (int buf = 0; t < ntiles; t += gridDim.x, buf ^= 1) {
        const bool ok = mbar_wait_bounded(&bars[buf], (parbits >> buf) & 1u, 1000000000ull);
        parbits ^= 1u << buf;
        const int64_t r0 = t * kEnc2Rows;
        const bool va = r0 + lane < n, vb = r0 + 32 + lane < n;
        const float *xa = xbuf + ((size_t)buf * kEnc2Rows + lane) * row_stride;
        const float *xb = xa + 32 * (size_t)row_stride;
        for (int m = warp; m < M; m += W) {
            uint64_t acc_a[8], acc_b[8];
            subspace_dists2<SC>(xa + m * s, xb + m * s, reinterpret_cast<const float4 *>(cs + (size_t)m * s * kK),
                                acc_a, acc_b);
            uint32_t ca = (va && ok) ? argmin16(acc_a) : 0u;
            uint32_t cb = (vb && ok) ? argmin16(acc_b) : 0u;
            uint32_t wa = ca << (4 * (lane & 7)), wb = cb << (4 * (lane & 7));
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) {
                wa |= __shfl_xor_sync(0xFFFFFFFFu, wa, off);
                wb |= __shfl_xor_sync(0xFFFFFFFFu, wb, off);
            }
            if ((lane & 7) == 0) {
                const int64_t v = r0 + lane;  // r0 is a multiple of 64: 8-vector groups stay in one block
                codes[((v >> 8) * M + m) * kRowWords + ((v & 255) >> 3)] = wa;
                const int64_t v2 = v + 32;
                codes[((v2 >> 8) * M + m) * kRowWords + ((v2 & 255) >> 3)] = wb;
            }
        }
        if (t == ntiles - 1) {
            // words of the last block past the last tile hold padding vectors: code 0
            const int64_t v_end = r0 + kEnc2Rows;
            const int w_end = (int)((v_end & 255) >> 3);
            if (w_end != 0)
                for (int m = warp; m < M; m += W)
                    for (int w = w_end + lane; w < kRowWords; w += 32)
                        codes[(((v_end - 1) >> 8) * M + m) * kRowWords + w] = 0u;
        }
        __syncthreads();  // every warp is done with this buffer
        if (warp == 0 && t + 2 * (int64_t)gridDim.x < ntiles) issue(t + 2 * (int64_t)gridDim.x, buf);
    }
}

int launch_encode_fp32(const float *X, int64_t n, int32_t J, int32_t M, const float *C, uint8_t *codes,
                       cudaStream_t stream) {
    if (J % 4 == 0 && aligned(X, 16)) {
        const int64_t ntiles = (n + kEncRows - 1) / kEncRows;
        if (ntiles == 0) return BOLT_OK;
        const int rs = enc_row_stride(J);
        const int sv = J / M;
        const size_t smem2 = (size_t)J * kK * 4 + 2 * (size_t)kEnc2Rows * rs * 4 + 2 * 8;
        if ((sv == 4 || sv == 8 || sv == 16) && smem2 <= 220 * 1024) {
            const int64_t nt2 = (n + kEnc2Rows - 1) / kEnc2Rows;
            auto kern = sv == 4 ? encode_staged2_kernel<4> : sv == 8 ? encode_staged2_kernel<8> : encode_staged2_kernel<16>;
            int rc = ensure_smem((const void *)kern, smem2);
            if (rc) return rc;
            int per_sm = 0;
            BOLT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kEnc2Threads, smem2));
            int64_t grid = nt2;
            const int64_t cap = (int64_t)device_sm_count() * (per_sm > 0 ? per_sm : 1);
            if (cap > 0 && grid > cap) grid = cap;
            kern<<<(int)grid, kEnc2Threads, smem2, stream>>>(X, n, J, M, C, reinterpret_cast<uint32_t *>(codes), rs);
            return check_launch("encode_staged2_kernel");
        }
        const size_t smem = (size_t)J * kK * 4 + 2 * (size_t)kEncRows * rs * 4 + 2 * 8;
        if (smem <= 220 * 1024) {
            auto kern = sv == 4 ? encode_staged_kernel<4>
                        : sv == 8 ? encode_staged_kernel<8>
                        : sv == 16 ? encode_staged_kernel<16> : encode_staged_kernel<0>;
            int rc = ensure_smem((const void *)kern, smem);
            if (rc) return rc;
            int64_t grid = ntiles;
            const int64_t cap = (int64_t)device_sm_count() * 2;
            if (cap > 0 && grid > cap) grid = cap;
            kern<<<(int)grid, kEncThreads, smem, stream>>>(X, n, J, M, C, reinterpret_cast<uint32_t *>(codes), rs);
            return check_launch("encode_staged_kernel");
        }
    }
    return launch_encode_simple(X, n, J, M, C, codes, stream);
}

int launch_encode_simple(const float *X, int64_t n, int32_t J, int32_t M, const float *C, uint8_t *codes,
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
    int rc = bolt::check_jm_wide(J, M);
    if (rc) return rc;
    rc = bolt::check_nm_wide(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(precision == BOLT_PREC_FP32 || precision == BOLT_PREC_BF16_RECHECK, BOLT_EINVAL,
                 "bad precision %d", precision);
    cudaStream_t s = (cudaStream_t)stream;
    if (n_rechecked) BOLT_CUDA(cudaMemsetAsync(n_rechecked, 0, sizeof(int64_t), s));
    if (n == 0) return BOLT_OK;
    BOLT_REQUIRE(X && centroids && codes, BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(X, 16) && bolt::aligned(codes, 16) && bolt::aligned(centroids, 16), BOLT_EINVAL,
                 "X, centroids and codes must be 16-byte aligned");
    if (precision == BOLT_PREC_BF16_RECHECK && M <= 256 && bolt::encode_tc_supported(J, M))
        return bolt::launch_encode_tc(X, n, J, M, centroids, codes, n_rechecked, s);
    return bolt::launch_encode_fp32(X, n, J, M, centroids, codes, s);
}
