// Multi-query scan over tiles of queries (Sec. 3.1: the approximate distance
// of a query to a vector is the sum over the M tables of the entries the
// vector's codes pick; Sec. 3.2: vectorized lookups over blocks of codes),
// shared by the uint16 sums scan and the approximate matrix product of
// Sec. 4.4 (rows of A are queries with dot tables, followed by the
// dequantization of Sec. 3.2).
//
// Tasks are (tile of QB queries, 256-vector code block) pairs in tile-major
// order.  Every CTA owns an equal, contiguous share of them, and the grid is
// a whole number of waves of resident CTAs, so every SM does the same work.
// The grid has at least as many CTAs as there are query tiles, so a share
// holds at most one tile's worth of tasks and spans at most two tiles, whose
// tables the CTA stages in shared memory.  The CTA's warps take the share's tasks in turn.
// For a task, each code word of the block is prepared once and looked up in
// the QB tables of the tile; code words are loaded PF codebooks ahead.
#pragma once

#include "scan_core.cuh"

namespace bolt {

constexpr int kTileThreads = 256;

// Epilogue of the sums scan: the 8 uint16 sums of a lane, vectors v0..v0+7 of query q.
struct TileOutSums16 {
    uint16_t *sums;
    __device__ __forceinline__ void operator()(int64_t q, int64_t v0, int64_t n, uint4 packed) const {
        uint16_t *dst = sums + q * n + v0;
        if (v0 + 8 <= n && aligned(dst, 16)) {
            *reinterpret_cast<uint4 *>(dst) = packed;
        } else {
            const uint32_t w[4] = {packed.x, packed.y, packed.z, packed.w};
            for (int i = 0; i < 8 && v0 + i < n; ++i) dst[i] = (uint16_t)(w[i >> 1] >> (16 * (i & 1)));
        }
    }
};

// Epilogue of the approximate matrix product: S / a + sum_m b_m as fp32.
struct TileOutDequant {
    float *out;
    float inv_a, bias;
    __device__ __forceinline__ void operator()(int64_t q, int64_t v0, int64_t n, uint4 packed) const {
        const uint32_t w4[4] = {packed.x, packed.y, packed.z, packed.w};
        float f[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            f[i] = __fadd_rn(__fmul_rn((float)((w4[i >> 1] >> (16 * (i & 1))) & 0xFFFFu), inv_a), bias);
        float *dst = out + q * n + v0;
        if (v0 + 8 <= n && aligned(dst, 16)) {
            reinterpret_cast<float4 *>(dst)[0] = make_float4(f[0], f[1], f[2], f[3]);
            reinterpret_cast<float4 *>(dst)[1] = make_float4(f[4], f[5], f[6], f[7]);
        } else {
            for (int i = 0; i < 8 && v0 + i < n; ++i) dst[i] = f[i];
        }
    }
};

template <int QB, class Out>
__global__ void __launch_bounds__(kTileThreads) tile_scan_kernel(const uint32_t *__restrict__ codes, int64_t n,
                                                                 int32_t M, const uint8_t *__restrict__ luts,
                                                                 int64_t nq, int64_t ntasks, Out out) {
    extern __shared__ uint4 lut_s[];  // [2][QB][M]: the share's first and second query tile
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
        const int64_t q = (rt0 + i / (QB * M)) * QB + qm / M;
        lut_s[i] = q < nq ? lut_g[q * M + qm % M] : make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    int64_t t = t0 + warp;
    if (t >= t1) return;
    int64_t rt = t / nb, b = t - rt * nb;
    for (; t < t1; t += kTileThreads / 32) {
        const uint4 *lt = lut_s + (rt - rt0) * QB * M;
        const int64_t q0 = rt * QB;
        const int nr = (int)min((int64_t)QB, nq - q0);
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
            out(q0 + qq, v0, n, pack_sums(e_lo, o_lo, e_hi, o_hi));
        }
        b += kTileThreads / 32;
        while (b >= nb) {
            b -= nb;
            ++rt;
        }
    }
}

// Whole waves: a multiple of the resident CTAs, at least one CTA per query
// tile (so a share spans at most two tiles); small problems get fewer CTAs,
// so that each has a task for every warp.
template <int QB, class Out>
int launch_tile_scan(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, Out out,
                     cudaStream_t s, const char *what) {
    const size_t smem = 2 * (size_t)QB * M * 16;
    auto kern = tile_scan_kernel<QB, Out>;
    int rc = ensure_smem((const void *)kern, smem);
    if (rc) return rc;
    const int64_t nb = num_blocks(n);
    const int64_t tiles = (nq + QB - 1) / QB;
    const int64_t ntasks = tiles * nb;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTileThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t slots = (int64_t)device_sm_count() * per_sm;
    int64_t grid = slots > 0 ? slots * ((tiles + slots - 1) / slots) : tiles;
    const int64_t warps = kTileThreads / 32;
    if (grid > (ntasks + warps - 1) / warps) grid = (ntasks + warps - 1) / warps;
    if (grid < tiles) grid = tiles;
    BOLT_REQUIRE(grid <= 0x7FFFFFFFLL, BOLT_EUNSUPPORTED, "%s: too many query tiles", what);
    kern<<<(unsigned)grid, kTileThreads, smem, s>>>(reinterpret_cast<const uint32_t *>(codes), n, M, luts, nq,
                                                    ntasks, out);
    return check_launch(what);
}

}  // namespace bolt
