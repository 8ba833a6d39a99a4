// Tensor-core encoder for Bolt's h (Sec. 3.1: i_m = argmin_i d(c_i^(m), x^(m));
// K = 16, Sec. 3.2) on tcgen05 with bf16 operands and fp32 accumulation in
// tensor memory, followed by an fp32 re-check that makes the codes equal to
// the canonical fp32 encoder's.
//
// Scores.  argmin_k ||x - c_k||^2 = argmin_k (||c_k||^2 - 2 x.c_k) per subspace.
// A K = 16 slice of the dims covers 16/s subspaces (s = J/M in {4, 8, 16}; for
// s = 32 two slices accumulate one subspace), so one MMA of shape
// 128 x (256/s) x 16 computes x.c for 128 vectors against all centroids of
// those subspaces: B is the block-diagonal centroid slice (zeros outside each
// centroid's own dims).
//
// Split operands.  Every fp32 operand v is held as two bf16 values, hi =
// bf16(v) and lo = bf16(v - hi), and each slice takes three MMAs into the same
// fp32 accumulator: hi.hi + hi.lo + lo.hi.  The dropped terms (lo.lo and the
// rounding of lo) are below 3.02 * 2^-16 |x||c| per product, so
//   |dot_k - x.c_k| <= E1 * sum_j |x_j||c_kj|,  E1 = 4 * 2^-16 + (3s + 4) * 2^-23
// (2^-23 per fp32 accumulation step in the tensor core).
//
// Margin.  For each (vector, subspace) the score S_k = ||c_k||^2 - 2 dot_k
// differs from the exact s_k = ||c_k||^2 - 2 x.c_k by at most
//   eps = 2 E1 X C + (s+3) u (C2 + 2 X C)
// (u = 2^-24; X >= ||x^(m)||, C >= max_k ||c_k||, C2 >= max_k ||c_k||^2, and
// sum_j |x_j||c_kj| <= X C by Cauchy-Schwarz) and the
// canonical fp32 distance D_k differs from the exact ||x - c_k||^2 by at most
// eta = (s+3) u (X + C)^2.  A centroid with S_k > S_best + 2 (eps + eta)
// therefore has D_k > D_best and cannot be the canonical argmin; the kernel
// uses twice that margin.  When more than one centroid lies inside it, the
// canonical fp32 distances of those candidates are recomputed from the fp32
// inputs in shared memory and the smallest (lowest index on ties) wins.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <mutex>

#include "encode.cuh"
#include "tma.cuh"

namespace bolt {

constexpr int kTcRows = 128;      // vectors per tile: MMA M and TMEM lanes
constexpr int kTcThreads = 128;   // thread r owns row r (TMEM lane r)
constexpr int kTcKC = 32;         // dims per chunk: two K = 16 slices
constexpr int kTcStageBytes = kTcRows * kTcKC * 4;  // one 128 x 32 fp32 chunk (TMA box), 16 KB
constexpr int kTcStages = 2;                         // TMA ring depth
constexpr uint64_t kTcWait = 1000000000ull;  // 1 s bound on every wait

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 16 consecutive fp32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor for a K-major operand without swizzle: the
// operand is tiled into core matrices of 8 rows x 16 bytes (8 bf16), each
// stored as 128 contiguous bytes; lbo = byte step between core matrices along
// K, sbo = byte step between 8-row groups; bits 46-47 hold descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor for kind::f16: D fp32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Byte offset of element (row, k) in a K-major no-swizzle tile with `rows` rows.
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k, int rows) {
    return (uint32_t)(((k >> 3) * (rows >> 3) + (row >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <int S>
struct TcShape {
    static constexpr int SPC = kTcKC / S;                   // subspaces per chunk
    static constexpr int NS = S <= 16 ? 256 / S : 16;       // MMA N per slice
    static constexpr int COLS = SPC * 16;                   // TMEM columns per chunk
    static constexpr int NCOL = 2 * COLS < 32 ? 32 : 2 * COLS;  // two accumulator buffers (power of 2)
    static constexpr int SLICE_BYTES = NS * 16 * 2;         // bf16 B tile per K slice
};

// Element (r, j) of a staged 128 x 32 fp32 chunk written by TMA with the
// 128-byte swizzle: row r is 128 bytes, its 16-byte unit u sits at unit
// u ^ (r & 7), so the 8 rows a quarter-warp reads hit 8 different banks.
__device__ __forceinline__ uint32_t swz_off(int r, int j) {
    return (uint32_t)(r * 128 + ((((j >> 2) ^ (r & 7))) << 4) + (j & 3) * 4);
}

// 2-D tiled TMA load of box (32 dims, 128 rows) at (x = dim, y = row).

// Canonical fp32 distance (the encoder's definition) of subvector (r, dims
// j0..j0+s) of a staged chunk to one centroid c (s contiguous floats).
__device__ __forceinline__ float canon_dist(const uint8_t *stage, int r, int j0, const float *__restrict__ c, int s) {
    float acc = 0.0f;
    for (int j = 0; j < s; ++j) {
        const float x = *reinterpret_cast<const float *>(stage + swz_off(r, j0 + j));
        const float t = __fsub_rn(x, __ldg(c + j));
        acc = __fmaf_rn(t, t, acc);
    }
    return acc;
}

template <int S>
__global__ void __launch_bounds__(kTcThreads) encode_tc_kernel(const __grid_constant__ CUtensorMap xmap, int64_t n,
                                                               int32_t J, int32_t M, const float *__restrict__ C,
                                                               uint32_t *__restrict__ codes,
                                                               unsigned long long *__restrict__ n_rechecked) {
    using SH = TcShape<S>;
    extern __shared__ __align__(1024) uint8_t tsm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nslices = J / 16;
    const int nchunks = J / kTcKC;

    // shared memory: fp32 staging x2 (1024-aligned, swizzled) | A tiles | B slices | norms | barriers
    // the swizzled TMA destination must be 1024-byte aligned
    uint8_t *p = tsm + ((1024u - (smem_u32(tsm) & 1023u)) & 1023u);
    uint8_t *X32 = p;
    p += kTcStages * kTcStageBytes;
    uint8_t *A = p;  // two buffers, each a hi tile then a lo tile
    p += 2 * 2 * kTcRows * kTcKC * 2;  // 2 x 16 KB
    uint8_t *B = p;  // hi slices, then lo slices
    p += 2 * (size_t)nslices * SH::SLICE_BYTES;
    float *cn2 = reinterpret_cast<float *>(p);  // [M][16] fp32 ||c_k||^2
    p += (size_t)M * kK * 4;
    float *cmax = reinterpret_cast<float *>(p);  // [M][4]: margin polynomial p0, p1, p2 (rounded up)
    p += (size_t)M * 4 * 4;
    uint64_t *bars = reinterpret_cast<uint64_t *>(p);  // [0..kTcStages): staging; [6], [7]: MMA buffers
    p += 8 * 8;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(p);  // [0] TMEM base, [1] rechecks, [2] failure

    // ---- one-time set-up: norms and the bf16 B slices
    for (int mk = tid; mk < M * kK; mk += kTcThreads) {
        const float *c = C + (size_t)mk * S;
        float acc = 0.0f;
        for (int j = 0; j < S; ++j) acc = __fmaf_rn(c[j], c[j], acc);
        cn2[mk] = acc;
    }
    // Margin 4 (eps + eta) = p0 + p1 X + p2 X^2 per codebook, with
    //   eps + eta = 2 E1 X C + U (C2 + 2 X C) + U (X + C)^2
    // (C = max_k ||c_k||, C2 = max_k ||c_k||^2, computed in fp64 and rounded up).
    for (int m = tid; m < M; m += kTcThreads) {
        double mx = 0.0, mx2 = 0.0;
        for (int k = 0; k < kK; ++k) {
            double d2 = 0.0;
            for (int j = 0; j < S; ++j) {
                const double v = (double)C[((size_t)m * kK + k) * S + j];
                d2 += v * v;
            }
            mx2 = fmax(mx2, d2);
            mx = fmax(mx, sqrt(d2));
        }
        const double Cm = mx * (1.0 + 1e-6) + 1e-30, C2m = mx2 * (1.0 + 1e-6) + 1e-30;
        const double e1 = 4.0 * 1.52587890625e-05 + (double)(3 * S + 4) * 1.1920928955078125e-07;
        const double u = (double)(S + 3) * 5.9604644775390625e-08;
        const double p0 = 4.0 * (u * C2m + u * Cm * Cm);
        const double p1 = 4.0 * (2.0 * e1 * Cm + 2.0 * u * Cm + 2.0 * u * Cm);
        const double p2 = 4.0 * u;
        cmax[4 * m + 0] = (float)(p0 * (1.0 + 1e-6));
        cmax[4 * m + 1] = (float)(p1 * (1.0 + 1e-6));
        cmax[4 * m + 2] = (float)(p2 * (1.0 + 1e-6));
        cmax[4 * m + 3] = 0.0f;
    }
    for (int e = tid; e < nslices * SH::NS * 16; e += kTcThreads) {
        const int T = e / (SH::NS * 16), n = (e / 16) % SH::NS, k = e % 16;
        float v;
        if (S <= 16) {
            const int m = T * (16 / S) + n / 16, kk = n % 16, d = k - S * (n / 16);
            v = (d >= 0 && d < S) ? C[((size_t)m * kK + kk) * S + d] : 0.0f;
        } else {
            const int m = (16 * T) / S, d0 = 16 * T - m * S;
            v = C[((size_t)m * kK + n) * S + d0 + k];
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16 *>(B + (size_t)T * SH::SLICE_BYTES + core_off(n, k, SH::NS)) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(B + (size_t)(nslices + T) * SH::SLICE_BYTES + core_off(n, k, SH::NS)) = lo;
    }
    if (tid == 0) {
        for (int i = 0; i < kTcStages; ++i) mbar_init(&bars[i], 1);
        mbar_init(&bars[6], 1);
        mbar_init(&bars[7], 1);
        tslot[1] = 0;
        tslot[2] = 0;
    }
    fence_mbar_init();
    fence_proxy_async_smem();  // B written by threads, read by the tensor cores
    if (warp == 0) {
        tmem_alloc(&tslot[0], SH::NCOL);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot[0];

    const int64_t ntiles = (n + kTcRows - 1) / kTcRows;
    constexpr uint32_t kIdesc = idesc_bf16_f32(kTcRows, SH::NS);
    const uint32_t a_addr = smem_u32(A), b_addr = smem_u32(B);

    // This CTA's chunks in order: q -> tile blockIdx.x + (q / nchunks) * gridDim.x,
    // dims (q % nchunks) * 32.  Chunk q is staged in ring slot q % kTcStages,
    // converted into A buffer q % 2 and multiplied into TMEM buffer q % 2.
    const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t total = (uint32_t)(my_tiles * nchunks);
    auto q_tile = [&](uint32_t q) -> int64_t { return blockIdx.x + (int64_t)(q / nchunks) * gridDim.x; };
    auto stage = [&](uint32_t q) {  // one TMA per chunk; rows past n read as zeros
        if (tid == 0 && q < total) {
            const int sl = (int)(q % kTcStages);
            mbar_arrive_expect_tx(&bars[sl], (uint32_t)kTcStageBytes);
            tma_load_2d(X32 + (size_t)sl * kTcStageBytes, &xmap, (int)(q % nchunks) * kTcKC,
                        (int)(q_tile(q) * kTcRows), &bars[sl]);
        }
    };
    for (uint32_t q = 0; q < kTcStages; ++q) stage(q);  // fill the ring; slot q % kTcStages is refilled
                                                         // with chunk q + kTcStages after chunk q's epilogue

    bool failed = false;
    unsigned my_rechecks = 0;
    float xn_prev[SH::SPC];
#pragma unroll
    for (int i = 0; i < SH::SPC; ++i) xn_prev[i] = 0.0f;
    for (uint32_t g = 0; g <= total; ++g) {
        float xn[SH::SPC];
#pragma unroll
        for (int i = 0; i < SH::SPC; ++i) xn[i] = 0.0f;
        if (g < total) {
            // ---- chunk g: fp32 -> bf16 hi/lo A tiles and subspace norms; MMAs
            const int sl = (int)(g % kTcStages);
            const bool ok_x = mbar_wait_bounded(&bars[sl], (g / kTcStages) & 1u, kTcWait);
            if (__syncthreads_or(!ok_x)) {
                failed = true;
                break;
            }
            const uint8_t *xs_stage = X32 + (size_t)sl * kTcStageBytes;
            uint8_t *Ab = A + (size_t)(g & 1u) * (2 * kTcRows * kTcKC * 2);
#pragma unroll
            for (int kc = 0; kc < kTcKC / 8; ++kc) {
                const float4 lo = *reinterpret_cast<const float4 *>(xs_stage + swz_off(tid, 8 * kc));
                const float4 hi = *reinterpret_cast<const float4 *>(xs_stage + swz_off(tid, 8 * kc + 4));
                const float v[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                __nv_bfloat162 h[4], l[4];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    h[qq] = __floats2bfloat162_rn(v[2 * qq], v[2 * qq + 1]);
                    const float2 hf = __bfloat1622float2(h[qq]);
                    l[qq] = __floats2bfloat162_rn(v[2 * qq] - hf.x, v[2 * qq + 1] - hf.y);
                }
                *reinterpret_cast<uint4 *>(Ab + core_off(tid, 8 * kc, kTcRows)) = *reinterpret_cast<const uint4 *>(h);
                *reinterpret_cast<uint4 *>(Ab + kTcRows * kTcKC * 2 + core_off(tid, 8 * kc, kTcRows)) =
                    *reinterpret_cast<const uint4 *>(l);
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) xn[(8 * kc + qq) / S] = __fmaf_rn(v[qq], v[qq], xn[(8 * kc + qq) / S]);
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const int c = (int)(g % nchunks);
                const uint32_t a_base = a_addr + (g & 1u) * (2 * kTcRows * kTcKC * 2);
                const uint32_t d_base = tmem + (g & 1u) * SH::COLS;
#pragma unroll
                for (int tl = 0; tl < 2; ++tl) {
                    const int T = c * 2 + tl;
                    const uint32_t a_off = tl * (2 * (kTcRows / 8) * 128);
                    const uint64_t ah = umma_desc(a_base + a_off, (kTcRows / 8) * 128, 128);
                    const uint64_t al = umma_desc(a_base + kTcRows * kTcKC * 2 + a_off, (kTcRows / 8) * 128, 128);
                    const uint64_t bh = umma_desc(b_addr + T * SH::SLICE_BYTES, (SH::NS / 8) * 128, 128);
                    const uint64_t bl = umma_desc(b_addr + (nslices + T) * SH::SLICE_BYTES, (SH::NS / 8) * 128, 128);
                    const uint32_t dcol = S <= 16 ? tl * SH::NS : 0;
                    tc_mma(d_base + dcol, ah, bh, kIdesc, (S > 16 && tl > 0) ? 1u : 0u);
                    tc_mma(d_base + dcol, ah, bl, kIdesc, 1u);
                    tc_mma(d_base + dcol, al, bh, kIdesc, 1u);
                }
                tc_commit(&bars[6 + (g & 1u)]);
            }
        }
        if (g >= 1) {
            // ---- epilogue of chunk g-1 (its MMAs ran while chunk g was converted)
            const uint32_t e = g - 1;
            const bool ok_m = mbar_wait_bounded(&bars[6 + (e & 1u)], (e >> 1) & 1u, kTcWait);
            if (__syncthreads_or(!ok_m)) {
                failed = true;
                break;
            }
            tc_fence_after();
            const int64_t t = q_tile(e);
            const int c = (int)(e % nchunks);
            const uint8_t *xs_stage = X32 + (size_t)(e % kTcStages) * kTcStageBytes;
            const int64_t v = t * kTcRows + tid;
            const bool valid = v < n;
#pragma unroll
            for (int i = 0; i < SH::SPC; ++i) {
                const int m = c * SH::SPC + i;
                float d[16];
                tmem_ld16(tmem + (e & 1u) * SH::COLS + ((uint32_t)(warp * 32) << 16) + (uint32_t)(i * 16), d);
                const float4 *c2 = reinterpret_cast<const float4 *>(cn2 + m * kK);
                float sc[16];
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    const float4 cc = c2[k4];
                    sc[4 * k4 + 0] = __fmaf_rn(-2.0f, d[4 * k4 + 0], cc.x);
                    sc[4 * k4 + 1] = __fmaf_rn(-2.0f, d[4 * k4 + 1], cc.y);
                    sc[4 * k4 + 2] = __fmaf_rn(-2.0f, d[4 * k4 + 2], cc.z);
                    sc[4 * k4 + 3] = __fmaf_rn(-2.0f, d[4 * k4 + 3], cc.w);
                }
                float best = sc[0];
#pragma unroll
                for (int k = 1; k < 16; ++k) best = fminf(best, sc[k]);
                // margin 4 (eps + eta) as a quadratic in X with per-codebook coefficients
                const float Xn = sqrtf(xn_prev[i]) * 1.0001f + 1e-30f;
                const float4 pc = reinterpret_cast<const float4 *>(cmax)[m];
                const float lim = best + __fmaf_rn(__fmaf_rn(pc.z, Xn, pc.y), Xn, pc.x);
                uint32_t mask = 0;
#pragma unroll
                for (int k = 0; k < 16; ++k) mask |= (sc[k] <= lim ? 1u : 0u) << k;
                if (!(lim < INFINITY)) mask = 0xFFFFu;  // non-finite scores: check every centroid
                // a unique candidate is the tensor-core minimum itself
                uint32_t code = (uint32_t)(__ffs(mask) - 1) & 15u;
                if (__popc(mask) > 1) {
                    float bd = INFINITY;
                    code = 0;
                    for (int k = 0; k < 16; ++k) {
                        if (!(mask & (1u << k))) continue;
                        const float dk = canon_dist(xs_stage, tid, i * S, C + ((size_t)m * kK + k) * S, S);
                        if (dk < bd) {
                            bd = dk;
                            code = (uint32_t)k;
                        }
                    }
                    if (valid) ++my_rechecks;
                }
                if (!valid) code = 0;
                uint32_t word = code << (4 * (lane & 7));
                word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
                word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
                word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
                if ((lane & 7) == 0) codes[((v >> 8) * M + m) * kRowWords + ((v & 255) >> 3)] = word;
            }
            if (t == ntiles - 1 && c == nchunks - 1 && ((t + 1) * kTcRows) % kBlockVecs != 0) {
                // second half of the last block holds padding vectors: code 0
                const int64_t blk = (t * kTcRows) >> 8;
                for (int ee = tid; ee < M * 16; ee += kTcThreads)
                    codes[(blk * M + ee / 16) * kRowWords + 16 + (ee % 16)] = 0u;
            }
            tc_fence_before();
            __syncthreads();  // TMEM buffer e % 2 and ring slot e % kTcStages are free again
            stage(e + kTcStages);
        }
#pragma unroll
        for (int i = 0; i < SH::SPC; ++i) xn_prev[i] = xn[i];
    }
    // Leave cleanly: wait (bounded) for copies in flight, free tensor memory.
    if (failed) {
        // give copies and MMAs still in flight a bounded chance to land before
        // the shared and tensor memory go away
        const uint64_t t0 = globaltimer_ns();
        while (globaltimer_ns() - t0 < kTcWait / 10) {
        }
        if (tid == 0) tslot[2] = 1;
    }
    if (my_rechecks) atomicAdd(&tslot[1], my_rechecks);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, SH::NCOL);
    }
    if (tid == 0 && n_rechecked) {
        if (tslot[2]) atomicExch(n_rechecked, ~0ull);  // -1: a wait gave up
        else if (tslot[1]) atomicAdd(n_rechecked, (unsigned long long)tslot[1]);
    }
}

bool encode_tc_supported(int32_t J, int32_t M) {
    const int s = J / M;
    return (s == 4 || s == 8 || s == 16 || s == 32) && J % kTcKC == 0;
}

static int make_x_map(const float *X, int64_t n, int32_t J, CUtensorMap *map) {
    auto enc = tensor_map_encoder();
    BOLT_REQUIRE(enc, BOLT_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    const cuuint64_t dims[2] = {(cuuint64_t)J, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)J * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kTcKC, (cuuint32_t)kTcRows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)X, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    BOLT_REQUIRE(r == CUDA_SUCCESS, BOLT_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return BOLT_OK;
}

template <int S>
static int launch_tc(const float *X, int64_t n, int32_t J, int32_t M, const float *C, uint8_t *codes,
                     int64_t *n_rechecked, cudaStream_t stream) {
    using SH = TcShape<S>;
    const int nslices = J / 16;
    const size_t smem = 1024 + kTcStages * (size_t)kTcStageBytes + 2 * 2 * (size_t)kTcRows * kTcKC * 2 +
                        2 * (size_t)nslices * SH::SLICE_BYTES + (size_t)M * kK * 4 + (size_t)M * 4 * 4 + 8 * 8 + 16;
    if (smem > 200 * 1024) return launch_encode_fp32(X, n, J, M, C, codes, stream);
    auto kern = encode_tc_kernel<S>;
    int rc = ensure_smem((const void *)kern, smem);
    if (rc) return rc;
    const int64_t ntiles = (n + kTcRows - 1) / kTcRows;
    // at most 512 / NCOL CTAs may hold tensor memory on one SM at a time;
    // shared memory keeps the resident CTAs per SM within that
    int per_sm = (int)((227 * 1024) / (smem + 1024));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 512 / SH::NCOL) per_sm = 512 / SH::NCOL;
    int64_t grid = ntiles;
    const int64_t cap = (int64_t)device_sm_count() * per_sm;
    if (cap > 0 && grid > cap) grid = cap;
    CUtensorMap map;
    rc = make_x_map(X, n, J, &map);
    if (rc) return rc;
    kern<<<(int)grid, kTcThreads, smem, stream>>>(map, n, J, M, C, reinterpret_cast<uint32_t *>(codes),
                                                  reinterpret_cast<unsigned long long *>(n_rechecked));
    return check_launch("encode_tc_kernel");
}

int launch_encode_tc(const float *X, int64_t n, int32_t J, int32_t M, const float *C, uint8_t *codes,
                     int64_t *n_rechecked, cudaStream_t stream) {
    if (n == 0) return BOLT_OK;
    if (!aligned(X, 16)) return launch_encode_fp32(X, n, J, M, C, codes, stream);
    switch (J / M) {
        case 4: return launch_tc<4>(X, n, J, M, C, codes, n_rechecked, stream);
        case 8: return launch_tc<8>(X, n, J, M, C, codes, n_rechecked, stream);
        case 16: return launch_tc<16>(X, n, J, M, C, codes, n_rechecked, stream);
        default: return launch_tc<32>(X, n, J, M, C, codes, n_rechecked, stream);
    }
}

}  // namespace bolt
