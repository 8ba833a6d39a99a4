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
// inputs and the smallest (lowest index on ties) wins.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <mutex>

#include "encode.cuh"
#include "tma.cuh"

namespace bolt {

constexpr int kTcRows = 128;      // vectors per tile: MMA M and TMEM lanes
constexpr int kTcKC = 32;         // dims per chunk: two K = 16 slices
constexpr int kTcStageBytes = kTcRows * kTcKC * 4;  // one 128 x 32 fp32 chunk (TMA box), 16 KB
// 1 s; divided by 10, the bound on draining copies and MMAs in flight after a
// failure (the roles' waits for one another use data_wait_limit_ns())
constexpr uint64_t kTcWait = 1000000000ull;

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
// 16 consecutive fp32 columns of this thread's tensor-memory lane, without
// waiting: the values are valid after tmem_wait_ld(v).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
          "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
        : "r"(taddr));
}
// Wait for this thread's tensor-memory loads; v is an operand so that no use
// of the loaded registers is scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld(float (&v)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                   "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]),
                   "+f"(v[15]));
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

// ------------------------------------------------------------------ warp-specialized pipeline
// Warp roles:
//   warp 0        MMA issuer (one thread) and owner of the tensor memory
//   warp 1        bulk-copy producer: 128 x 32 fp32 chunks into a ring of kWsX stages
//   warps 2..9    converters in two groups of four that take alternate chunks,
//                 one row per thread: fp32 -> bf16 hi/lo tiles (core-matrix
//                 layout) and the squared norm of every subspace
//   warps 10..25  epilogue in four groups of four (one warp per tensor-memory
//                 lane quarter, warp id mod 4); group g takes chunks g, g + 4,
//                 ..., every subspace of them: scores from tensor memory, argmin
//                 with the margin, fp32 re-check of near ties (x read from
//                 global memory), codes
// Each role's warps work on different chunks at once (a warp of a group has
// two or four chunk periods for one chunk), so the latency of one chunk's
// chain of shared-memory, tensor-memory and shuffle steps is covered by the
// other groups' chunks.
// The roles run ahead of one another through rings of mbarriers:
//   xfull/xfree   fp32 stage   (producer -> converters -> producer)
//   afull/afree   bf16 tiles   (converters -> MMA -> converters)
//   accfull/free  accumulators (MMA -> epilogue -> MMA), one tensor-memory
//                 buffer of COLS columns per slot
//   nfull/nfree   norms        (converters -> epilogue -> converters)
// Every wait is bounded (1 s); a role that gives up sets the CTA's failure
// flag, every other role leaves at its next wait, and the CTA waits (bounded)
// for its own copies and MMAs in flight before freeing the tensor memory.
// Ring depths: the bf16 tiles and the accumulators are held until the MMAs
// that use them complete (about 2 us after issue), so both rings hold several
// chunks; the fp32 stages cover the copy latency.
constexpr int kConvGroups = 2;  // converter groups (alternate chunks)
constexpr int kEpiGroups = 4;   // epilogue groups (every fourth chunk)
constexpr int kWsWarps = 2 + 4 * kConvGroups + 4 * kEpiGroups;
constexpr int kWsThreads = kWsWarps * 32;
constexpr int kWsXMax = 6;  // staged fp32 chunks (as many as fit, at least 2)
constexpr int kWsA = 4;     // converted bf16 chunks
constexpr int kMmaWarp = 0, kProducerWarp = 1;
constexpr int kConvWarp0 = 2, kConvWarps = 4 * kConvGroups, kEpiWarp0 = kConvWarp0 + kConvWarps;
constexpr int kABytes = 2 * kTcRows * kTcKC * 2;  // hi tile + lo tile of one chunk, 16 KB
constexpr int kMaxWsB = 8;
constexpr size_t kWsSmemCap = 224 * 1024;
// barrier slots
constexpr int kBarXFull = 0, kBarXFree = kBarXFull + kWsXMax, kBarAFull = kBarXFree + kWsXMax,
              kBarAFree = kBarAFull + kWsA, kBarAccFull = kBarAFree + kWsA, kBarAccFree = kBarAccFull + kMaxWsB,
              kBarNFull = kBarAccFree + kMaxWsB, kBarNFree = kBarNFull + kMaxWsB, kBarCount = kBarNFree + kMaxWsB;

template <int S>
struct WsShape {
    using SH = TcShape<S>;
    static constexpr int NB = SH::COLS >= 128 ? 4 : 8;  // accumulator slots (at most 512 columns)
    static_assert(NB % kEpiGroups == 0 && NB % kConvGroups == 0, "a group's chunks keep their slots");
    static constexpr int NCOLS_USED = NB * SH::COLS;
    static constexpr int NCOL = NCOLS_USED < 32 ? 32 : NCOLS_USED;  // power of two
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// try_wait with a suspend-time hint: a waiting thread sleeps (up to 20 us)
// until the phase completes instead of spinning on issue slots the other
// roles of its scheduler need.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// Wait for phase `par` of bar; false if it does not complete within limit_ns
// (the failure flag is then set) or another role has already failed.
__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t par, volatile uint32_t *fail, uint64_t limit_ns) {
    if (limit_ns < kPollBelowNs) {  // tests of the timeout path: non-blocking polls decide
        const bool ok = mbar_poll_bounded(bar, par, limit_ns);
        if (!ok) *fail = 1u;
        return ok && !*fail;
    }
    if (mbar_try_wait(bar, par)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait_sleep(bar, par)) {
        if (*fail) return false;
        if (globaltimer_ns() - t0 > limit_ns) {
            *fail = 1u;
            return false;
        }
    }
    return true;
}

// Approximate square root (the hardware instruction; relative error far
// below the 1e-4 slack the margin adds).
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed fp32 pairs (each half rounds exactly like the scalar instruction).
__device__ __forceinline__ uint64_t tc_f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t tc_f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t tc_f2_pack(float lo, float hi) {
    return (uint64_t)__float_as_uint(lo) | ((uint64_t)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float tc_f2_lo(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float tc_f2_hi(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

// Canonical fp32 squared distances of x's subvector xr to the candidate
// centroids (bits of mask) of one codebook cb (16 x S floats), in increasing
// index order; the smallest wins, the lower index on ties.
template <int S>
__device__ __forceinline__ uint32_t recheck_argmin(const float (&xr)[S], const float *cb, uint32_t mask) {
    float bd = INFINITY;
    uint32_t code = 0;
    for (uint32_t mm = mask; mm; mm &= mm - 1) {
        const int k = __ffs(mm) - 1;
        const float *cv = cb + k * S;
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const float t = __fsub_rn(xr[j], cv[j]);
            acc = __fmaf_rn(t, t, acc);
        }
        if (acc < bd) {
            bd = acc;
            code = (uint32_t)k;
        }
    }
    return code;
}

template <int S>
__global__ void __launch_bounds__(kWsThreads, 1)
    encode_tc_kernel(const __grid_constant__ CUtensorMap xmap, const float *__restrict__ Xg, int64_t n, int32_t J,
                     int32_t M, const float *__restrict__ C, uint32_t *__restrict__ codes,
                     unsigned long long *__restrict__ n_rechecked, int kWsX, int c_smem, uint64_t wait_ns) {
    using SH = TcShape<S>;
    using WS = WsShape<S>;
    constexpr int NB = WS::NB;
    extern __shared__ __align__(1024) uint8_t tsm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nslices = J / 16;
    const int nchunks = J / kTcKC;

    // shared memory: fp32 stages (1024-aligned, swizzled) | bf16 A tiles | B slices | norms | ||c||^2 |
    //                margin coefficients | fp32 centroids (when c_smem) | barriers | slots
    uint8_t *p = tsm + ((1024u - (smem_u32(tsm) & 1023u)) & 1023u);
    uint8_t *X32 = p;
    p += kWsX * kTcStageBytes;
    uint8_t *A = p;
    p += kWsA * kABytes;
    uint8_t *B = p;  // hi slices, then lo slices
    p += 2 * (size_t)nslices * SH::SLICE_BYTES;
    float *nrm = reinterpret_cast<float *>(p);  // [NB][SPC][128] squared subspace norms
    p += (size_t)NB * SH::SPC * kTcRows * 4;
    float *cn2 = reinterpret_cast<float *>(p);  // [M][16] fp32 ||c_k||^2
    p += (size_t)M * kK * 4;
    float *cmax = reinterpret_cast<float *>(p);  // [M][4]: margin polynomial p0, p1, p2 (rounded up)
    p += (size_t)M * 4 * 4;
    float *csm = reinterpret_cast<float *>(p);  // [M][16][S] fp32 centroids for the re-check
    if (c_smem) p += (size_t)M * kK * S * 4;
    uint64_t *bars = reinterpret_cast<uint64_t *>(p);
    p += kBarCount * 8;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(p);  // [0] TMEM base, [1] rechecks, [2] failure
    volatile uint32_t *fail = tslot + 2;

    // ---- one-time set-up: norms, margin coefficients and the bf16 B slices
    if (c_smem)
        for (int e = tid; e < M * kK * S; e += kWsThreads) csm[e] = C[e];
    for (int mk = tid; mk < M * kK; mk += kWsThreads) {
        const float *c = C + (size_t)mk * S;
        float acc = 0.0f;
        for (int j = 0; j < S; ++j) acc = __fmaf_rn(c[j], c[j], acc);
        cn2[mk] = acc;
    }
    // Margin 4 (eps + eta) = p0 + p1 X + p2 X^2 per codebook (kernel header),
    // with C = max_k ||c_k|| and C2 = max_k ||c_k||^2 in fp64, rounded up.
    for (int m = tid; m < M; m += kWsThreads) {
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
    for (int e = tid; e < nslices * SH::NS * 16; e += kWsThreads) {
        const int T = e / (SH::NS * 16), nn = (e / 16) % SH::NS, k = e % 16;
        float v;
        if (S <= 16) {
            const int m = T * (16 / S) + nn / 16, kk = nn % 16, d = k - S * (nn / 16);
            v = (d >= 0 && d < S) ? C[((size_t)m * kK + kk) * S + d] : 0.0f;
        } else {
            const int m = (16 * T) / S, d0 = 16 * T - m * S;
            v = C[((size_t)m * kK + nn) * S + d0 + k];
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16 *>(B + (size_t)T * SH::SLICE_BYTES + core_off(nn, k, SH::NS)) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(B + (size_t)(nslices + T) * SH::SLICE_BYTES + core_off(nn, k, SH::NS)) = lo;
    }
    if (tid == 0) {
        for (int i = 0; i < kWsXMax; ++i) {
            mbar_init(&bars[kBarXFull + i], 1);
            mbar_init(&bars[kBarXFree + i], 4);
        }
        for (int i = 0; i < kWsA; ++i) {
            mbar_init(&bars[kBarAFull + i], 4);
            mbar_init(&bars[kBarAFree + i], 1);
        }
        for (int i = 0; i < kMaxWsB; ++i) {
            mbar_init(&bars[kBarAccFull + i], 1);
            mbar_init(&bars[kBarAccFree + i], 4);
            mbar_init(&bars[kBarNFull + i], 4);
            mbar_init(&bars[kBarNFree + i], 4);
        }
        tslot[1] = 0;
        tslot[2] = 0;
    }
    fence_mbar_init();
    fence_proxy_async_smem();  // B written by threads, read by the tensor cores
    if (warp == kMmaWarp) {
        tmem_alloc(&tslot[0], WS::NCOL);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot[0];

    const int64_t ntiles = (n + kTcRows - 1) / kTcRows;
    // This CTA's chunks in order: q -> tile blockIdx.x + (q / nchunks) * gridDim.x, dims (q % nchunks) * 32.
    const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t total = (uint32_t)(my_tiles * nchunks);
    unsigned my_rechecks = 0;

    if (warp == kProducerWarp) {
        // ---------------- producer
        if (lane == 0) {
            // stage xs = q % kWsX of round q / kWsX; chunk c of tile t (counters, no divisions)
            uint32_t q = 0, xs = 0, xround = 0;
            int c = 0;
            int64_t t = blockIdx.x;
            for (; q < total; ++q) {
                if (q >= (uint32_t)kWsX && !ws_wait(&bars[kBarXFree + xs], (xround - 1) & 1u, fail, wait_ns)) break;
                mbar_arrive_expect_tx(&bars[kBarXFull + xs], (uint32_t)kTcStageBytes);
                tma_load_2d(X32 + (size_t)xs * kTcStageBytes, &xmap, c * kTcKC, (int)(t * kTcRows), &bars[kBarXFull + xs]);
                if (++xs == (uint32_t)kWsX) {
                    xs = 0;
                    ++xround;
                }
                if (++c == nchunks) {
                    c = 0;
                    t += gridDim.x;
                }
            }
            // copies issued but perhaps not consumed (after a failure): let them land
            if (*fail)
                for (uint32_t j = (q > kWsX ? q - kWsX : 0); j < q; ++j)
                    mbar_wait_bounded(&bars[kBarXFull + j % kWsX], (j / kWsX) & 1u, kTcWait / 10);
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t kIdesc = idesc_bf16_f32(kTcRows, SH::NS);
            // Descriptors of the first A tile and of the first B slice; the
            // others differ only in the start-address field (address >> 4 in
            // bits 0-13, below 2^14 for every shared-memory address), so they
            // are these plus the byte offset >> 4.
            const uint64_t a_desc0 = umma_desc(smem_u32(A), (kTcRows / 8) * 128, 128);
            const uint64_t b_desc0 = umma_desc(smem_u32(B), (SH::NS / 8) * 128, 128);
            uint32_t q = 0;
            int c = 0;  // chunk q % nchunks
            for (; q < total; ++q) {
                const uint32_t a = q % kWsA, bb = q % NB;
                if (!ws_wait(&bars[kBarAFull + a], (q / kWsA) & 1u, fail, wait_ns)) break;
                if (q >= (uint32_t)NB && !ws_wait(&bars[kBarAccFree + bb], ((q / NB) - 1) & 1u, fail, wait_ns)) break;
                tc_fence_after();
                const uint32_t d_base = tmem + bb * SH::COLS;
#pragma unroll
                for (int tl = 0; tl < 2; ++tl) {
                    const int T = c * 2 + tl;
                    const uint64_t ah = a_desc0 + ((a * kABytes + tl * (2 * (kTcRows / 8) * 128)) >> 4);
                    const uint64_t al = ah + ((kTcRows * kTcKC * 2) >> 4);
                    const uint64_t bh = b_desc0 + ((uint32_t)(T * SH::SLICE_BYTES) >> 4);
                    const uint64_t bl = b_desc0 + ((uint32_t)((nslices + T) * SH::SLICE_BYTES) >> 4);
                    const uint32_t dcol = S <= 16 ? tl * SH::NS : 0;
                    tc_mma(d_base + dcol, ah, bh, kIdesc, (S > 16 && tl > 0) ? 1u : 0u);
                    tc_mma(d_base + dcol, ah, bl, kIdesc, 1u);
                    tc_mma(d_base + dcol, al, bh, kIdesc, 1u);
                }
                tc_commit(&bars[kBarAFree + a]);
                tc_commit(&bars[kBarAccFull + bb]);
                if (++c == nchunks) c = 0;
            }
            // MMAs still in flight after a failure: let them finish before the tensor memory is freed
            if (*fail && q > 0) mbar_wait_bounded(&bars[kBarAccFull + (q - 1) % NB], ((q - 1) / NB) & 1u, kTcWait / 10);
        }
    } else if (warp < kEpiWarp0) {
        // ---------------- converters
        const int r = ((warp - kConvWarp0) & 3) * 32 + lane;
        const uint32_t g = (uint32_t)((warp - kConvWarp0) >> 2);  // this warp's group: chunks g, g + kConvGroups, ...
        uint32_t xs = g, xround = 0;                               // stage q % kWsX of round q / kWsX
        for (uint32_t q = g; q < total; q += kConvGroups) {
            const uint32_t a = q % kWsA, bb = q % NB;
            bool ok = ws_wait(&bars[kBarXFull + xs], xround & 1u, fail, wait_ns);
            if (ok && q >= kWsA) ok = ws_wait(&bars[kBarAFree + a], ((q / kWsA) - 1) & 1u, fail, wait_ns);
            if (ok && q >= (uint32_t)NB) ok = ws_wait(&bars[kBarNFree + bb], ((q / NB) - 1) & 1u, fail, wait_ns);
            if (!__all_sync(0xFFFFFFFFu, ok)) break;
            const uint8_t *xs_stage = X32 + (size_t)xs * kTcStageBytes;
            uint8_t *Ab = A + (size_t)a * kABytes;
            uint64_t xn2[SH::SPC];  // squared norm of each subspace, even and odd dims
#pragma unroll
            for (int i = 0; i < SH::SPC; ++i) xn2[i] = 0ull;
#pragma unroll
            for (int kc = 0; kc < kTcKC / 8; ++kc) {
                const float4 lo = *reinterpret_cast<const float4 *>(xs_stage + swz_off(r, 8 * kc));
                const float4 hi = *reinterpret_cast<const float4 *>(xs_stage + swz_off(r, 8 * kc + 4));
                const float v[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                __nv_bfloat162 h[4], l[4];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    h[qq] = __floats2bfloat162_rn(v[2 * qq], v[2 * qq + 1]);
                    const float2 hf = __bfloat1622float2(h[qq]);
                    const uint64_t vv = tc_f2_pack(v[2 * qq], v[2 * qq + 1]);
                    const uint64_t lv = tc_f2_sub(vv, tc_f2_pack(hf.x, hf.y));
                    l[qq] = __floats2bfloat162_rn(tc_f2_lo(lv), tc_f2_hi(lv));
                    xn2[(8 * kc + 2 * qq) / S] = tc_f2_fma(vv, vv, xn2[(8 * kc + 2 * qq) / S]);
                }
                *reinterpret_cast<uint4 *>(Ab + core_off(r, 8 * kc, kTcRows)) = *reinterpret_cast<const uint4 *>(h);
                *reinterpret_cast<uint4 *>(Ab + kTcRows * kTcKC * 2 + core_off(r, 8 * kc, kTcRows)) =
                    *reinterpret_cast<const uint4 *>(l);
            }
#pragma unroll
            for (int i = 0; i < SH::SPC; ++i)
                nrm[((size_t)bb * SH::SPC + i) * kTcRows + r] = __fadd_rn(tc_f2_lo(xn2[i]), tc_f2_hi(xn2[i]));
            fence_proxy_async_smem();  // this thread's A tiles, for the tensor cores
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&bars[kBarAFull + a]);
                mbar_arrive(&bars[kBarXFree + xs]);
                mbar_arrive(&bars[kBarNFull + bb]);
            }
            xs += kConvGroups;
            if (xs >= (uint32_t)kWsX) {
                xs -= kWsX;
                ++xround;
            }
        }
    } else {
        // ---------------- epilogue
        const int lq = warp & 3;                        // tensor-memory lane quarter
        const uint32_t g = (uint32_t)((warp - kEpiWarp0) >> 2);  // chunks g, g + kEpiGroups, ...
        const bool pad_writer = lq == 0;  // writes the padding codes of the last block
        const int r = lq * 32 + lane;     // this thread's row of the tile
        constexpr int PL = SH::SPC >= 2 ? 2 : 1;  // subspaces per tensor-memory load
        // tile and chunk of q, advanced with q (no divisions in the loop)
        int64_t t = blockIdx.x + (int64_t)(g / nchunks) * gridDim.x;
        int c = (int)(g % nchunks);
        for (uint32_t q = g; q < total; q += kEpiGroups) {
            const uint32_t bb = q % NB;
            bool ok = ws_wait(&bars[kBarAccFull + bb], (q / NB) & 1u, fail, wait_ns);
            if (ok) ok = ws_wait(&bars[kBarNFull + bb], (q / NB) & 1u, fail, wait_ns);
            if (!__all_sync(0xFFFFFFFFu, ok)) break;
            tc_fence_after();
            const int64_t v = t * kTcRows + r;
            const bool valid = v < n;
#pragma unroll
            for (int i0 = 0; i0 < SH::SPC; i0 += PL) {
                float d[PL][16];
#pragma unroll
                for (int ii = 0; ii < PL; ++ii)
                    tmem_ld16_nowait(tmem + bb * SH::COLS + ((uint32_t)(lq * 32) << 16) + (uint32_t)((i0 + ii) * 16),
                                     d[ii]);
#pragma unroll
                for (int ii = 0; ii < PL; ++ii) tmem_wait_ld(d[ii]);
#pragma unroll
                for (int ii = 0; ii < PL; ++ii) {
                    const int i = i0 + ii;
                    const int m = c * SH::SPC + i;
                    const float4 *c2 = reinterpret_cast<const float4 *>(cn2 + m * kK);
                    float sc[16];
                    const uint64_t m2 = tc_f2_pack(-2.0f, -2.0f);
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        const float4 cc = c2[k4];
                        const uint64_t s01 = tc_f2_fma(m2, tc_f2_pack(d[ii][4 * k4 + 0], d[ii][4 * k4 + 1]), tc_f2_pack(cc.x, cc.y));
                        const uint64_t s23 = tc_f2_fma(m2, tc_f2_pack(d[ii][4 * k4 + 2], d[ii][4 * k4 + 3]), tc_f2_pack(cc.z, cc.w));
                        sc[4 * k4 + 0] = tc_f2_lo(s01);
                        sc[4 * k4 + 1] = tc_f2_hi(s01);
                        sc[4 * k4 + 2] = tc_f2_lo(s23);
                        sc[4 * k4 + 3] = tc_f2_hi(s23);
                    }
                    // minimum as a tree (fminf is exact: any order gives the same value)
                    float mn[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) mn[k] = fminf(sc[k], sc[k + 8]);
#pragma unroll
                    for (int k = 0; k < 4; ++k) mn[k] = fminf(mn[k], mn[k + 4]);
                    const float best = fminf(fminf(mn[0], mn[2]), fminf(mn[1], mn[3]));
                    // margin 4 (eps + eta) as a quadratic in X with per-codebook coefficients
                    const float Xn = sqrt_approx(nrm[((size_t)bb * SH::SPC + i) * kTcRows + r]) * 1.0001f + 1e-30f;
                    const float4 pc = reinterpret_cast<const float4 *>(cmax)[m];
                    const float lim = best + __fmaf_rn(__fmaf_rn(pc.z, Xn, pc.y), Xn, pc.x);
                    uint32_t mask = 0;
#pragma unroll
                    for (int k = 0; k < 16; ++k) mask |= (sc[k] <= lim ? 1u : 0u) << k;
                    if (!(lim < INFINITY)) mask = 0xFFFFu;  // non-finite scores: check every centroid
                    // a unique candidate is the tensor-core minimum itself
                    uint32_t code = (uint32_t)(__ffs(mask) - 1) & 15u;
                    if (__popc(mask) > 1 && valid) {
                        // canonical fp32 distances of the candidates, in increasing
                        // index order (ties keep the lower index); x's subvector
                        // (16-byte aligned: X is, rows are J % 32 == 0 floats, S % 4 == 0)
                        // is read once
                        const float4 *xv = reinterpret_cast<const float4 *>(Xg + v * J + (int64_t)m * S);
                        float xr[S];
#pragma unroll
                        for (int j4 = 0; j4 < S / 4; ++j4) {
                            const float4 t4 = __ldg(xv + j4);
                            xr[4 * j4 + 0] = t4.x;
                            xr[4 * j4 + 1] = t4.y;
                            xr[4 * j4 + 2] = t4.z;
                            xr[4 * j4 + 3] = t4.w;
                        }
                        // one call site per address space, so that the shared-memory
                        // copy is read with shared-memory loads
                        code = c_smem ? recheck_argmin<S>(xr, csm + (size_t)m * kK * S, mask)
                                      : recheck_argmin<S>(xr, C + (size_t)m * kK * S, mask);
                        ++my_rechecks;
                    }
                    if (!valid) code = 0;
                    uint32_t word = code << (4 * (lane & 7));
                    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
                    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
                    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
                    if ((lane & 7) == 0) codes[((v >> 8) * M + m) * kRowWords + ((v & 255) >> 3)] = word;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&bars[kBarAccFree + bb]);
                mbar_arrive(&bars[kBarNFree + bb]);
            }
            if (pad_writer && t == ntiles - 1 && c == nchunks - 1 && ((t + 1) * kTcRows) % kBlockVecs != 0) {
                // second half of the last block holds padding vectors: code 0
                const int64_t blk = (t * kTcRows) >> 8;
                for (int ee = lane; ee < M * 16; ee += 32)
                    codes[(blk * M + ee / 16) * kRowWords + 16 + (ee % 16)] = 0u;
            }
            c += kEpiGroups;
            while (c >= nchunks) {
                c -= nchunks;
                t += gridDim.x;
            }
        }
    }

    if (my_rechecks) atomicAdd(&tslot[1], my_rechecks);
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem, WS::NCOL);
    }
    if (tid == 0 && n_rechecked) {
        if (*fail) atomicExch(n_rechecked, ~0ull);  // -1: a wait gave up
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
    using WS = WsShape<S>;
    const int nslices = J / 16;
    const size_t fixed = 1024 + kWsA * (size_t)kABytes + 2 * (size_t)nslices * SH::SLICE_BYTES +
                         (size_t)WS::NB * SH::SPC * kTcRows * 4 + (size_t)M * kK * 4 + (size_t)M * 4 * 4 +
                         kBarCount * 8 + 16;
    // fp32 centroids in shared memory for the re-check when they fit beside
    // at least 3 fp32 stages (else it reads them from global memory)
    const size_t cbytes = (size_t)M * kK * S * 4;
    const int c_smem = fixed + cbytes + 3 * (size_t)kTcStageBytes <= kWsSmemCap ? 1 : 0;
    const size_t fixed_c = fixed + (c_smem ? cbytes : 0);
    // fp32 stages: enough bulk copies in flight to cover the memory latency
    // (up to kWsXMax), within kWsSmemCap of shared memory; at least two
    int nx = kWsXMax;
    while (nx > 2 && fixed_c + (size_t)nx * kTcStageBytes > kWsSmemCap) --nx;
    const size_t smem = fixed_c + (size_t)nx * kTcStageBytes;
    if (smem > kWsSmemCap) return launch_encode_fp32(X, n, J, M, C, codes, stream);
    auto kern = encode_tc_kernel<S>;
    int rc = ensure_smem((const void *)kern, smem);
    if (rc) return rc;
    const int64_t ntiles = (n + kTcRows - 1) / kTcRows;
    // CTAs per SM: shared memory, the threads of an SM, and at most 512 / NCOL
    // CTAs holding tensor memory at a time
    int per_sm = (int)((227 * 1024) / (smem + 1024));
    if (per_sm > 2048 / kWsThreads) per_sm = 2048 / kWsThreads;
    if (per_sm > 512 / WS::NCOL) per_sm = 512 / WS::NCOL;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = ntiles;
    const int64_t cap = (int64_t)device_sm_count() * per_sm;
    if (cap > 0 && grid > cap) grid = cap;
    CUtensorMap map;
    rc = make_x_map(X, n, J, &map);
    if (rc) return rc;
    kern<<<(int)grid, kWsThreads, smem, stream>>>(map, X, n, J, M, C, reinterpret_cast<uint32_t *>(codes),
                                                  reinterpret_cast<unsigned long long *>(n_rechecked), nx,
                                                  c_smem, data_wait_limit_ns());
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
