// Exact top-k over the uint32 sums of 1 <= M <= 4096 codebooks (Sec. 3.1:
// the approximate distance sums all M tables; the uint16 form holds it only
// while 255 M <= 65535).  Nearest neighbours for L2 and L1 tables (smallest
// sum), maximum inner product for dot tables (largest sum), ties to the lower
// vector index, as in bolt_topk.
//
// Keys.  s' = S (L2, L1) or 255 M - S (dot), so smaller s' is better for
// every metric; s' < 255 * 4096 < 2^20.
//
// Passes (grid of G CTAs per query, each CTA a contiguous index range):
//   1. the uint32 scan writes every sum (scan.cu, bolt_scan_u32's kernel),
//   2. hist_hi: counts of s' >> 8 (4096 bins) per query,
//   3. hist_lo: inside the bin b* where the running count reaches k' =
//      min(k, n), counts of s' & 255 (256 bins): the exact k'-th key value v*
//      and the number `below` of sums s' < v* follow,
//   4. count_eq: every CTA counts its sums equal to v*,
//   5. select: sums below v* go to the candidate list in any order (there
//      are exactly `below` < k' of them); of the sums equal to v*, the
//      k' - below with the lowest indices are taken, in index order, by a
//      prefix over the CTAs' counts and a block scan inside each CTA,
//   6. sort: one CTA per query sorts the k' keys (s' << 32 | index).
// The candidate list therefore holds exactly k' keys per query whatever the
// number of ties.
#include "common.cuh"

namespace bolt {

constexpr int kU32Hi = 4096, kU32Lo = 256;
constexpr int kU32Threads = 256;
constexpr int kU32Chunk = 16384;  // indices per CTA and query (at most)
constexpr int kU32MaxGrid = 512;
constexpr int kU32MaxK = 1024;

struct U32WS {
    uint32_t *sums;     // [nq][n]
    uint32_t *hi;       // [nq][4096]
    uint32_t *lo;       // [nq][256]
    uint32_t *eq;       // [nq][G] per-CTA counts of sums equal to v*
    uint32_t *nlt;      // [nq] candidates below v* placed so far
    uint64_t *cand;     // [nq][k]
};

static size_t u32_align(size_t x) { return (x + 255) / 256 * 256; }

static int u32_grid(int64_t n) {
    int64_t g = (n + kU32Chunk - 1) / kU32Chunk;
    if (g < 1) g = 1;
    if (g > kU32MaxGrid) g = kU32MaxGrid;
    return (int)g;
}

static size_t u32_header_bytes(int64_t nq, int G) {
    return u32_align((size_t)nq * (kU32Hi + kU32Lo) * 4) + u32_align((size_t)nq * G * 4) + u32_align((size_t)nq * 4);
}

static int64_t u32_workspace_bytes(int64_t n, int64_t nq, int32_t k) {
    const int G = u32_grid(n);
    return (int64_t)(u32_align((size_t)nq * n * 4) + u32_header_bytes(nq, G) + u32_align((size_t)nq * k * 8));
}

static U32WS carve_u32(void *ws, int64_t n, int64_t nq, int32_t k) {
    const int G = u32_grid(n);
    uint8_t *p = static_cast<uint8_t *>(ws);
    U32WS w;
    w.sums = reinterpret_cast<uint32_t *>(p);
    p += u32_align((size_t)nq * n * 4);
    w.hi = reinterpret_cast<uint32_t *>(p);
    w.lo = w.hi + (size_t)nq * kU32Hi;
    p += u32_align((size_t)nq * (kU32Hi + kU32Lo) * 4);
    w.eq = reinterpret_cast<uint32_t *>(p);
    p += u32_align((size_t)nq * G * 4);
    w.nlt = reinterpret_cast<uint32_t *>(p);
    p += u32_align((size_t)nq * 4);
    w.cand = reinterpret_cast<uint64_t *>(p);
    (void)k;
    return w;
}

__device__ __forceinline__ uint32_t key_of(uint32_t S, int32_t metric, uint32_t smax) {
    return metric == BOLT_METRIC_DOT ? smax - S : S;
}

// Block-wide: the smallest bin b with (count of bins <= b) >= kk over the
// global histogram h[0..NB) (kk >= 1 and <= the total); returns b and the
// count of the bins below it.  scratch: NB + 64 words of shared memory.
template <int NB>
__device__ void kth_bin(const uint32_t *__restrict__ h, uint32_t kk, uint32_t *scratch, uint32_t &bin,
                        uint32_t &below) {
    constexpr int PER = NB / kU32Threads;  // bins per thread (NB a multiple of 256 or 256 itself)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *wsum = scratch + NB;
    uint32_t v[PER > 0 ? PER : 1];
    uint32_t local = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        v[i] = __ldcg(h + tid * PER + i);
        local += v[i];
    }
    uint32_t incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    const uint32_t excl = before + incl - local;
    if (excl < kk && kk <= excl + local) {
        uint32_t c = excl;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if (c + v[i] >= kk) {
                wsum[32] = (uint32_t)(tid * PER + i);
                wsum[33] = c;
                break;
            }
            c += v[i];
        }
    }
    __syncthreads();
    bin = wsum[32];
    below = wsum[33];
    __syncthreads();
}

__global__ void __launch_bounds__(kU32Threads) u32_hist_hi_kernel(U32WS w, int64_t n, int32_t metric, uint32_t smax,
                                                                  int64_t per_cta) {
    __shared__ uint32_t h[kU32Hi];
    const int64_t q = blockIdx.y;
    for (int i = threadIdx.x; i < kU32Hi; i += kU32Threads) h[i] = 0;
    __syncthreads();
    const int64_t lo = blockIdx.x * per_cta, hi = min(n, lo + per_cta);
    const uint32_t *s = w.sums + q * n;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kU32Threads) atomicAdd(&h[key_of(s[i], metric, smax) >> 8], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kU32Hi; i += kU32Threads)
        if (h[i]) atomicAdd(&w.hi[q * kU32Hi + i], h[i]);
}

__global__ void __launch_bounds__(kU32Threads) u32_hist_lo_kernel(U32WS w, int64_t n, int32_t metric, uint32_t smax,
                                                                  int64_t per_cta, uint32_t kk) {
    __shared__ uint32_t scratch[kU32Hi + 64];
    __shared__ uint32_t h[kU32Lo];
    const int64_t q = blockIdx.y;
    uint32_t bstar, below;
    kth_bin<kU32Hi>(w.hi + q * kU32Hi, kk, scratch, bstar, below);
    for (int i = threadIdx.x; i < kU32Lo; i += kU32Threads) h[i] = 0;
    __syncthreads();
    const int64_t lo = blockIdx.x * per_cta, hi = min(n, lo + per_cta);
    const uint32_t *s = w.sums + q * n;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kU32Threads) {
        const uint32_t kv = key_of(s[i], metric, smax);
        if ((kv >> 8) == bstar) atomicAdd(&h[kv & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kU32Lo; i += kU32Threads)
        if (h[i]) atomicAdd(&w.lo[q * kU32Lo + i], h[i]);
}

// The exact k'-th key value v* and the count of keys below it.
__device__ __forceinline__ void kth_value(const U32WS &w, int64_t q, uint32_t kk, uint32_t *scratch, uint32_t &vstar,
                                          uint32_t &below) {
    uint32_t bstar, below_hi, lstar, below_lo;
    kth_bin<kU32Hi>(w.hi + q * kU32Hi, kk, scratch, bstar, below_hi);
    kth_bin<kU32Lo>(w.lo + q * kU32Lo, kk - below_hi, scratch, lstar, below_lo);
    vstar = (bstar << 8) | lstar;
    below = below_hi + below_lo;
}

__global__ void __launch_bounds__(kU32Threads) u32_count_eq_kernel(U32WS w, int64_t n, int32_t metric, uint32_t smax,
                                                                   int64_t per_cta, uint32_t kk) {
    __shared__ uint32_t scratch[kU32Hi + 64];
    const int64_t q = blockIdx.y;
    uint32_t vstar, below;
    kth_value(w, q, kk, scratch, vstar, below);
    const int64_t lo = blockIdx.x * per_cta, hi = min(n, lo + per_cta);
    const uint32_t *s = w.sums + q * n;
    uint32_t c = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kU32Threads) c += key_of(s[i], metric, smax) == vstar ? 1u : 0u;
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&w.eq[q * gridDim.x + blockIdx.x], c);
}

__global__ void __launch_bounds__(kU32Threads) u32_select_kernel(U32WS w, int64_t n, int32_t metric, uint32_t smax,
                                                                 int64_t per_cta, uint32_t kk, int32_t k) {
    __shared__ uint32_t scratch[kU32Hi + 64];
    __shared__ uint32_t wcnt[kU32Threads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q = blockIdx.y;
    uint32_t vstar, below;
    kth_value(w, q, kk, scratch, vstar, below);
    const uint32_t need_eq = kk - below;
    // equal keys of the CTAs before this one come first (index order)
    uint32_t off = 0;
    for (int c = lane; c < (int)blockIdx.x; c += 32) off += __ldcg(&w.eq[q * gridDim.x + c]);
    off = __reduce_add_sync(0xFFFFFFFFu, off);
    uint64_t *cand = w.cand + q * k;
    const int64_t lo = blockIdx.x * per_cta, hi = min(n, lo + per_cta);
    const uint32_t *s = w.sums + q * n;
    uint32_t run = 0;  // equal keys of this CTA before the current round
    for (int64_t base = lo; base < hi; base += kU32Threads) {
        const int64_t i = base + tid;
        const uint32_t kv = i < hi ? key_of(s[i], metric, smax) : 0xFFFFFFFFu;
        if (kv < vstar) {
            const uint32_t pos = atomicAdd(&w.nlt[q], 1u);  // < below <= k by the histograms
            if (pos < below) cand[pos] = ((uint64_t)kv << 32) | (uint64_t)i;
        }
        const bool eq = kv == vstar;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, eq);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = 0, tot = 0;
        for (int ww = 0; ww < kU32Threads / 32; ++ww) {
            before += ww < warp ? wcnt[ww] : 0u;
            tot += wcnt[ww];
        }
        const uint32_t rank = off + run + before + __popc(bal & ((1u << lane) - 1u));
        if (eq && rank < need_eq) cand[below + rank] = ((uint64_t)kv << 32) | (uint64_t)i;
        run += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) u32_sort_kernel(U32WS w, int32_t k, uint32_t kk, int32_t metric,
                                                        uint32_t smax, uint32_t *__restrict__ out_sums,
                                                        int64_t *__restrict__ out_idx) {
    __shared__ uint64_t keys[kU32MaxK];
    const int64_t q = blockIdx.x;
    int P = 1;
    while (P < (int)kk) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) keys[i] = i < (int)kk ? __ldcg(w.cand + q * k + i) : ~0ull;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
                const int a = 2 * i - (i & (stride - 1));
                const int b = a + stride;
                const bool asc = (a & size) == 0;
                const uint64_t x = keys[a], y = keys[b];
                if ((x > y) == asc) {
                    keys[a] = y;
                    keys[b] = x;
                }
            }
            __syncthreads();
        }
    }
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        if (r < (int)kk) {
            const uint32_t kv = (uint32_t)(keys[r] >> 32);
            out_sums[q * k + r] = metric == BOLT_METRIC_DOT ? smax - kv : kv;
            out_idx[q * k + r] = (int64_t)(uint32_t)keys[r];
        } else {
            out_sums[q * k + r] = 0;
            out_idx[q * k + r] = -1;
        }
    }
}

int launch_scan_u32(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, uint32_t *sums,
                    cudaStream_t stream);

static int launch_topk_u32(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                           int32_t metric, uint32_t *out_sums, int64_t *out_idx, void *workspace, cudaStream_t s) {
    const U32WS w = carve_u32(workspace, n, nq, k);
    const int G = u32_grid(n);
    BOLT_CUDA(cudaMemsetAsync(w.hi, 0, u32_header_bytes(nq, G), s));  // histograms, per-CTA counts, counters
    const uint32_t smax = 255u * (uint32_t)M;
    const uint32_t kk = (uint32_t)(n < k ? n : k);
    if (kk > 0) {
        int rc = launch_scan_u32(codes, n, M, luts, nq, w.sums, s);
        if (rc) return rc;
        const int64_t per_cta = (n + G - 1) / G;
        const dim3 grid(G, (unsigned)nq);
        u32_hist_hi_kernel<<<grid, kU32Threads, 0, s>>>(w, n, metric, smax, per_cta);
        u32_hist_lo_kernel<<<grid, kU32Threads, 0, s>>>(w, n, metric, smax, per_cta, kk);
        u32_count_eq_kernel<<<grid, kU32Threads, 0, s>>>(w, n, metric, smax, per_cta, kk);
        u32_select_kernel<<<grid, kU32Threads, 0, s>>>(w, n, metric, smax, per_cta, kk, k);
    }
    u32_sort_kernel<<<(unsigned)nq, 1024, 0, s>>>(w, k, kk, metric, smax, out_sums, out_idx);
    return check_launch("topk_u32 kernels");
}

}  // namespace bolt

extern "C" {

int64_t bolt_topk_u32_workspace_bytes(int64_t n, int32_t M, int64_t nq, int32_t k) {
    bolt::clear_error();
    if (bolt::check_nm_wide(n, M) || nq < 0 || k < 1 || k > bolt::kU32MaxK) return -1;
    return bolt::u32_workspace_bytes(n, nq, k);
}

int bolt_topk_u32(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                  int32_t metric, uint32_t *out_sums, int64_t *out_idx, void *workspace, int64_t workspace_bytes,
                  void *stream) {
    bolt::clear_error();
    int rc = bolt::check_nm_wide(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(nq >= 0, BOLT_EINVAL, "nq=%lld < 0", (long long)nq);
    BOLT_REQUIRE(k >= 1 && k <= bolt::kU32MaxK, BOLT_EUNSUPPORTED, "k=%d outside [1, %d]", k, bolt::kU32MaxK);
    BOLT_REQUIRE(bolt::rank_metric_ok(metric), BOLT_EINVAL,
                 "bad metric %d", metric);
    BOLT_REQUIRE(n < (int64_t)1 << 31, BOLT_EUNSUPPORTED, "n=%lld: indices must fit 31 bits", (long long)n);
    BOLT_REQUIRE(nq <= 65535, BOLT_EUNSUPPORTED, "nq=%lld > 65535 per call", (long long)nq);
    if (nq == 0) return BOLT_OK;
    BOLT_REQUIRE(luts && out_sums && out_idx && (codes || n == 0), BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(luts, 16) && (n == 0 || bolt::aligned(codes, 16)), BOLT_EINVAL,
                 "codes and luts must be 16-byte aligned");
    const int64_t need = bolt::u32_workspace_bytes(n, nq, k);
    cudaStream_t s = (cudaStream_t)stream;
    if (workspace == nullptr) {
        void *tmp = nullptr;
        BOLT_CUDA(cudaMallocAsync(&tmp, (size_t)need, s));
        rc = bolt::launch_topk_u32(codes, n, M, luts, nq, k, metric, out_sums, out_idx, tmp, s);
        cudaError_t e = cudaFreeAsync(tmp, s);
        if (rc == BOLT_OK && e != cudaSuccess) {
            bolt::set_error("cudaFreeAsync failed: %s", cudaGetErrorString(e));
            rc = BOLT_ECUDA;
        }
        return rc;
    }
    BOLT_REQUIRE(workspace_bytes >= need, BOLT_ENOMEM, "workspace of %lld bytes < %lld needed",
                 (long long)workspace_bytes, (long long)need);
    BOLT_REQUIRE(bolt::aligned(workspace, 256), BOLT_EINVAL, "workspace must be 256-byte aligned");
    return bolt::launch_topk_u32(codes, n, M, luts, nq, k, metric, out_sums, out_idx, workspace, s);
}

}  // extern "C"
