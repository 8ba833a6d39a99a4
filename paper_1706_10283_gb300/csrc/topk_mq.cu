// Fused scan + exact top-k for databases larger than the shared-memory size
// class, for one or many queries per launch sequence.
//
// 1. Sample bound (mq_sample_kernel).  For every query, the sums of 1,024
//    evenly spread code blocks go into a histogram of s' (s' = S for L2,
//    255*M - S for dot).  The upper edge T of the bin holding the sample's
//    k-th smallest s' bounds the k-th smallest s' of the whole database (the
//    sample is part of it), so no vector with s' > T can be in the top k.
// 2. Filter (mq_filter_kernel).  One pass over the codes; each warp scans a
//    256-vector block for a tile of up to 16 queries at once (every code word
//    loaded and prepared once) and appends the keys (s' << 32 | index) with
//    s' <= T of each query to that query's candidate list.
// 3. Select (mq_select_kernel).  One CTA per query: a histogram of the
//    candidates gives the exact k-th smallest s' (T*) and the count below
//    it; every candidate below T* is kept, and of those equal to T* the
//    lowest indices (sorted), so ties go to the lower index.
// 4. Fallback.  A query whose candidate list overflowed, or whose ties at T*
//    are too many to sort, is marked; the streaming kernel (topk.cu) then
//    runs for the marked queries only (its CTAs for other queries return at
//    once), so the result is exact whatever the data.
#include "topk.cuh"

#include "scan_core.cuh"

namespace bolt {

constexpr int kMqThreads = 256;
constexpr int kMqWarps = kMqThreads / 32;
constexpr int kMqSampleBlocks = 1024;  // sample size in 256-vector blocks
constexpr int kMqChunk = 16;           // sample blocks per CTA
constexpr int kMqSelThreads = 512;
constexpr int kMqTieCap = 8192;  // keys equal to T* the select kernel can order
constexpr int kMqMaxQt = 16;
constexpr int kMqLutRows = 1024;  // table rows (16 bytes) a filter CTA stages
constexpr int kMqStages = 4;      // bulk-copy stages per filter warp
constexpr uint64_t kMqWait = 1000000000ull;  // 1 s bound on every mbarrier wait

struct MqWS {
    uint32_t *sh;      // [nq][kBins] sample histogram
    uint32_t *ticket;  // [nq]
    uint32_t *thr;     // [nq] inclusive bound on s'
    uint32_t *cnt;     // [nq] candidates found (may exceed cap)
    uint32_t *active;  // [nq] 1: the query falls back to the streaming kernel
    uint32_t *ch;      // [nq][kBins] histogram of the candidates' s' (filled by the filter)
    uint64_t *cand;    // [nq][cap]
};


// Smallest bin b with (#entries in bins < b) < kk <= (#in bins <= b), for a
// block of T threads; returns b and sets below.  kk <= total required.
template <int T>
__device__ __forceinline__ uint32_t mq_find(const uint32_t *hist, uint32_t kk, uint32_t *scratch, uint32_t &below) {
    constexpr int BPT = kBins / T;
    constexpr int W = T / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t v[BPT], local = 0;
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        v[i] = hist[tid * BPT + i];
        local += v[i];
    }
    uint32_t incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) scratch[2 + warp] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += scratch[2 + w];
    const uint32_t excl = before + incl - local;
    if (excl < kk && kk <= excl + local) {
        uint32_t c = excl;
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            if (c < kk && kk <= c + v[i]) {
                scratch[0] = (uint32_t)(tid * BPT + i);
                scratch[1] = c;
            }
            c += v[i];
        }
    }
    __syncthreads();
    below = scratch[1];
    const uint32_t b = scratch[0];
    __syncthreads();
    (void)W;
    return b;
}

// ------------------------------------------------------------------ 1. sample bound
template <int MT>
__global__ void __launch_bounds__(kMqThreads) mq_sample_kernel(const uint32_t *__restrict__ codes, int64_t n,
                                                               int32_t M, const uint8_t *__restrict__ luts,
                                                               int32_t k, int32_t metric, MqWS ws, int ns,
                                                               int hshift) {
    __shared__ uint32_t hist[kBins];
    __shared__ uint4 lut[256];
    __shared__ uint32_t scratch[2 + kMqWarps];
    __shared__ uint32_t last;
    if (MT > 0) M = MT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q = blockIdx.y;
    const int64_t nb = num_blocks(n);
    for (int i = tid; i < kBins; i += kMqThreads) hist[i] = 0;
    const uint4 *lut_g = reinterpret_cast<const uint4 *>(luts + q * M * kK);
    for (int i = tid; i < M; i += kMqThreads) lut[i] = __ldg(lut_g + i);
    __syncthreads();
    const uint32_t smax = 255u * (uint32_t)M;
    for (int jj = warp; jj < kMqChunk; jj += kMqWarps) {
        const int j = blockIdx.x * kMqChunk + jj;
        if (j >= ns) break;
        const int64_t b = (int64_t)j * nb / ns;  // distinct blocks (ns <= nb), evenly spread
        const uint32_t *row = codes + b * M * kRowWords + lane;
        Acc8 acc;
        acc.zero();
        if (MT > 0) {
#pragma unroll
            for (int m = 0; m < MT; ++m) acc.add(prep_word(__ldg(row + m * kRowWords)), lut[m]);
        } else {
#pragma unroll 4
            for (int m = 0; m < M; ++m) acc.add(prep_word(__ldg(row + (int64_t)m * kRowWords)), lut[m]);
        }
        uint32_t e_lo, o_lo, e_hi, o_hi;
        acc.finish(e_lo, o_lo, e_hi, o_hi);
        const uint4 pk = pack_sums(e_lo, o_lo, e_hi, o_hi);
        const uint32_t w[4] = {pk.x, pk.y, pk.z, pk.w};
        const int64_t v0 = b * kBlockVecs + 8 * lane;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (v0 + i < n) {
                const uint32_t S = (w[i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
                const uint32_t sp = metric == BOLT_METRIC_DOT ? smax - S : S;
                atomicAdd(&hist[sp >> hshift], 1u);
            }
        }
    }
    __syncthreads();
    uint32_t *gh = ws.sh + q * kBins;
    for (int i = tid; i < kBins; i += kMqThreads)
        if (hist[i]) atomicAdd(&gh[i], hist[i]);
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(&ws.ticket[q], 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    uint32_t total = 0;
    for (int i = tid; i < kBins; i += kMqThreads) {
        hist[i] = __ldcg(gh + i);
        total += hist[i];
    }
    total = __reduce_add_sync(0xFFFFFFFFu, total);
    if (lane == 0) scratch[2 + warp] = total;
    __syncthreads();
    total = 0;
    for (int w = 0; w < kMqWarps; ++w) total += scratch[2 + w];
    __syncthreads();
    if (total < (uint32_t)k) {
        if (tid == 0) ws.thr[q] = 0xFFFFu;  // sample smaller than k: every vector is a candidate
        return;
    }
    uint32_t below;
    const uint32_t B = mq_find<kMqThreads>(hist, (uint32_t)k, scratch, below);
    if (tid == 0) ws.thr[q] = ((B + 1u) << hshift) - 1u;
}

// ------------------------------------------------------------------ 2. filter
static int mq_max_qt(int32_t M) {
    int qt = kMqMaxQt;
    while (qt > 1 && qt * M > kMqLutRows) qt >>= 1;
    return qt;
}


// Append the lane's keys (s' << 32 | index) with s' < lim to query q's
// list.  Kept out of line: it runs for few blocks, and inlining one copy per
// query of a tile crowds the instruction cache of the lookup loop.  Called by
// all 32 lanes together.
__device__ __noinline__ void mq_append(uint4 pk, uint32_t lim, int64_t q, int64_t v0, int64_t n, const MqWS &ws,
                                       int64_t cap, int hshift, int lane) {
    const uint32_t w[4] = {pk.x, pk.y, pk.z, pk.w};
    uint32_t cm = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t sp = (w[i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
        if (v0 + i < n && sp < lim) cm |= 1u << i;
    }
    const uint32_t c = __popc(cm);
    uint32_t incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += x;
    }
    uint32_t base = 0;
    if (lane == 31 && incl) base = atomicAdd(&ws.cnt[q], incl);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    uint32_t pos = base + incl - c;
    uint64_t *list = ws.cand + q * cap;
    uint32_t *ch = ws.ch + q * kBins;
    for (int i = 0; i < 8; ++i) {
        if (cm & (1u << i)) {
            const uint32_t sp = (w[i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
            if ((int64_t)pos < cap) list[pos] = ((uint64_t)sp << 32) | (uint64_t)(v0 + i);
            atomicAdd(&ch[sp >> hshift], 1u);
            ++pos;
        }
    }
}

// Candidates of one scanned block for QT queries: keys (s' << 32 | index)
// with s' <= thr[t] are appended to query q0 + t's list.
template <int QT>
__device__ __forceinline__ void mq_emit(Acc8 (&acc)[QT], int64_t b, int M, int64_t n, const uint32_t *thr,
                                        int64_t q0, int32_t metric, const MqWS &ws, int64_t cap, int hshift,
                                        int lane) {
    const uint32_t smax = 255u * (uint32_t)M;
    const uint32_t smax2 = smax | (smax << 16);
    const int64_t v0 = b * kBlockVecs + 8 * lane;
    const bool swar = smax <= 0x7FFFu;
#pragma unroll
    for (int t = 0; t < QT; ++t) {
        uint32_t e_lo, o_lo, e_hi, o_hi;
        acc[t].finish(e_lo, o_lo, e_hi, o_hi);
        if (metric == BOLT_METRIC_DOT) {
            e_lo = smax2 - e_lo;
            o_lo = smax2 - o_lo;
            e_hi = smax2 - e_hi;
            o_hi = smax2 - o_hi;
        }
        const uint32_t lim = thr[t] + 1u;  // candidate iff s' < lim
        bool maybe = v0 < n;
        if (swar && lim <= 0x7FFFu) {
            // top bit of (s' + 2^15 - lim) per 16-bit lane is clear iff s' < lim
            const uint32_t nt2 = 0u - (lim | (lim << 16));
            const uint32_t d = ((e_lo | 0x80008000u) + nt2) & ((o_lo | 0x80008000u) + nt2) &
                               ((e_hi | 0x80008000u) + nt2) & ((o_hi | 0x80008000u) + nt2);
            maybe = maybe && (~d & 0x80008000u) != 0u;
        }
        if (!__any_sync(0xFFFFFFFFu, maybe)) continue;
        mq_append(pack_sums(e_lo, o_lo, e_hi, o_hi), lim, q0 + t, v0, n, ws, cap, hshift, lane);
    }
}

// Filter CTA: 8 warps; warp w scans blocks b0 + w, b0 + w + 8, ... < b1 for
// the tile's QT queries.  Each warp streams its blocks through a private ring
// of kMqStages shared-memory stages filled by 1-D bulk copies (lane 0 keeps
// kMqStages blocks in flight), so the lookups never wait on a single load.
template <int MT, int QT>
__global__ void __launch_bounds__(kMqThreads, (QT <= 2 ? 3 : 2))
    mq_filter_kernel(const uint32_t *__restrict__ codes, int64_t n, int32_t M, const uint8_t *__restrict__ luts,
                     int32_t metric, MqWS ws, int64_t cap, int64_t blocks_per_cta, int64_t q_base, int hshift) {
    extern __shared__ __align__(128) uint8_t fsm[];
    if (MT > 0) M = MT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q0 = q_base + (int64_t)blockIdx.y * QT;
    const int64_t nb = num_blocks(n);
    const int64_t b0 = (int64_t)blockIdx.x * blocks_per_cta;
    const int64_t b1 = min(nb, b0 + blocks_per_cta);
    if (b0 >= b1) return;
    const uint32_t blk_bytes = (uint32_t)M * kRowBytes;
    uint8_t *p = fsm;
    uint64_t *bars = reinterpret_cast<uint64_t *>(p);  // [kMqWarps][kMqStages]
    p += kMqWarps * kMqStages * 8;
    uint32_t *thr = reinterpret_cast<uint32_t *>(p);  // [QT]
    p += 64;
    uint4 *lut = reinterpret_cast<uint4 *>(p);  // [QT][M]
    p += (size_t)QT * M * 16;
    uint8_t *ring = p + (size_t)warp * kMqStages * blk_bytes;
    if (tid < kMqWarps * kMqStages) mbar_init(&bars[tid], 1);
    fence_mbar_init();
    const uint4 *src = reinterpret_cast<const uint4 *>(luts) + q0 * M;
    for (int i = tid; i < QT * M; i += kMqThreads) lut[i] = __ldg(src + i);
    if (tid < QT) thr[tid] = __ldcg(ws.thr + q0 + tid);
    __syncthreads();
    uint64_t *mybars = bars + warp * kMqStages;
    const int64_t first = b0 + warp;
    const int64_t nmine = first < b1 ? (b1 - first + kMqWarps - 1) / kMqWarps : 0;
    if (lane == 0)
        for (int st = 0; st < kMqStages && st < nmine; ++st) {
            const int64_t b = first + (int64_t)st * kMqWarps;
            mbar_arrive_expect_tx(&mybars[st], blk_bytes);
            bulk_g2s(ring + (size_t)st * blk_bytes, codes + b * M * kRowWords, blk_bytes, &mybars[st]);
        }
    bool failed = false;
    int64_t i = 0;
    for (; i < nmine; ++i) {
        const int st = (int)(i % kMqStages);
        const uint32_t par = (uint32_t)((i / kMqStages) & 1);
        const bool ok = mbar_wait_bounded(&mybars[st], par, kMqWait);
        if (!__all_sync(0xFFFFFFFFu, ok)) {
            failed = true;
            break;
        }
        const uint32_t *words = reinterpret_cast<const uint32_t *>(ring + (size_t)st * blk_bytes);
        Acc8 acc[QT];
#pragma unroll
        for (int t = 0; t < QT; ++t) acc[t].zero();
        if (MT > 0) {
            // keep the loop body near 64 word-query steps: fully unrolled
            // 16 x 16 steps overflow the instruction cache
            constexpr int kU = QT >= 8 ? 4 : (QT >= 4 ? 8 : 16);
#pragma unroll kU
            for (int m = 0; m < MT; ++m) {
                const WordSel w = prep_word(words[m * kRowWords + lane]);
#pragma unroll
                for (int t = 0; t < QT; ++t) acc[t].add(w, lut[t * MT + m]);
            }
        } else {
#pragma unroll 4
            for (int m = 0; m < M; ++m) {
                const WordSel w = prep_word(words[m * kRowWords + lane]);
#pragma unroll
                for (int t = 0; t < QT; ++t) acc[t].add(w, lut[t * M + m]);
            }
        }
        __syncwarp();
        if (lane == 0 && i + kMqStages < nmine) {  // refill this stage
            const int64_t b = first + (i + kMqStages) * kMqWarps;
            mbar_arrive_expect_tx(&mybars[st], blk_bytes);
            bulk_g2s(ring + (size_t)st * blk_bytes, codes + b * M * kRowWords, blk_bytes, &mybars[st]);
        }
        mq_emit<QT>(acc, first + i * kMqWarps, M, n, thr, q0, metric, ws, cap, hshift, lane);
    }
    if (failed) {
        // a wait gave up: these queries take the exact fallback; let copies in
        // flight land (bounded) before the shared memory goes away
        if (lane == 0) {
            for (int t = 0; t < QT; ++t) atomicExch(&ws.active[q0 + t], 1u);
            for (int64_t j = i; j < nmine && j < i + kMqStages; ++j)
                mbar_wait_bounded(&mybars[j % kMqStages], (uint32_t)((j / kMqStages) & 1), kMqWait / 10);
        }
        __syncwarp();
    }
}

size_t mq_filter_smem(int32_t M, int qt) {
    return (size_t)kMqWarps * kMqStages * 8 + 64 + (size_t)qt * M * 16 + (size_t)kMqWarps * kMqStages * M * kRowBytes;
}

// ------------------------------------------------------------------ 3. select
// Visit list[0..total) in batches of 8 keys per thread (all 8 loads in
// flight before any is used): f(key).
template <typename F>
__device__ __forceinline__ void mq_each(const uint64_t *list, uint32_t total, F f) {
    constexpr int U = 8;
    for (uint32_t base = 0; base < total; base += U * kMqSelThreads) {
        uint64_t v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t e = base + u * kMqSelThreads + threadIdx.x;
            v[u] = e < total ? __ldcg(list + e) : ~0ull;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (v[u] != ~0ull) f(v[u]);
    }
}

__global__ void __launch_bounds__(kMqSelThreads) mq_select_kernel(int64_t n, int32_t M, int32_t k, int32_t metric,
                                                                 MqWS ws, int64_t cap, int hshift,
                                                                 uint16_t *__restrict__ out_sums,
                                                                 int64_t *__restrict__ out_idx) {
    extern __shared__ __align__(16) uint8_t smem_sel[];
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem_sel);             // [kBins]
    uint64_t *fin = reinterpret_cast<uint64_t *>(smem_sel + kBins * 4);  // [2 * 1024]
    uint64_t *eqb = fin + 2 * 1024;                                      // [kMqTieCap]
    __shared__ uint32_t scratch[2 + kMqSelThreads / 32];
    __shared__ uint32_t nlt_s, neq_s;
    const int tid = threadIdx.x;
    const int64_t q = blockIdx.x;
    const uint32_t total = __ldcg(ws.cnt + q);
    if ((int64_t)total > cap) {  // list overflowed: exact fallback
        if (tid == 0) ws.active[q] = 1u;
        return;
    }
    const uint64_t *list = ws.cand + q * cap;
    const uint32_t smax = 255u * (uint32_t)M;
    {
        // the filter counted every candidate in this histogram
        constexpr int BPT = kBins / kMqSelThreads;
        uint32_t hv[BPT];
#pragma unroll
        for (int i = 0; i < BPT; ++i) hv[i] = __ldcg(ws.ch + q * kBins + tid + i * kMqSelThreads);
#pragma unroll
        for (int i = 0; i < BPT; ++i) hist[tid + i * kMqSelThreads] = hv[i];
    }
    if (tid == 0) nlt_s = neq_s = 0;
    __syncthreads();
    const uint32_t kk = min((uint32_t)k, total);
    uint32_t Tstar = 0, c_lt = 0, c_eq = 0;
    if (kk > 0) {
        uint32_t below;
        const uint32_t B = mq_find<kMqSelThreads>(hist, kk, scratch, below);
        Tstar = B;
        c_lt = below;
        c_eq = hist[B];
        __syncthreads();
        if (hshift > 0) {
            const uint32_t mask = (1u << hshift) - 1u;
            for (int i = tid; i < kBins; i += kMqSelThreads) hist[i] = 0;
            __syncthreads();
            mq_each(list, total, [&](uint64_t key) {
                const uint32_t v = (uint32_t)(key >> 32);
                if ((v >> hshift) == B) atomicAdd(&hist[v & mask], 1u);
            });
            __syncthreads();
            uint32_t below2;
            const uint32_t f = mq_find<kMqSelThreads>(hist, kk - below, scratch, below2);
            Tstar = (B << hshift) | f;
            c_lt = below + below2;
            c_eq = hist[f];
            __syncthreads();
        }
    }
    const uint32_t r = kk - c_lt;  // keys equal to T* to keep, lowest index first
    if (r < c_eq && c_eq > (uint32_t)kMqTieCap) {  // too many ties to order here: exact fallback
        if (tid == 0) ws.active[q] = 1u;
        return;
    }
    // gather: keys below T* (order irrelevant, sorted below) and keys equal to T*
    mq_each(list, total, [&](uint64_t key) {
        const uint32_t v = (uint32_t)(key >> 32);
        if (v < Tstar) fin[atomicAdd(&nlt_s, 1u)] = key;
        else if (v == Tstar && r > 0) {
            const uint32_t p = atomicAdd(&neq_s, 1u);
            if (r == c_eq) fin[c_lt + p] = key;  // all of them are kept
            else eqb[p] = key;
        }
    });
    __syncthreads();
    if (r > 0 && r < c_eq) {
        // the r lowest indices among the ties: bitonic sort of eqb[0..P)
        int P = 1;
        while (P < (int)c_eq) P <<= 1;
        for (int i = (int)c_eq + tid; i < P; i += kMqSelThreads) eqb[i] = ~0ull;
        __syncthreads();
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < P / 2; i += kMqSelThreads) {
                    const int lo = 2 * i - (i & (stride - 1));
                    const int hi = lo + stride;
                    const bool asc = (lo & size) == 0;
                    const uint64_t a = eqb[lo], bq = eqb[hi];
                    if ((a > bq) == asc) {
                        eqb[lo] = bq;
                        eqb[hi] = a;
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t i = tid; i < r; i += kMqSelThreads) fin[c_lt + i] = eqb[i];
        __syncthreads();
    }
    // order the kk survivors by (s', index)
    const int kout = (int)kk;
    uint64_t *res = fin;
    if (kout <= 256) {
        uint64_t *sorted = fin + 1024;
        for (int e = tid; e < kout; e += kMqSelThreads) {
            const uint64_t key = fin[e];
            int rank = 0;
            for (int j = 0; j < kout; ++j) rank += fin[j] < key ? 1 : 0;
            sorted[rank] = key;
        }
        __syncthreads();
        res = sorted;
    } else {
        int P = 1;
        while (P < kout) P <<= 1;
        for (int i = kout + tid; i < P; i += kMqSelThreads) fin[i] = ~0ull;
        __syncthreads();
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < P / 2; i += kMqSelThreads) {
                    const int lo = 2 * i - (i & (stride - 1));
                    const int hi = lo + stride;
                    const bool asc = (lo & size) == 0;
                    const uint64_t a = fin[lo], bq = fin[hi];
                    if ((a > bq) == asc) {
                        fin[lo] = bq;
                        fin[hi] = a;
                    }
                }
                __syncthreads();
            }
        }
    }
    for (int i = tid; i < k; i += kMqSelThreads) {
        if (i < kout) {
            const uint32_t sp = (uint32_t)(res[i] >> 32);
            out_sums[q * k + i] = (uint16_t)(metric == BOLT_METRIC_DOT ? smax - sp : sp);
            out_idx[q * k + i] = (int64_t)(uint32_t)res[i];
        } else {
            out_sums[q * k + i] = 0;
            out_idx[q * k + i] = -1;
        }
    }
    (void)n;
}

// ------------------------------------------------------------------ host side
static size_t mq_align(size_t x, size_t a) { return (x + a - 1) / a * a; }

void plan_topk_mq(int64_t n, int32_t M, int32_t k, int sms, TopkPlan *plan) {
    const int64_t nb = num_blocks(n);
    const int64_t ns = nb < kMqSampleBlocks ? nb : kMqSampleBlocks;
    // expected candidates: about k * n / (sample vectors); room for 4x that
    int64_t cap = (int64_t)k * (nb / (ns > 0 ? ns : 1) + 1) * 4;
    if (cap < 16384) cap = 16384;
    if (cap > n) cap = n;
    if (cap < k) cap = k;
    plan->mq = 1;
    plan->mq_ns = (int)ns;
    plan->mq_cap = cap;
    int hshift = 0;
    while (((255 * M) >> hshift) >= kBins) ++hshift;
    plan->mq_hshift = hshift;
    (void)sms;
}

static size_t mq_header_bytes(int64_t nq) {
    // sample and candidate histograms + 4 counters per query
    return (size_t)2 * nq * kBins * 4 + mq_align((size_t)nq * 16, 256);
}

int64_t topk_mq_workspace_bytes(const TopkPlan &plan, int64_t nq, int32_t k) {
    return (int64_t)(mq_header_bytes(nq) + mq_align((size_t)nq * plan.mq_cap * 8, 256)) +
           topk_stream_workspace_bytes(plan, nq, k);
}

template <int MT>
static void launch_sample_w(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                            int32_t metric, const MqWS &w, const TopkPlan &plan, cudaStream_t s) {
    dim3 grid((unsigned)((plan.mq_ns + kMqChunk - 1) / kMqChunk), (unsigned)nq);
    mq_sample_kernel<MT><<<grid, kMqThreads, 0, s>>>(reinterpret_cast<const uint32_t *>(codes), n, M, luts, k,
                                                     metric, w, plan.mq_ns, plan.mq_hshift);
}

template <int MT, int QT>
static int launch_filter_w(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int32_t metric,
                           const MqWS &w, int64_t cap, int64_t bpc, int64_t gx, int64_t gy, int64_t q_base,
                           int hshift, cudaStream_t s) {
    auto kern = mq_filter_kernel<MT, QT>;
    const size_t smem = mq_filter_smem(M, QT);
    int rc = ensure_smem((const void *)kern, smem);
    if (rc) return rc;
    kern<<<dim3((unsigned)gx, (unsigned)gy), kMqThreads, smem, s>>>(reinterpret_cast<const uint32_t *>(codes), n, M,
                                                                     luts, metric, w, cap, bpc, q_base, hshift);
    return check_launch("mq_filter_kernel");
}

template <int MT>
static int launch_filter_m(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int32_t metric,
                           const MqWS &w, int64_t cap, int64_t bpc, int64_t gx, int64_t gy, int qt, int64_t q_base,
                           int hshift, cudaStream_t s) {
    switch (qt) {
        case 16: return launch_filter_w<MT, 16>(codes, n, M, luts, metric, w, cap, bpc, gx, gy, q_base, hshift, s);
        case 8: return launch_filter_w<MT, 8>(codes, n, M, luts, metric, w, cap, bpc, gx, gy, q_base, hshift, s);
        case 4: return launch_filter_w<MT, 4>(codes, n, M, luts, metric, w, cap, bpc, gx, gy, q_base, hshift, s);
        case 2: return launch_filter_w<MT, 2>(codes, n, M, luts, metric, w, cap, bpc, gx, gy, q_base, hshift, s);
        default: return launch_filter_w<MT, 1>(codes, n, M, luts, metric, w, cap, bpc, gx, gy, q_base, hshift, s);
    }
}

static int launch_filter(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int32_t metric,
                         const MqWS &w, int64_t cap, int64_t bpc, int64_t gx, int64_t gy, int qt, int64_t q_base,
                         int hshift, cudaStream_t s) {
    if (M == 8) return launch_filter_m<8>(codes, n, M, luts, metric, w, cap, bpc, gx, gy, qt, q_base, hshift, s);
    if (M == 16) return launch_filter_m<16>(codes, n, M, luts, metric, w, cap, bpc, gx, gy, qt, q_base, hshift, s);
    if (M == 32) return launch_filter_m<32>(codes, n, M, luts, metric, w, cap, bpc, gx, gy, qt, q_base, hshift, s);
    return launch_filter_m<0>(codes, n, M, luts, metric, w, cap, bpc, gx, gy, qt, q_base, hshift, s);
}

int launch_topk_mq(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                   int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, const TopkPlan &plan,
                   cudaStream_t stream) {
    BOLT_REQUIRE(nq <= 65535, BOLT_EUNSUPPORTED, "nq=%lld > 65535 per call", (long long)nq);
    uint8_t *p = static_cast<uint8_t *>(workspace);
    MqWS w;
    w.sh = reinterpret_cast<uint32_t *>(p);
    w.ch = reinterpret_cast<uint32_t *>(p + (size_t)nq * kBins * 4);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(p + (size_t)2 * nq * kBins * 4);
    w.ticket = ctr;
    w.thr = ctr + nq;
    w.cnt = ctr + 2 * nq;
    w.active = ctr + 3 * nq;
    p += mq_header_bytes(nq);
    w.cand = reinterpret_cast<uint64_t *>(p);
    p += mq_align((size_t)nq * plan.mq_cap * 8, 256);
    void *stream_ws = p;
    BOLT_CUDA(cudaMemsetAsync(workspace, 0, mq_header_bytes(nq), stream));
    // 1. sample bound
    if (M == 8) launch_sample_w<8>(codes, n, M, luts, nq, k, metric, w, plan, stream);
    else if (M == 16) launch_sample_w<16>(codes, n, M, luts, nq, k, metric, w, plan, stream);
    else if (M == 32) launch_sample_w<32>(codes, n, M, luts, nq, k, metric, w, plan, stream);
    else launch_sample_w<0>(codes, n, M, luts, nq, k, metric, w, plan, stream);
    int rc = check_launch("mq_sample_kernel");
    if (rc) return rc;
    // 2. filter: query tiles of maxqt, then the remainder in powers of two;
    // one launch per tile size, about one wave of CTAs in total
    const int64_t nb = num_blocks(n);
    const int maxqt = mq_max_qt(M);
    const int64_t full = nq / maxqt;
    const int rem = (int)(nq - full * maxqt);
    const int64_t tiles = full + __builtin_popcount((unsigned)rem);
    const int sms = device_sm_count() > 0 ? device_sm_count() : 1;
    const int occ = maxqt <= 2 || nq <= 2 ? 3 : 2;  // resident filter CTAs per SM
    int64_t gx = ((int64_t)occ * sms + tiles - 1) / tiles;
    if (gx > nb) gx = nb;
    if (gx < 1) gx = 1;
    const int64_t bpc = (nb + gx - 1) / gx;
    gx = (nb + bpc - 1) / bpc;
    rc = BOLT_OK;
    int64_t qb = 0;
    if (full > 0) {
        rc = launch_filter(codes, n, M, luts, metric, w, plan.mq_cap, bpc, gx, full, maxqt, 0, plan.mq_hshift, stream);
        qb = full * maxqt;
    }
    for (int bit = maxqt >> 1; bit >= 1 && rc == BOLT_OK; bit >>= 1)
        if (rem & bit) {
            rc = launch_filter(codes, n, M, luts, metric, w, plan.mq_cap, bpc, gx, 1, bit, qb, plan.mq_hshift, stream);
            qb += bit;
        }
    if (rc) return rc;
    // 3. select
    const size_t sel_smem = (size_t)kBins * 4 + (size_t)2 * 1024 * 8 + (size_t)kMqTieCap * 8;
    rc = ensure_smem((const void *)mq_select_kernel, sel_smem);
    if (rc) return rc;
    mq_select_kernel<<<(unsigned)nq, kMqSelThreads, sel_smem, stream>>>(n, M, k, metric, w, plan.mq_cap,
                                                                        plan.mq_hshift, out_sums, out_idx);
    rc = check_launch("mq_select_kernel");
    if (rc) return rc;
    // 4. exact fallback for the marked queries (no work for the others)
    return launch_topk_stream(codes, n, M, luts, nq, k, metric, out_sums, out_idx, stream_ws, plan, w.active,
                              stream);
}

}  // namespace bolt
