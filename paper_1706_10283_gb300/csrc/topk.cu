// Fused Bolt scan + exact top-k (nearest neighbours for L2 sums, maximum
// inner product for dot sums; Sec. 1.2 motivates both searches).
//
// Keys.  A candidate is the 64-bit key (s' << 32 | index) with s' = S for L2
// and s' = 255*M - S for dot, so "smaller key" is "better" for both metrics
// and equal sums break ties toward the lower index.  Bit 63 marks a candidate
// already counted in the global histogram (masked out of every comparison).
//
// Work split.  Each query is handled by `grid` CTAs, one contiguous range of
// 256-vector code blocks per CTA.  A CTA processes its blocks in rounds: in
// round r warp w takes block lo + r*WARPS + w, so every block of round r+1
// has larger indices than every block of rounds <= r.  Each warp streams its
// blocks through a private ring of shared-memory stages filled by 1-D TMA
// bulk copies (non-multicast) completing on an mbarrier.
//
// Threshold.  Every warp counts its first unit's sums in shared two-level
// histograms (fine bins of width 2^hshift, coarse bins of 16 fine bins);
// after a barrier among those warps the CTA's k-th smallest first-round sum
// gives its first threshold, and the counts up to that bin (at least k
// distinct vectors) are added to per-query global fine and coarse
// histograms, one add per non-empty bin.
//
// Candidates.  Lanes append sums below the CTA's threshold to a shared
// buffer.  When it runs full the CTA histograms the buffer by s' bin (4096
// bins of width 2^hshift), keeps every entry up to the bin of its k-th
// smallest and lowers its threshold to just past that bin.  Warps are not in
// lockstep, so a warp that lags can still bring a key with a lower index
// than kept ones: thresholds stay inclusive of the k-th bin, and when the
// CTA selects its exact k-th key instead, a tie rule rejects only keys equal
// to it in s' with a higher index.
//
// Global bound.  Each vector is counted in the global histograms at most
// once (first-round keys at seeding, later keys when a compaction or the
// final publication adds the CTA's uncounted entries), so the bin where their
// running count reaches k bounds the k-th smallest sum of the whole query.
// Every 4 rounds one warp in turn reads the coarse then the fine counts and
// lowers the CTA's threshold to that bin, without stopping the other warps.
//
// Merge.  Each CTA writes its candidates up to the current global bound (at
// most 2k, else its exact top k) to its own slot of a per-query list (the
// count, then the keys); the last CTA to finish (atomic ticket) reads the
// slot counts while one warp finds the final bound bin of the global
// histogram, gathers the keys into shared memory (when there are more than
// 1024, only those at or below that bin), selects the exact k smallest keys,
// sorts them and writes the result.
//
// Tables.  For dot the CTA complements its tables (255 - D is the byte
// complement), so the lookups produce s' directly.
#include <mutex>

#include "scan_core.cuh"
#include "topk.cuh"

namespace bolt {

// 1 s: the bound on the warps' wait for one another and, divided by 10, on
// draining copies in flight after a failure (waits for the CTA's own code
// copies use data_wait_limit_ns(), 1 s by default)
constexpr uint64_t kWaitLimit = 1000000000ull;
// phase stamps (diagnostic builds): 0 start, 1 first threshold, 2 loop end,
// 3 published, 4 end (last CTA), 5 keys published, 6 merge total, 7 merge
// survivors, 8 last CTA's counts and bound, 9 gathered
BOLT_STAMP_ARRAY(g_stamps_topk);
constexpr int kMaxStages = 8;
constexpr size_t kStageBudget = 128 * 1024;
constexpr int kMaxK = 1024;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr int kSeedBins = kBins / 16;  // coarse bins (16 fine bins each) of the two-level histograms

// Barrier 1 among the first `warps` warps of the CTA (the warps that have a
// first unit); barrier 0 is __syncthreads.
__device__ __forceinline__ void seed_barrier(uint32_t warps) {
    asm volatile("bar.sync 1, %0;" ::"r"(warps * 32u) : "memory");
}
__device__ __forceinline__ uint32_t vmisc_hist(const uint32_t *h, int i) {
    return *reinterpret_cast<const volatile uint32_t *>(h + i);
}

// k-th bin search by one warp over a two-level histogram: coarse[256] and
// fine[4096], fine bin f inside coarse bin f >> 4.  The coarse bin where the
// running count reaches k, then the fine bin inside it; fbin is that fine
// bin and in_bin the fine counts of cbin up to it.  kGlobal: counts in
// global memory, read through L2 (they grow while being read: a fine count
// may trail its coarse count, and without a fine hit the whole coarse bin is
// returned).  False when the total is below k.
template <bool kGlobal>
__device__ __forceinline__ bool warp_kth_bin(const uint32_t *coarse, const uint32_t *fine, uint32_t k, int lane,
                                             uint32_t &cbin, uint32_t &fbin, uint32_t &in_bin, uint32_t (&c)[8]) {
    if (kGlobal) {
        const uint4 *g4 = reinterpret_cast<const uint4 *>(coarse + lane * 8);
        const uint4 a = __ldcg(g4), b = __ldcg(g4 + 1);
        c[0] = a.x, c[1] = a.y, c[2] = a.z, c[3] = a.w, c[4] = b.x, c[5] = b.y, c[6] = b.z, c[7] = b.w;
    } else {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(coarse + lane * 8);
        const uint4 a = s4[0], b = s4[1];
        c[0] = a.x, c[1] = a.y, c[2] = a.z, c[3] = a.w, c[4] = b.x, c[5] = b.y, c[6] = b.z, c[7] = b.w;
    }
    uint32_t tot = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) tot += c[i];
    uint32_t incl = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += t;
    }
    const uint32_t crossing = __ballot_sync(0xFFFFFFFFu, incl >= k && incl - tot < k);
    if (!crossing) return false;
    const int src = __ffs(crossing) - 1;
    uint32_t cb = 0, before = 0;
    if (lane == src) {
        uint32_t run = incl - tot;
        bool hit = false;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (!hit && run + c[i] >= k) {
                cb = (uint32_t)(lane * 8 + i);
                before = run;
                hit = true;
            }
            run += c[i];
        }
    }
    cb = __shfl_sync(0xFFFFFFFFu, cb, src);
    before = __shfl_sync(0xFFFFFFFFu, before, src);
    uint32_t fi = 0;
    if (lane < 16) fi = kGlobal ? __ldcg(fine + cb * 16 + lane) : reinterpret_cast<const volatile uint32_t *>(fine)[cb * 16 + lane];
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, fi, off);
        if (lane >= off) fi += t;
    }
    const uint32_t hitm = __ballot_sync(0xFFFFFFFFu, lane < 16 && before + fi >= k);
    const int fl = hitm ? __ffs(hitm) - 1 : 15;
    cbin = cb;
    fbin = cb * 16u + (uint32_t)fl;
    in_bin = __shfl_sync(0xFFFFFFFFu, fi, fl);
    return true;
}

constexpr uint64_t kFlag = 1ull << 63;  // "already counted in the global histogram"

__device__ __forceinline__ uint64_t kv(uint64_t key) { return key & ~kFlag; }

// ------------------------------------------------------------------ block-wide selection
// Exact radix selection over keys (byte digits, warp-aggregated counts).
template <int T>
struct BlockSel {
    uint32_t *hist;  // 256 counters
    uint32_t *res;   // [0] digit, [1] count below digit

    // Histogram of the byte at `shift` over keys whose bits above the byte
    // match `prefix` (bits above shift+8), warp-aggregated.
    __device__ void histogram(const uint64_t *keys, int cnt, uint64_t prefix, int shift) {
        const int tid = threadIdx.x;
        for (int i = tid; i < 256; i += T) hist[i] = 0;
        __syncthreads();
        const uint64_t hmask = (shift + 8 >= 64) ? 0ull : (~0ull << (shift + 8));
        for (int base = 0; base < cnt; base += T) {
            const int i = base + tid;
            uint32_t bin = 0xFFFFFFFFu;
            if (i < cnt) {
                const uint64_t key = kv(keys[i]);
                if ((key & hmask) == (prefix & hmask)) bin = (uint32_t)(key >> shift) & 255u;
            }
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, bin);
            if (bin != 0xFFFFFFFFu && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
        }
        __syncthreads();
    }

    // Smallest digit d with (#below d) < kk <= (#below d) + hist[d]; writes
    // res[0] = d, res[1] = #below d.  Requires 1 <= kk <= total.
    __device__ void find(uint32_t kk) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            uint32_t v[8], local = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                v[i] = hist[lane * 8 + i];
                local += v[i];
            }
            uint32_t incl = local;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
                if (lane >= off) incl += t;
            }
            const uint32_t excl = incl - local;
            if (excl < kk && kk <= incl) {
                uint32_t c = excl;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (c + v[i] >= kk) {
                        res[0] = lane * 8 + i;
                        res[1] = c;
                        break;
                    }
                    c += v[i];
                }
            }
        }
        __syncthreads();
    }

    // k-th smallest s' = key >> 32 (with multiplicity).  Returns s*, and the
    // number of keys with s' < s* and s' == s*.
    __device__ uint32_t kth_sum(const uint64_t *keys, int cnt, uint32_t kk, uint32_t &n_less, uint32_t &n_eq) {
        histogram(keys, cnt, 0ull, 40);
        find(kk);
        const uint32_t d1 = res[0], b1 = res[1];
        __syncthreads();
        histogram(keys, cnt, (uint64_t)d1 << 40, 32);
        find(kk - b1);
        const uint32_t d2 = res[0], b2 = res[1];
        n_eq = hist[d2];
        __syncthreads();
        n_less = b1 + b2;
        return (d1 << 8) | d2;
    }

    // Exact k-th smallest key.
    __device__ uint64_t kth_key(const uint64_t *keys, int cnt, uint32_t kk) {
        uint32_t n_less, n_eq;
        const uint32_t s = kth_sum(keys, cnt, kk, n_less, n_eq);
        uint64_t prefix = (uint64_t)s << 32;
        uint32_t k2 = kk - n_less;
        for (int shift = 24; shift >= 0; shift -= 8) {
            histogram(keys, cnt, prefix, shift);
            find(k2);
            prefix |= (uint64_t)res[0] << shift;
            k2 -= res[1];
            __syncthreads();
        }
        return prefix;
    }

    // Bitonic sort of keys[0..P), P a power of two.
    __device__ void sort_pow2(uint64_t *keys, int P) {
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < P / 2; i += T) {
                    const int lo = 2 * i - (i & (stride - 1));
                    const int hi = lo + stride;
                    const bool asc = (lo & size) == 0;
                    const uint64_t a = keys[lo], b = keys[hi];
                    if ((a > b) == asc) {
                        keys[lo] = b;
                        keys[hi] = a;
                    }
                }
                __syncthreads();
            }
        }
    }
};

// ------------------------------------------------------------------ kernel
constexpr uint32_t kThrAll = 0x10000u;  // insert iff s' < thr: everything passes
constexpr int kRankSortMax = 1024;      // merge sorts by rank counting up to this many keys
constexpr int kTmpKeys = kBins / 2;     // survivors that fit in the histogram area as keys

// Block-wide histogram of the buffer over s' bins and k-th bin search.
template <int T>
struct BinSel {
    uint32_t *hist;  // kBins counters
    uint32_t *res;   // [0] bin, [1] count with bin <= res[0], [2..2+T/32) warp sums
    int hshift;

    __device__ void clear() {
        for (int i = threadIdx.x; i < kBins; i += T) hist[i] = 0;
        __syncthreads();
    }
    __device__ void count(const uint64_t *keys, int cnt) {
        clear();
        for (int i = threadIdx.x; i < cnt; i += T) atomicAdd(&hist[(uint32_t)(kv(keys[i]) >> 32) >> hshift], 1u);
        __syncthreads();
    }
    // Copy the global histogram in: every load is issued before any store so
    // the L2 round trips overlap.
    __device__ void load_global(const uint32_t *g) {
        constexpr int BPT = kBins / T;
        uint32_t v[BPT];
#pragma unroll
        for (int i = 0; i < BPT; ++i) v[i] = __ldcg(g + threadIdx.x + i * T);
#pragma unroll
        for (int i = 0; i < BPT; ++i) hist[threadIdx.x + i * T] = v[i];
        __syncthreads();
    }
    // Smallest bin b with (#entries in bins <= b) >= kk: res[0] = b, res[1] =
    // that count.  res[0] = kBins and res[1] = total when total < kk.
    __device__ void find(uint32_t kk) {
        constexpr int BPT = kBins / T;
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        uint32_t *wsum = res + 2;
        uint32_t local = 0;
#pragma unroll 8
        for (int i = 0; i < BPT; ++i) local += hist[tid * BPT + i];
        uint32_t incl = local;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        if (tid == 0) {
            res[0] = kBins;
            res[1] = 0;
        }
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < T / 32; ++w) {
            const uint32_t c = wsum[w];
            before += w < warp ? c : 0;
            total += c;
        }
        const uint32_t excl = before + incl - local;
        if (total < kk) {
            if (tid == 0) res[1] = total;
        } else if (excl < kk && kk <= excl + local) {
            uint32_t c = excl;
            for (int i = 0; i < BPT; ++i) {
                c += hist[tid * BPT + i];
                if (c >= kk) {
                    res[0] = tid * BPT + i;
                    res[1] = c;
                    break;
                }
            }
        }
        __syncthreads();
    }
};

// Stable in-place compaction of keys[0..cnt) keeping pred(key); returns the
// new count.  wcnt: T/32 scratch words.
template <int T, typename P>
__device__ int keep_if(uint64_t *keys, int cnt, uint32_t *wcnt, P pred) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int out = 0;
    for (int base = 0; base < cnt; base += T) {
        const int i = base + tid;
        const uint64_t key = i < cnt ? keys[i] : 0ull;
        const bool keep = i < cnt && pred(key);
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < T / 32; ++w) {
            const int c = wcnt[w];
            off += w < warp ? c : 0;
            tot += c;
        }
        if (keep) keys[out + off + __popc(bal & lanemask_lt())] = key;
        out += tot;
        __syncthreads();
    }
    return out;
}

// MT > 0 fixes the codebook count at compile time (fully unrolled lookups);
// MT = 0 reads it from M.
// BPI: code blocks per unit of work (one bulk copy, one loop iteration).
template <int WARPS, int MT, int BPI>
__global__ void __launch_bounds__(WARPS * 32, 1)
    topk_kernel(const uint32_t *__restrict__ codes, int64_t n, int32_t M, const uint8_t *__restrict__ luts,
                int32_t k, int32_t metric, TopkWS ws, int stages, int cap, int hshift, int64_t blocks_per_cta,
                int out_cap, uint16_t *__restrict__ out_sums, int64_t *__restrict__ out_idx,
                const uint32_t *__restrict__ active, uint64_t wait_ns) {
    constexpr int T = WARPS * 32;
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q = blockIdx.y;
    if (active != nullptr && active[q] == 0u) return;  // only the queries marked for this kernel
    const int G = gridDim.x, cta = blockIdx.x;
    if (MT > 0) M = MT;
    BOLT_STAMP(g_stamps_topk, q, cta, 0);
    const uint32_t blk_bytes = (uint32_t)M * kRowBytes;
    const uint32_t stage_bytes = BPI * blk_bytes;

    uint8_t *p = smem;
    uint8_t *stage_base = p;
    p += (size_t)WARPS * stages * stage_bytes;
    uint64_t *keys = reinterpret_cast<uint64_t *>(p);
    p += (size_t)cap * 8;
    uint4 *lut = reinterpret_cast<uint4 *>(p);
    p += (size_t)M * 16;
    uint64_t *bars = reinterpret_cast<uint64_t *>(p);
    p += (size_t)WARPS * kMaxStages * 8;
    uint32_t *hist = reinterpret_cast<uint32_t *>(p);
    p += kBins * 4;
    uint32_t *misc = reinterpret_cast<uint32_t *>(p);
    p += 128 * 4;
    uint32_t *chist = reinterpret_cast<uint32_t *>(p);  // [kSeedBins] coarse counts of the first round
    // misc: [0] buffer count [1] insert threshold [2] failure flag [3] last CTA
    //       [26], [27] tie rule: a key with s' == misc[26] and index > misc[27] is not inserted
    //       [4] scratch [8..26) BinSel results [32..48) keep_if counts [48..50) test barrier
    //       [64..66) BlockSel
    BinSel<T> bins{hist, misc + 8, hshift};
    BlockSel<T> sel{hist, misc + 64};
    uint32_t *wcnt = misc + 32;
    volatile uint32_t *vmisc = misc;
    uint32_t *ghist = ws.ghist + q * kBins;
    uint32_t *gcoarse = ws.gcoarse + q * (kBins / 16);

    // Indices fit in 32 bits (n < 2^31 vectors).  Work units are BPI
    // consecutive blocks; the CTA owns units [u_lo, u_hi).
    const uint32_t nb = (uint32_t)num_blocks(n);
    const uint32_t nu = (nb + BPI - 1) / BPI;
    const uint32_t u_lo = (uint32_t)min((int64_t)nu, (int64_t)cta * blocks_per_cta);
    const uint32_t u_hi = (uint32_t)min((int64_t)nu, (int64_t)u_lo + blocks_per_cta);
    const uint32_t last_block = nb - 1;  // the only block that can hold vectors past n
    const uint32_t blk_words = (uint32_t)M * kRowWords;
    uint64_t *mybars = bars + warp * stages;
    uint8_t *mystage = stage_base + (size_t)warp * stages * stage_bytes;
    // bytes of unit u (the last unit may hold fewer than BPI blocks)
    auto unit_bytes = [&](uint32_t u) -> uint32_t { return min((uint32_t)BPI, nb - u * BPI) * blk_bytes; };

    // lane 0 of each warp is the producer of its ring
    uint32_t pending = 0;  // stages with a copy in flight (lane 0)
    uint32_t phase = 0;    // parity of the next completion of each stage (lane 0)
    if (lane == 0) {
        // each warp's ring barriers are its own: initialize them and start
        // the first copies before the rest of the setup
        for (int s = 0; s < stages; ++s) mbar_init(&mybars[s], 1);
        fence_mbar_init();
        for (int s = 0; s < stages; ++s) {
            const uint32_t u = u_lo + (uint32_t)s * WARPS + warp;
            if (u < u_hi) {
                const uint32_t bytes = unit_bytes(u);
                mbar_arrive_expect_tx(&mybars[s], bytes);
                bulk_g2s(mystage + (size_t)s * stage_bytes, codes + (size_t)u * BPI * blk_words, bytes, &mybars[s]);
                pending |= 1u << s;
            }
        }
    }

    // For dot the tables are complemented (255 - D is the byte complement),
    // so the scan yields s' = 255*M - S directly.
    const uint4 *lut_g = reinterpret_cast<const uint4 *>(luts + q * M * kK);
    const uint32_t lut_x = metric == BOLT_METRIC_DOT ? 0xFFFFFFFFu : 0u;
    for (int i = tid; i < M; i += T) {
        const uint4 t = lut_g[i];
        lut[i] = make_uint4(t.x ^ lut_x, t.y ^ lut_x, t.z ^ lut_x, t.w ^ lut_x);
    }
    // Tests of the timeout path (data-wait limit below kPollBelowNs): every
    // warp's first wait is on misc[48..49], an mbarrier that nothing arrives
    // on, so it gives up and the CTA takes its failure path with real copies
    // in flight (they complete on their own barriers and are drained).
    const bool test_stall = wait_ns < kPollBelowNs;
    uint64_t *dead = reinterpret_cast<uint64_t *>(misc + 48);
    if (tid == 0) {
        if (test_stall) {
            mbar_init(dead, 1);
            fence_mbar_init();
        }
        misc[0] = 0;
        misc[1] = kThrAll;
        misc[2] = 0;
        misc[3] = 0;
        misc[6] = 0;  // cooperative-phase requests
        misc[26] = 0xFFFFFFFFu;  // no tie rule
        misc[7] = 0;  // warps out of blocks
    }
    for (int i = tid; i < kBins; i += T) hist[i] = 0u;  // seeding histograms (first round)
    for (int i = tid; i < kSeedBins; i += T) chist[i] = 0u;
    __syncthreads();

    // Global bound.  prefetch(): issue the loads of the global histogram into
    // registers.  finish(): hist := that snapshot plus this CTA's entries not
    // yet counted, which are also added to the global histogram and flagged;
    // then lower the threshold to the bin holding the k-th smallest count.
    constexpr int GPT = kBins / T;
    uint32_t gv[GPT];
    auto prefetch = [&]() {
#pragma unroll
        for (int i = 0; i < GPT; ++i) gv[i] = __ldcg(ghist + tid + i * T);
    };
    auto finish = [&](int cnt) -> uint32_t {
#pragma unroll
        for (int i = 0; i < GPT; ++i) hist[tid + i * T] = gv[i];
        __syncthreads();
        for (int i = tid; i < cnt; i += T) {
            const uint64_t key = keys[i];
            if (!(key & kFlag)) {
                atomicAdd(&hist[(uint32_t)(key >> 32) >> hshift], 1u);
                keys[i] = key | kFlag;
            }
        }
        __syncthreads();
        // this CTA's new entries per bin: one global add per non-empty bin
#pragma unroll
        for (int i = 0; i < GPT; ++i) {
            const uint32_t d = hist[tid + i * T] - gv[i];
            if (d) {
                atomicAdd(&ghist[tid + i * T], d);
                atomicAdd(&gcoarse[(tid + i * T) >> 4], d);
            }
        }
        bins.find((uint32_t)k);
        const uint32_t bg = bins.res[0];
        if (tid == 0 && bg < (uint32_t)kBins) {
            const uint32_t gthr = (bg + 1u) << hshift;
            if (gthr < vmisc[1]) vmisc[1] = gthr;
        }
        __syncthreads();
        return bg;
    };

    // Global bound read by one warp from the global histograms.  Counts only
    // grow and count distinct vectors, so any snapshot gives a valid bound.
    auto warp_refresh = [&]() {
        uint32_t cbin, fbin, in_bin, c[8];
        if (warp_kth_bin<true>(gcoarse, ghist, (uint32_t)k, lane, cbin, fbin, in_bin, c) && lane == 0)
            atomicMin(&misc[1], (fbin + 1u) << hshift);
    };

    bool failed = false;
    const uint32_t smax = 255u * (uint32_t)M;  // largest possible sum
    const bool swar = smax <= 0x7FFFu;  // sums fit in 15 bits (M <= 128)
    const uint32_t gate = (uint32_t)(cap - WARPS * BPI * kBlockVecs / 2);  // compact above this count
    // before the first compaction: compact as soon as a few blocks are in
    const uint32_t early = min(gate, max((uint32_t)(2 * k), (uint32_t)(WARPS * BPI * kBlockVecs)));
    const uint32_t one = kMulOne;
    bool compacted = false;  // same value in every thread (set in cooperative())

    // Cooperative compaction.  Warps run independently; a warp that finds the
    // buffer full (or above the compaction gate) sets misc[6] and every warp
    // joins at its next check (the request is only cleared inside the phase,
    // between two barriers, so each warp joins each phase exactly once).
    auto cooperative = [&]() {
        __syncthreads();
        const int cnt = (int)vmisc[0];
        // Keep every entry up to the bin of the k-th smallest s'.
        prefetch();  // global histogram loads overlap the local selection
        bins.count(keys, cnt);
        bins.find((uint32_t)k);
        const uint32_t bstar = bins.res[0], c_le = bins.res[1];
        int kept;
        uint32_t own;
        if (cnt <= k) {
            kept = cnt;
            own = vmisc[1];
        } else if (c_le <= (uint32_t)kTmpKeys) {
            // Few survivors: append them to the (now free) histogram area,
            // then copy them back to the front of the buffer.
            uint64_t *tmp = reinterpret_cast<uint64_t *>(hist);
            if (tid == 0) misc[5] = 0;
            __syncthreads();
            for (int i0 = 0; i0 < cnt; i0 += T) {
                const int i = i0 + tid;
                const uint64_t key = i < cnt ? keys[i] : 0ull;
                const bool keep = i < cnt && ((uint32_t)(kv(key) >> 32) >> hshift) <= bstar;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
                if (bal) {
                    const int leader = __ffs(bal) - 1;
                    uint32_t base = 0;
                    if (lane == leader) base = atomicAdd(&misc[5], (uint32_t)__popc(bal));
                    base = __shfl_sync(0xFFFFFFFFu, base, leader);
                    if (keep) tmp[base + __popc(bal & lanemask_lt())] = key;
                }
            }
            __syncthreads();
            kept = (int)vmisc[5];
            for (int i = tid; i < kept; i += T) keys[i] = tmp[i];
            __syncthreads();
            // inclusive: a warp that lags may still bring keys equal to
            // the bin's values with lower indices than kept ones
            own = (bstar + 1u) << hshift;
        } else if (c_le <= gate) {
            kept = keep_if<T>(keys, cnt, wcnt,
                              [&](uint64_t key) { return ((uint32_t)(kv(key) >> 32) >> hshift) <= bstar; });
            own = (bstar + 1u) << hshift;
        } else {  // one bin holds too many entries: exact k-th key
            const uint64_t kth = sel.kth_key(keys, cnt, (uint32_t)k);
            kept = keep_if<T>(keys, cnt, wcnt, [&](uint64_t key) { return kv(key) <= kth; });
            // keys after the k-th key cannot enter: s' above it, or equal
            // with a higher index (warps are not in lockstep, so a lower
            // index can still arrive)
            own = (uint32_t)(kth >> 32) + 1u;
            if (tid == 0) {
                misc[26] = (uint32_t)(kth >> 32);
                misc[27] = (uint32_t)kth;
            }
        }
        if (tid == 0) {
            misc[0] = (uint32_t)kept;
            if (own < vmisc[1]) vmisc[1] = own;
        }
        __syncthreads();
        finish(kept);
        compacted = true;
        if (tid == 0) misc[6] = 0;
        __syncthreads();
    };
    auto requests = [&]() -> uint32_t {
        uint32_t f = lane == 0 ? vmisc[6] : 0u;
        return __shfl_sync(0xFFFFFFFFu, f, 0);
    };

    // warps that have a first unit take part in seeding the threshold
    const uint32_t seeders = u_hi > u_lo ? min((uint32_t)WARPS, u_hi - u_lo) : 0u;
    uint32_t st = 0, par = 0;  // stage and parity of this warp's current unit
    uint32_t j = 0;            // units done by this warp
    uint32_t next_refresh = 4u * (uint32_t)warp + 1u;  // this warp's next refresh round

    for (uint32_t u = u_lo + warp;; u += WARPS, ++j) {
        if (requests()) cooperative();
        if (u >= u_hi || failed) break;
        uint64_t *wbar = test_stall && j == 0 ? dead : &mybars[st];
        if (!__all_sync(0xFFFFFFFFu, test_stall ? mbar_test_wait(wbar, par) : mbar_try_wait(wbar, par))) {
            const bool ok = test_stall ? mbar_poll_bounded(wbar, par, wait_ns) : mbar_wait_bounded(wbar, par, wait_ns);
            if (!__all_sync(0xFFFFFFFFu, ok)) {
                failed = true;
                if (j == 0) seed_barrier(seeders);  // the other seeders still count on this warp
                continue;
            }
        }
        const uint32_t *words = reinterpret_cast<const uint32_t *>(mystage + (size_t)st * stage_bytes);
        Acc8 acc[BPI];
#pragma unroll
        for (int h = 0; h < BPI; ++h) acc[h].zero();
        // (a missing second block of the last unit reads stale stage data; its
        // sums are masked out below)
        if (MT > 0) {
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const uint4 t = lut[m];
#pragma unroll
                for (int h = 0; h < BPI; ++h) acc[h].add(prep_word(words[h * blk_words + m * kRowWords + lane]), t);
            }
        } else {
#pragma unroll 4
            for (int m = 0; m < M; ++m) {
                const uint4 t = lut[m];
#pragma unroll
                for (int h = 0; h < BPI; ++h) acc[h].add(prep_word(words[h * blk_words + m * kRowWords + lane]), t);
            }
        }
        __syncwarp();
        if (lane == 0) {
            pending &= ~(1u << st);
            phase ^= 1u << st;
            const uint32_t u2 = u + (uint32_t)stages * WARPS;
            if (u2 < u_hi) {
                const uint32_t bytes = unit_bytes(u2);
                mbar_arrive_expect_tx(&mybars[st], bytes);
                bulk_g2s(mystage + (size_t)st * stage_bytes, codes + (size_t)u2 * BPI * blk_words, bytes,
                         &mybars[st]);
                pending |= 1u << st;
            }
        }
        if (++st == (uint32_t)stages) {
            st = 0;
            par ^= 1u;
        }
        // sw[h]: the unit's 8 sums s' per lane in 16-bit lanes (s'_0 | s'_2 << 16,
        // s'_1 | s'_3 << 16, then vectors 4..7); sum_of(h, i) is vector i's s'.
        // Vector vbase + 256 h + i exists iff its index is below n (a missing
        // second block of the last unit lies past n).
        uint32_t sw[BPI][4];
#pragma unroll
        for (int h = 0; h < BPI; ++h) acc[h].finish(sw[h][0], sw[h][1], sw[h][2], sw[h][3]);
        const uint32_t vbase = u * (uint32_t)(BPI * kBlockVecs) + 8u * lane;
        // every block of the unit lies before the last block: all its vectors exist
        const bool whole = u * (uint32_t)BPI + (uint32_t)(BPI - 1) < last_block;
        auto sum_of = [&](int h, int i) -> uint32_t {
            return (sw[h][(i & 1) + 2 * (i >> 2)] >> (16 * ((i >> 1) & 1))) & 0xFFFFu;
        };
        auto exists = [&](int h, int i) -> bool { return vbase + (uint32_t)(h * kBlockVecs + i) < (uint32_t)n; };
        uint32_t thr = vmisc[1];
        if (j == 0) {
            // Seed the threshold from the CTA's first round: every warp counts
            // its first unit's sums in shared fine and coarse histograms;
            // after all of them have, the k-th smallest s' of those vectors
            // lies in fine bin b, so k vectors have s' < (b + 1) << hshift and
            // no larger s' can enter the top k.
#pragma unroll
            for (int h = 0; h < BPI; ++h)
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const uint32_t sp = sum_of(h, i);
                    if (whole || exists(h, i)) {
                        atomicAdd(&hist[sp >> hshift], 1u);
                        atomicAdd(&chist[sp >> (hshift + 4)], 1u);
                    }
                }
            seed_barrier(seeders);
            BOLT_STAMP(g_stamps_topk, q, cta, 1);
            uint32_t cbin, fbin, in_bin, c[8];
            if (warp_kth_bin<false>(chist, hist, (uint32_t)k, lane, cbin, fbin, in_bin, c)) {
                const uint32_t seed = (fbin + 1u) << hshift;
                if (lane == 0) atomicMin(&misc[1], seed);
                thr = min(thr, seed);
                // Publish the first-round counts up to bin b (at least k
                // distinct vectors, the keys inserted below) to the global
                // histograms, one add per non-empty bin.
                if (warp == 0) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const uint32_t cb = (uint32_t)(lane * 8 + i);
                        if (cb < cbin && c[i]) atomicAdd(&gcoarse[cb], c[i]);
                    }
                    if (lane == 0) atomicAdd(&gcoarse[cbin], in_bin);
                }
                for (uint32_t f0 = (uint32_t)warp * 256u; f0 <= fbin; f0 += WARPS * 256u) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const uint32_t f = f0 + (uint32_t)(lane * 8 + i);
                        const uint32_t v = f <= fbin ? hist[f] : 0u;
                        if (v) atomicAdd(&ghist[f], v);
                    }
                }
            }
        }
        // Threshold filter: with s' < 2^15 the top bit of (s' + 2^15 - thr) in
        // each 16-bit lane is clear exactly when s' < thr, with no borrow
        // between lanes; one AND over the unit's words tests all its sums.
        // The last unit (and any M with wider sums) goes to the exact test.
        bool maybe = true;
        if (whole && swar && thr <= 0x7FFFu) {
            const uint32_t nt2 = 0x80008000u - (thr | (thr << 16));
            uint32_t d = 0xFFFFFFFFu;
#pragma unroll
            for (int h = 0; h < BPI; ++h)
                d &= imad(sw[h][0], one, nt2) & imad(sw[h][1], one, nt2) & imad(sw[h][2], one, nt2) &
                     imad(sw[h][3], one, nt2);
            maybe = (~d & 0x80008000u) != 0u;
        }
        if (__any_sync(0xFFFFFFFFu, maybe)) {
            // first-round keys are already in the global counts (seeding)
            const uint64_t counted = j == 0 ? kFlag : 0ull;
            uint32_t tie_v = vmisc[26], tie_i = vmisc[27];
            for (int attempt = 0;; ++attempt) {
                // One warp prefix sum places every lane's candidates; the slots
                // are reserved with a compare-and-swap that never passes cap.
                uint32_t cm = 0;
#pragma unroll
                for (int h = 0; h < BPI; ++h)
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const uint32_t sp = sum_of(h, i);
                        const uint32_t v = vbase + (uint32_t)(h * kBlockVecs + i);
                        if (sp < thr && v < (uint32_t)n && !(sp == tie_v && v > tie_i)) cm |= 1u << (8 * h + i);
                    }
                const uint32_t c = __popc(cm);
                uint32_t incl = c;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
                    if (lane >= off) incl += t;
                }
                uint32_t base = 0, ok = 1;
                if (lane == 31 && incl) {
                    ok = 0;
                    for (int spin = 0; spin < (1 << 20); ++spin) {
                        const uint32_t old = vmisc[0];
                        if (old + incl > (uint32_t)cap) break;
                        if (atomicCAS(&misc[0], old, old + incl) == old) {
                            base = old;
                            ok = 1;
                            break;
                        }
                    }
                }
                ok = __shfl_sync(0xFFFFFFFFu, ok, 31);
                if (ok) {
                    base = __shfl_sync(0xFFFFFFFFu, base, 31);
                    uint32_t pos = base + incl - c;
#pragma unroll
                    for (int h = 0; h < BPI; ++h)
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            if (cm & (1u << (8 * h + i))) {
                                const uint32_t sp = sum_of(h, i);
                                keys[pos++] =
                                    ((uint64_t)sp << 32) | (uint64_t)(vbase + (uint32_t)(h * kBlockVecs + i)) | counted;
                            }
                        }
                    break;
                }
                // Buffer full: compact with the whole CTA, then retry with the
                // tighter threshold.
                if (lane == 0) atomicOr(&misc[6], 1u);
                cooperative();
                thr = vmisc[1];
                tie_v = vmisc[26];
                tie_i = vmisc[27];
            }
            if (lane == 0 && vmisc[0] > (compacted ? gate : early)) atomicOr(&misc[6], 1u);
        }
        // every 4 rounds one warp (in turn) lowers the threshold to the
        // global bound: warp w at its rounds 4w + 1 + 4 WARPS t
        if (j == next_refresh) {
            warp_refresh();
            next_refresh += 4u * WARPS;
        }
    }
    // This warp is out of blocks: start the loads of the global histogram
    // for the final bound (a later cooperative phase reloads them), then keep
    // joining cooperative phases until every warp is done (each of them
    // reaches this point in bounded time).
    prefetch();
    if (lane == 0) atomicAdd(&misc[7], 1u);
    {
        const uint64_t t0 = globaltimer_ns();
        while (true) {
            uint32_t f = 0, d = 0;
            if (lane == 0) {
                f = vmisc[6];
                d = vmisc[7];
            }
            f = __shfl_sync(0xFFFFFFFFu, f, 0);
            d = __shfl_sync(0xFFFFFFFFu, d, 0);
            if (f) {
                cooperative();
                continue;
            }
            if (d == (uint32_t)WARPS) break;
            __nanosleep(64);
            if (globaltimer_ns() - t0 > 4 * kWaitLimit) {
                failed = true;
                break;
            }
        }
    }
    __syncthreads();

    BOLT_STAMP(g_stamps_topk, q, cta, 2);
    // Wait (bounded) for copies still in flight after a failure, so that no
    // bulk copy targets this CTA's shared memory after it exits.
    if (failed && lane == 0) {
        for (int s = 0; s < stages; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&mybars[s], (phase >> s) & 1u, kWaitLimit / 10);
    }
    if (failed) atomicOr(&misc[2], 1u);
    __syncthreads();

    // Candidates of this CTA up to the global bound (at most 2k of them),
    // published to the CTA's own slot of the query's list: slot[0] holds the
    // count, the keys follow.
    int cnt = (int)vmisc[0];
    const uint32_t bg = finish(cnt);
    cnt = keep_if<T>(keys, cnt, wcnt,
                     [&](uint64_t key) { return ((uint32_t)(kv(key) >> 32) >> hshift) <= bg; });
    if (cnt > out_cap) {
        const uint64_t kth = sel.kth_key(keys, cnt, (uint32_t)k);
        cnt = keep_if<T>(keys, cnt, wcnt, [&](uint64_t key) { return kv(key) <= kth; });
    }
    const int64_t slot_len = (int64_t)out_cap + 1;
    uint64_t *slots = ws.cand + q * (slot_len * G);
    uint64_t *slot = slots + cta * slot_len;
    for (int i = tid; i < cnt; i += T) slot[1 + i] = kv(keys[i]);
    if (tid == 0) {
        slot[0] = (uint64_t)cnt;
        if (misc[2]) atomicOr(&ws.status[q], 1u);
    }
    __threadfence();
    __syncthreads();
    BOLT_STAMP(g_stamps_topk, q, cta, 3);
    BOLT_STAMP_VALUE(g_stamps_topk, q, cta, 5, cnt);
    if (tid == 0) misc[3] = (atomicAdd(&ws.ticket[q], 1u) == (uint32_t)(G - 1)) ? 1u : 0u;
    __syncthreads();
    if (vmisc[3] == 0) return;
    __threadfence();

    // Last CTA.  Warp 0: exclusive prefix of the slot counts (off[c], with
    // off[G] the total) and the failure status; warp 1, at the same time: the
    // final bound bin from the complete global histogram (every CTA added
    // its counts before taking its ticket).  Then all threads gather the
    // keys, only those at or below the bound bin when there are more than
    // kRankSortMax of them; the (unique) keys are selected and sorted below.
    uint32_t *off = hist;  // [G + 1]; the histogram area is free in the last CTA
    if (warp == 0) {
        uint32_t run = 0;
        for (int c0 = 0; c0 < G; c0 += 256) {
            uint32_t v[8], loc = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = c0 + lane * 8 + i;
                v[i] = c < G ? (uint32_t)__ldcg(slots + c * slot_len) : 0u;
                loc += v[i];
            }
            uint32_t incl = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += t;
            }
            uint32_t e = run + incl - loc;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = c0 + lane * 8 + i;
                if (c < G) off[c] = e;
                e += v[i];
            }
            run += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
        if (lane == 0) {
            off[G] = run;
            misc[2] = __ldcg(&ws.status[q]);
        }
    } else if (warp == 1) {
        uint32_t cbin, fbin, in_bin, c[8];
        const bool ok = warp_kth_bin<true>(gcoarse, ghist, (uint32_t)k, lane, cbin, fbin, in_bin, c);
        if (lane == 0) misc[5] = ok ? fbin : 0xFFFFFFFFu;
    }
    __syncthreads();
    const uint32_t total = vmisc_hist(off, G);
    BOLT_STAMP(g_stamps_topk, q, cta, 8);
    BOLT_STAMP_VALUE(g_stamps_topk, q, cta, 6, total);
    const uint32_t bfin = total > (uint32_t)kRankSortMax ? vmisc[5] : 0xFFFFFFFFu;
    uint64_t *mk = reinterpret_cast<uint64_t *>(smem);
    uint32_t kept_all = 0;
    constexpr int kGather = 8;  // keys per thread per gather round: 4,096 keys in one round at 512 threads
    int steps = 0;  // binary-search steps over the G slots
    while ((1 << steps) < G) ++steps;
    for (uint32_t e0 = 0; e0 < total; e0 += kGather * T) {
        // slot of entry e: the last c with off[c] <= e (kGather searches in step)
        uint32_t e[kGather];
        int lo[kGather];
#pragma unroll
        for (int u = 0; u < kGather; ++u) {
            e[u] = e0 + u * T + tid;
            lo[u] = 0;
        }
        for (int bit = steps - 1; bit >= 0; --bit) {
#pragma unroll
            for (int u = 0; u < kGather; ++u) {
                const int mid = lo[u] + (1 << bit);
                if (mid < G && off[mid] <= e[u]) lo[u] = mid;
            }
        }
        uint64_t v[kGather];
#pragma unroll
        for (int u = 0; u < kGather; ++u)
            v[u] = e[u] < total ? __ldcg(slots + lo[u] * slot_len + 1 + (e[u] - off[lo[u]])) : ~0ull;
        // kept keys: warp ballots counted, a prefix over the warps, then the
        // writes (no shared-memory atomics)
        uint32_t bal[kGather], cw = 0;
#pragma unroll
        for (int u = 0; u < kGather; ++u) {
            bal[u] = __ballot_sync(0xFFFFFFFFu, v[u] != ~0ull && ((uint32_t)(v[u] >> 32) >> hshift) <= bfin);
            cw += __popc(bal[u]);
        }
        if (lane == 0) wcnt[warp] = cw;
        __syncthreads();
        uint32_t pos = kept_all, tot = 0;
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t c = wcnt[w];
            pos += w < warp ? c : 0u;
            tot += c;
        }
#pragma unroll
        for (int u = 0; u < kGather; ++u) {
            if (bal[u] & (1u << lane)) mk[pos + __popc(bal[u] & lanemask_lt())] = v[u];
            pos += __popc(bal[u]);
        }
        kept_all += tot;
        __syncthreads();
    }
    int g = (int)kept_all;
    BOLT_STAMP(g_stamps_topk, q, cta, 9);
    BOLT_STAMP_VALUE(g_stamps_topk, q, cta, 7, g);
    const bool bad = vmisc[2] != 0u;
    auto emit = [&](int r, uint64_t key) {
        const uint32_t sp = (uint32_t)(key >> 32);
        out_sums[q * k + r] = (uint16_t)(metric == BOLT_METRIC_DOT ? 255u * (uint32_t)M - sp : sp);
        out_idx[q * k + r] = bad ? -2 : (int64_t)(uint32_t)key;
    };
    const int kout = g < k ? g : k;
    if (g <= kRankSortMax) {
        // Keys are unique: each key's rank is the number of smaller keys,
        // counted by P threads (adjacent lanes) per key.
        int P = 1;
        while (P < 32 && g * P * 2 <= T) P <<= 1;
        const int part = tid & (P - 1);
        for (int base = 0; base < g; base += T / P) {
            const int e = base + tid / P;
            const uint64_t key = e < g ? mk[e] : ~0ull;
            int rank = 0;
            if (e < g)
                for (int jj = part; jj < g; jj += P) rank += mk[jj] < key ? 1 : 0;
            for (int off = 1; off < P; off <<= 1) rank += __shfl_xor_sync(0xFFFFFFFFu, rank, off);
            if (e < g && part == 0 && rank < k) emit(rank, key);
        }
    } else {
        const uint64_t kth = sel.kth_key(mk, g, (uint32_t)k);
        g = keep_if<T>(mk, g, wcnt, [&](uint64_t key) { return key <= kth; });
        int P = 1;
        while (P < kout) P <<= 1;
        for (int i = kout + tid; i < P; i += T) mk[i] = ~0ull;
        __syncthreads();
        sel.sort_pow2(mk, P);
        for (int r = tid; r < kout; r += T) emit(r, mk[r]);
    }
    for (int r = kout + tid; r < k; r += T) {
        out_sums[q * k + r] = 0;
        out_idx[q * k + r] = bad ? -2 : -1;
    }
    BOLT_STAMP(g_stamps_topk, q, cta, 4);
}

// ------------------------------------------------------------------ host side
static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int plan_topk(int64_t n, int32_t M, int32_t k, int64_t nq, TopkPlan *plan) {
    BOLT_REQUIRE(k >= 1 && k <= kMaxK, BOLT_EUNSUPPORTED, "k=%d outside [1, %d]", k, kMaxK);
    plan->small = 0;
    plan->nbc = 0;
    plan->mq = 0;
    const int sms = device_sm_count();
    // Tiny databases with several queries: fewer CTAs per query (still one
    // per SM over all the queries), each with a few blocks, so the last CTA
    // of a query merges fewer lists.  Applied only while a CTA keeps at most
    // 8 blocks.
    if (nq > 1 && sms > 0) {
        const int64_t nb = num_blocks(n), fill = (sms + nq - 1) / nq;
        if (fill < nb && fill < sms && (nb + fill - 1) / fill <= 8 && plan_topk_small(n, M, k, sms, plan, fill))
            return BOLT_OK;
    }
    if (plan_topk_small(n, M, k, sms, plan)) return BOLT_OK;
    int rc = plan_topk_stream(n, M, k, plan);
    if (rc) return rc;
    // several queries share each code pass in the multi-query pipeline; a
    // single query is faster in the fused streaming kernel
    if (n > 0 && nq >= kMqMinQueries) plan_topk_mq(n, M, k, device_sm_count(), plan);
    return BOLT_OK;
}

int plan_topk_stream(int64_t n, int32_t M, int32_t k, TopkPlan *plan) {
    // Two blocks per unit of work for small M on large databases (amortizes
    // per-unit overhead once every warp has many blocks to stream).
    const int64_t blocks_per_warp = num_blocks(n) / ((int64_t)(device_sm_count() > 0 ? device_sm_count() : 1) * 16);
    const int bpi = ((M == 8 || M == 16) && blocks_per_warp >= 16) ? 2 : 1;
    const size_t stage_bytes = (size_t)bpi * M * kRowBytes;
    int warps = 16, stages = 0;
    for (warps = 16; warps >= 2; warps >>= 1) {
        stages = (int)(kStageBudget / (warps * stage_bytes));
        if (stages > kMaxStages) stages = kMaxStages;
        if (stages >= 2) break;
    }
    BOLT_REQUIRE(stages >= 2, BOLT_EUNSUPPORTED, "M=%d too large for the top-k kernel", M);
    // room for one unit of candidates per warp above the compaction gate;
    // a multiple of 16 keeps the later shared-memory regions aligned
    const int cap = (k + 15) / 16 * 16 + warps * bpi * kBlockVecs;
    int hshift = 0;
    while (((255 * M) >> hshift) >= kBins) ++hshift;
    const int64_t nb = num_blocks(n);
    const int64_t nu = (nb + bpi - 1) / bpi;
    const size_t region = (size_t)warps * stages * stage_bytes + (size_t)cap * 8;
    const int64_t merge_keys = (int64_t)(region / 8);
    int64_t g = device_sm_count();
    if (g <= 0) g = 1;
    const int64_t by_work = (nu + warps - 1) / warps;  // at least one unit per warp
    if (g > by_work) g = by_work;
    if (g > merge_keys / k) g = merge_keys / k;  // the merge holds every CTA's list
    if (g < 1) g = 1;
    int64_t out_cap = merge_keys / g;  // candidates one CTA may hand to the merge (>= k)
    if (out_cap > 2 * k) out_cap = 2 * k;
    plan->warps = warps;
    plan->bpi = bpi;
    plan->stages = stages;
    plan->grid = (int)g;
    plan->cap = cap;
    plan->hshift = hshift;
    plan->out_cap = (int)out_cap;
    plan->list_cap = (int)(g * (out_cap + 1));  // one slot per CTA: count, then keys
    plan->blocks_per_cta = nu > 0 ? (nu + g - 1) / g : 0;  // units per CTA
    plan->smem_bytes = region + align_up((size_t)M * 16, 16) + (size_t)warps * kMaxStages * 8 + kBins * 4 + 128 * 4 +
                       kSeedBins * 4;
    return BOLT_OK;
}

size_t topk_header_bytes(int64_t nq) {
    return align_up((size_t)nq * 8, 256) + (size_t)nq * (kBins + kBins / 16) * 4;
}

int64_t topk_workspace_bytes(const TopkPlan &plan, int64_t nq, int32_t k) {
    if (plan.small) return topk_small_workspace_bytes(plan, nq, k);
    if (plan.mq) return topk_mq_workspace_bytes(plan, nq, k);
    return topk_stream_workspace_bytes(plan, nq, k);
}

int64_t topk_stream_workspace_bytes(const TopkPlan &plan, int64_t nq, int32_t k) {
    (void)k;
    return (int64_t)(topk_header_bytes(nq) + (size_t)nq * plan.list_cap * 8);
}

TopkWS carve_topk_ws(void *ws, const TopkPlan &plan, int64_t nq, int32_t k) {
    uint8_t *p = static_cast<uint8_t *>(ws);
    TopkWS w;
    w.ticket = reinterpret_cast<uint32_t *>(p);
    w.status = w.ticket + nq;
    p += align_up((size_t)nq * 8, 256);
    w.ghist = reinterpret_cast<uint32_t *>(p);
    p += (size_t)nq * kBins * 4;
    w.gcoarse = reinterpret_cast<uint32_t *>(p);
    p += (size_t)nq * (kBins / 16) * 4;
    w.cand = reinterpret_cast<uint64_t *>(p);
    (void)plan;
    (void)k;
    return w;
}

template <int WARPS, int MT, int BPI>
static int launch_w(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                    int32_t metric, uint16_t *out_sums, int64_t *out_idx, const TopkWS &w, const TopkPlan &plan,
                    const uint32_t *active, cudaStream_t stream) {
    auto kern = topk_kernel<WARPS, MT, BPI>;
    int rc = ensure_smem((const void *)kern, plan.smem_bytes);
    if (rc) return rc;
    dim3 grid(plan.grid, (unsigned)nq);
    kern<<<grid, WARPS * 32, plan.smem_bytes, stream>>>(reinterpret_cast<const uint32_t *>(codes), n, M, luts, k,
                                                         metric, w, plan.stages, plan.cap, plan.hshift,
                                                         plan.blocks_per_cta, plan.out_cap, out_sums, out_idx,
                                                         active, data_wait_limit_ns());
    return check_launch("topk_kernel");
}

int launch_topk(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, const TopkPlan &plan,
                cudaStream_t stream) {
    if (plan.small) return launch_topk_small(codes, n, M, luts, nq, k, metric, out_sums, out_idx, workspace, plan,
                                             stream);
    if (plan.mq) return launch_topk_mq(codes, n, M, luts, nq, k, metric, out_sums, out_idx, workspace, plan, stream);
    return launch_topk_stream(codes, n, M, luts, nq, k, metric, out_sums, out_idx, workspace, plan, nullptr, stream);
}

int launch_topk_stream(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                       int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, const TopkPlan &plan,
                       const uint32_t *active, cudaStream_t stream) {
    BOLT_REQUIRE(nq <= 65535, BOLT_EUNSUPPORTED, "nq=%lld > 65535 per call", (long long)nq);
    BOLT_CUDA(cudaMemsetAsync(workspace, 0, topk_header_bytes(nq), stream));
    const TopkWS w = carve_topk_ws(workspace, plan, nq, k);
#define BOLT_TOPK_ARGS codes, n, M, luts, nq, k, metric, out_sums, out_idx, w, plan, active, stream
    if (plan.warps == 16) {
        if (M == 8) return plan.bpi == 2 ? launch_w<16, 8, 2>(BOLT_TOPK_ARGS) : launch_w<16, 8, 1>(BOLT_TOPK_ARGS);
        if (M == 16) return plan.bpi == 2 ? launch_w<16, 16, 2>(BOLT_TOPK_ARGS) : launch_w<16, 16, 1>(BOLT_TOPK_ARGS);
        BOLT_REQUIRE(plan.bpi == 1, BOLT_EUNSUPPORTED, "no streaming kernel for M=%d with %d blocks per unit", M,
                     plan.bpi);
        if (M == 32) return launch_w<16, 32, 1>(BOLT_TOPK_ARGS);
        return launch_w<16, 0, 1>(BOLT_TOPK_ARGS);
    }
    // the generic instantiations stream one block per unit
    BOLT_REQUIRE(plan.bpi == 1, BOLT_EUNSUPPORTED, "no streaming kernel for %d warps, M=%d, %d blocks per unit",
                 plan.warps, M, plan.bpi);
    if (plan.warps == 8) return launch_w<8, 0, 1>(BOLT_TOPK_ARGS);
    if (plan.warps == 4) return launch_w<4, 0, 1>(BOLT_TOPK_ARGS);
    return launch_w<2, 0, 1>(BOLT_TOPK_ARGS);
#undef BOLT_TOPK_ARGS
}

}  // namespace bolt

#ifdef BOLT_PHASE_STAMPS
// Copies the streaming kernel's stamps (1024 CTAs x 16 slots) to host and,
// with clear != 0, zeroes them (diagnostic builds only).
extern "C" int bolt_debug_stamps_topk(unsigned long long *host, int clear) {
    if (cudaMemcpyFromSymbol(host, bolt::g_stamps_topk, sizeof(unsigned long long) * 1024 * 16) != cudaSuccess)
        return BOLT_ECUDA;
    if (clear) {
        static unsigned long long zero[1024 * 16];
        if (cudaMemcpyToSymbol(bolt::g_stamps_topk, zero, sizeof(zero)) != cudaSuccess) return BOLT_ECUDA;
    }
    return BOLT_OK;
}
#endif

extern "C" {

int64_t bolt_topk_workspace_bytes(int64_t n, int32_t M, int64_t nq, int32_t k) {
    bolt::clear_error();
    if (bolt::check_nm(n, M) || nq < 0) return -1;
    bolt::TopkPlan plan;
    if (bolt::plan_topk(n, M, k, nq, &plan)) return -1;
    return bolt::topk_workspace_bytes(plan, nq, k);
}

int bolt_topk(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
              int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, int64_t workspace_bytes,
              void *stream) {
    bolt::clear_error();
    int rc = bolt::check_nm(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(nq >= 0, BOLT_EINVAL, "nq=%lld < 0", (long long)nq);
    BOLT_REQUIRE(bolt::rank_metric_ok(metric), BOLT_EINVAL,
                 "bad metric %d", metric);
    bolt::TopkPlan plan;
    rc = bolt::plan_topk(n, M, k, nq, &plan);
    if (rc) return rc;
    if (nq == 0) return BOLT_OK;
    BOLT_REQUIRE(luts && out_sums && out_idx && (codes || n == 0), BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(luts, 16) && (n == 0 || bolt::aligned(codes, 16)), BOLT_EINVAL,
                 "codes and luts must be 16-byte aligned");
    const int64_t need = bolt::topk_workspace_bytes(plan, nq, k);
    cudaStream_t s = (cudaStream_t)stream;
    if (workspace == nullptr) {
        void *tmp = nullptr;
        BOLT_CUDA(cudaMallocAsync(&tmp, (size_t)need, s));
        rc = bolt::launch_topk(codes, n, M, luts, nq, k, metric, out_sums, out_idx, tmp, plan, s);
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
    return bolt::launch_topk(codes, n, M, luts, nq, k, metric, out_sums, out_idx, workspace, plan, s);
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free variant
// Some callers cannot allocate device memory at call time: code running while
// a CUDA graph is being captured with a strict capture mode, real-time or
// serving loops that forbid allocator calls (and their latency spikes) on the
// request path, and embedders whose own memory manager owns the device heap.
// bolt_topk_noalloc serves them: its scratch space is a fixed array compiled
// into the library, so the call itself never allocates or frees.
namespace bolt {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;  // 4 MiB, held by every GPU that loads the library

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (host code may not use the symbol itself as a device pointer).
static int noalloc_scratch(void **ptr) {
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    int dev = 0;
    BOLT_CUDA(cudaGetDevice(&dev));
    BOLT_REQUIRE(dev >= 0 && dev < 64, BOLT_EUNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (addr[dev] == nullptr) {
        void *p = nullptr;
        BOLT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        addr[dev] = p;
    }
    *ptr = addr[dev];
    return BOLT_OK;
}

}  // namespace bolt

extern "C" int bolt_topk_noalloc(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq,
                                 int32_t k, int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *stream) {
    bolt::clear_error();
    int rc = bolt::check_nm(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(nq >= 0, BOLT_EINVAL, "nq=%lld < 0", (long long)nq);
    BOLT_REQUIRE(bolt::rank_metric_ok(metric), BOLT_EINVAL,
                 "bad metric %d", metric);
    bolt::TopkPlan plan;
    rc = bolt::plan_topk(n, M, k, nq, &plan);
    if (rc) return rc;
    if (nq == 0) return BOLT_OK;
    BOLT_REQUIRE(luts && out_sums && out_idx && (codes || n == 0), BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(bolt::aligned(luts, 16) && (n == 0 || bolt::aligned(codes, 16)), BOLT_EINVAL,
                 "codes and luts must be 16-byte aligned");
    const int64_t need = bolt::topk_workspace_bytes(plan, nq, k);
    BOLT_REQUIRE(need <= (int64_t)bolt::kNoAllocScratchBytes, BOLT_ENOMEM,
                 "bolt_topk_noalloc: %lld queries with k=%d need %lld bytes of scratch, more than its fixed "
                 "%lld-byte array; use fewer queries per call or bolt_topk",
                 (long long)nq, k, (long long)need, (long long)bolt::kNoAllocScratchBytes);
    void *scratch = nullptr;
    rc = bolt::noalloc_scratch(&scratch);
    if (rc) return rc;
    // launch_topk zeroes the per-query header and histograms (cudaMemsetAsync)
    // before the kernel; the candidate lists need no clearing.
    return bolt::launch_topk(codes, n, M, luts, nq, k, metric, out_sums, out_idx, scratch, plan,
                             (cudaStream_t)stream);
}
