// Fused scan + exact top-k for databases whose codes fit, spread over one
// wave of CTAs, in shared memory (about 2.5M vectors at M = 16).
//
// Latency, not bandwidth, decides this size class: every CTA holds only a
// few dozen 256-vector blocks, so the kernel avoids every cooperative phase
// and global round trip of the streaming kernel.
//
// Per CTA (one contiguous range of blocks):
//   1. one thread starts 1-D bulk copies of the whole code range into shared
//      memory (chunks of 8 blocks, one mbarrier each) while the others load
//      the query table (complemented for dot: 255 - D is the byte
//      complement, so the lookups give s' = 255*M - S directly);
//   2. each warp scans blocks as their chunk lands, writes the 8 sums of each
//      lane as keys s' (s' = S for L2, 255*M - S for dot; 0xFFFF for padding
//      vectors) to a shared array in vector order, and counts them in a
//      4,096-bin histogram of s' >> hshift;
//   3. the exact k-th smallest s' (T) and the number below it (c_lt) come
//      from the histogram (plus a second count inside T's bin when bins are
//      wider than 1); the CTA adds the per-bin counts of the keys it keeps to
//      the query's global histogram (one atomic per non-empty bin);
//   4. every entry with s' <= T is appended (in any order) and ranked: the k
//      smallest keys (s' << 32 | index) are every s' < T and the lowest
//      indices with s' == T, the CTA's exact top-k, published to its slot of
//      a global list sorted by key.  With more than 64 surplus entries equal
//      to T an ordered compaction keeps the first ones in vector order
//      instead.
// The last CTA to finish (atomic ticket) reads the first 16 keys of every
// list.  If no list longer than 16 has its 16th key at or below the k-th
// smallest s' of these prefixes, the k smallest prefix keys are the answer.
// Otherwise it reads the global histogram, which gives the k-th smallest s'
// of the union of the lists and the number of keys below it; every list then
// contributes a prefix (binary search), the ties at the threshold taken in
// vector order (CTA ranges are ordered).  The k survivors are sorted and
// written.
#include "topk.cuh"

#include "scan_core.cuh"

namespace bolt {

// phase stamps (diagnostic builds): 0 start, 1 scan done, 2 k-th bin, 3 kept,
// 4 sorted list, 5 ticket; the last CTA: 6 loaded, 7 pool bound, 8 prefixes
// checked, 9 gathered, 10 sorted, 11 end; 13: fast keep, 14: fast merge
BOLT_STAMP_ARRAY(g_stamps_small);
constexpr int kSmallThreads = 512;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int kSmallChunk = 8;  // blocks per bulk copy
constexpr uint64_t kSmallWait = 1000000000ull;  // 1 s bound on every mbarrier wait
constexpr int kSmallMiscWords = 64;
constexpr uint32_t kPad = 0xFFFFu;  // s' of padding vectors (every real s' <= 255 * 256)
constexpr int kSmallPrefix = 16;     // keys per list the merge reads first

// Exclusive block-wide prefix sum of one value per thread (T = 512).
// wsum: kSmallWarps + 1 words of shared scratch.  Returns the prefix and the
// total; ends with a barrier so wsum may be reused at once.
__device__ __forceinline__ uint32_t small_scan(uint32_t v, uint32_t *wsum, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t x = lane < kSmallWarps ? wsum[lane] : 0u;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, x, off);
            if (lane >= off) x += t;
        }
        if (lane < kSmallWarps) wsum[lane] = x;  // inclusive warp totals
    }
    __syncthreads();
    const uint32_t before = warp > 0 ? wsum[warp - 1] : 0u;
    total = wsum[kSmallWarps - 1];
    __syncthreads();
    return before + incl - v;
}

// Smallest bin b of hist[0..kBins) with (#entries in bins < b) < kk <= (#in
// bins <= b); returns b and sets below = #entries in bins < b.  kk >= 1 and
// kk <= total are required.
__device__ __forceinline__ uint32_t small_find(const uint32_t *hist, uint32_t kk, uint32_t *misc, uint32_t *wsum,
                                               uint32_t &below) {
    constexpr int BPT = kBins / kSmallThreads;  // 8: two 16-byte loads per thread
    static_assert(BPT == 8, "bins per thread");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint4 a = reinterpret_cast<const uint4 *>(hist)[2 * tid], b = reinterpret_cast<const uint4 *>(hist)[2 * tid + 1];
    const uint32_t v[BPT] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t local = 0;
#pragma unroll
    for (int i = 0; i < BPT; ++i) local += v[i];
    uint32_t incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t excl = incl - local;
    for (int w = 0; w < warp; ++w) excl += wsum[w];
    if (excl < kk && kk <= excl + local) {
        uint32_t c = excl;
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            if (c < kk && kk <= c + v[i]) {
                misc[0] = (uint32_t)(tid * BPT + i);
                misc[1] = c;
            }
            c += v[i];
        }
    }
    __syncthreads();
    below = misc[1];
    const uint32_t bin = misc[0];
    __syncthreads();
    return bin;
}

// Ordered compaction: entry e (vector order) is kept if s' < T, or s' == T
// and fewer than r entries with s' == T precede it; emit(pos, e) receives its
// rank among the kept entries (so kept entries stay in vector order).
template <typename F, typename E>
__device__ __forceinline__ void small_keep(int L, uint32_t T, uint32_t r, F s, E emit, uint32_t *wsum) {
    const int tid = threadIdx.x;
    const int seg = (L + kSmallThreads - 1) / kSmallThreads;
    const int e0 = min(L, tid * seg), e1 = min(L, e0 + seg);
    uint32_t lt = 0, eq = 0;
    for (int e = e0; e < e1; ++e) {
        const uint32_t v = s(e);
        lt += v < T ? 1u : 0u;
        eq += v == T ? 1u : 0u;
    }
    uint32_t tl, te;
    uint32_t lt_before = small_scan(lt, wsum, tl);
    uint32_t eq_before = small_scan(eq, wsum, te);
    for (int e = e0; e < e1; ++e) {
        const uint32_t v = s(e);
        if (v < T) {
            emit(lt_before + min(eq_before, r), e);
            ++lt_before;
        } else if (v == T) {
            if (eq_before < r) emit(lt_before + eq_before, e);
            ++eq_before;
        }
    }
    __syncthreads();
}

// Of the n distinct keys of src (shared memory), writes those of rank < nout
// to dst[rank] as expand(key) (increasing order): each key's rank is the
// number of smaller keys, counted by P adjacent threads per key.
template <typename K, typename X>
__device__ __forceinline__ void small_rank_sort(const K *src, int n, uint64_t *dst, int nout, X expand) {
    const int tid = threadIdx.x;
    int P = 1;
    while (P < 32 && n * P * 2 <= kSmallThreads) P <<= 1;
    const int part = tid & (P - 1);
    for (int base = 0; base < n; base += kSmallThreads / P) {
        const int e = base + tid / P;
        const K key = e < n ? src[e] : K(0);
        int r0 = 0, r1 = 0, r2 = 0, r3 = 0;
        if (e < n) {
            int j = part;
            for (; j + 3 * P < n; j += 4 * P) {
                r0 += src[j] < key ? 1 : 0;
                r1 += src[j + P] < key ? 1 : 0;
                r2 += src[j + 2 * P] < key ? 1 : 0;
                r3 += src[j + 3 * P] < key ? 1 : 0;
            }
            for (; j < n; j += P) r0 += src[j] < key ? 1 : 0;
        }
        int rank = r0 + r1 + r2 + r3;
        for (int o = 1; o < P; o <<= 1) rank += __shfl_xor_sync(0xFFFFFFFFu, rank, o);
        if (e < n && part == 0 && rank < nout) dst[rank] = expand(key);
    }
}

__device__ __forceinline__ void small_rank_sort(const uint64_t *src, int n, uint64_t *dst, int nout) {
    small_rank_sort(src, n, dst, nout, [](uint64_t key) { return key; });
}

// Entries e < L of the CTA's sums (uint16 in vector order, padding 0xFFFF)
// with s' <= T, as 32-bit keys (s' << 16 | e) in any order: one count pass
// over 16-byte chunks, a prefix over threads, one writing pass.  L is a
// multiple of 8 and at most 65536.  wsum: kSmallWarps words.
__device__ __forceinline__ void small_keep_le(const uint16_t *sums, int L, uint32_t T, uint32_t *dst,
                                              uint32_t *wsum) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(sums);
    const int nc = L >> 3;
    uint32_t cnt = 0;
    for (int c = tid; c < nc; c += kSmallThreads) {
        const uint4 w = s4[c];
        const uint32_t x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) cnt += ((x[i] & 0xFFFFu) <= T ? 1u : 0u) + ((x[i] >> 16) <= T ? 1u : 0u);
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t pos = incl - cnt;
    for (int w = 0; w < warp; ++w) pos += wsum[w];
    for (int c = tid; c < nc; c += kSmallThreads) {
        const uint4 w = s4[c];
        const uint32_t x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t lo = x[i] & 0xFFFFu, hi = x[i] >> 16, e = (uint32_t)c * 8u + 2u * i;
            if (lo <= T) dst[pos++] = (lo << 16) | e;
            if (hi <= T) dst[pos++] = (hi << 16) | (e + 1u);
        }
    }
    __syncthreads();
}

// Appends key(e) for every e in [0, L) with pred(e), in any order, to
// dst[0..): a counting pass of warp ballots, a prefix over the warps'
// counts, then a writing pass (no shared atomics).  L is a multiple of 256,
// so every ballot covers a whole warp.  wsum: kSmallWarps + 1 words.
template <typename Pr, typename Ky>
__device__ __forceinline__ void small_append(int L, Pr pred, Ky key, uint64_t *dst, uint32_t *wsum) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t cnt = 0;
    for (int e = tid; e < L; e += kSmallThreads) cnt += __popc(__ballot_sync(0xFFFFFFFFu, pred(e)));
    if (lane == 0) wsum[warp] = cnt;
    __syncthreads();
    uint32_t pos = 0;
    for (int w = 0; w < warp; ++w) pos += wsum[w];
    const uint32_t below = (1u << lane) - 1u;
    for (int e = tid; e < L; e += kSmallThreads) {
        const bool keep = pred(e);
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        if (keep) dst[pos + __popc(bal & below)] = key(e);
        pos += __popc(bal);
    }
    __syncthreads();
}

// Ascending bitonic sort of keys[0..P), P a power of two.
__device__ __forceinline__ void small_bitonic(uint64_t *keys, int P) {
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += kSmallThreads) {
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

__host__ __device__ constexpr size_t small_align_dev(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct SmallWS {
    uint32_t *ticket;  // [nq]
    uint32_t *status;  // [nq] bit 0: a bounded wait gave up
    uint32_t *ghist;   // [nq][kBins] histogram of s' >> hshift over every CTA's kept keys
    uint32_t *cnt;     // [nq][G] entries in each CTA's list
    uint64_t *keys;    // [nq][G][k rounded up to even] (s' << 32 | index), sorted within a list
};

template <int MT>
__global__ void __launch_bounds__(kSmallThreads, 2)
    topk_small_kernel(const uint32_t *__restrict__ codes, int64_t n, int32_t M, const uint8_t *__restrict__ luts,
                      int32_t k, int32_t metric, SmallWS ws, int nbc, int hshift,
                      uint16_t *__restrict__ out_sums, int64_t *__restrict__ out_idx) {
    extern __shared__ __align__(128) uint8_t smem[];
    if (MT > 0) M = MT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q = blockIdx.y;
    const int G = gridDim.x, cta = blockIdx.x;
    BOLT_STAMP(g_stamps_small, q, cta, 0);

    uint8_t *p = smem;
    uint32_t *hist = reinterpret_cast<uint32_t *>(p);
    p += kBins * 4;
    // misc: [0..2) find results, [2] failure bits, [3] last CTA, [5] merge:
    // total list entries, [6] merge: a list may hold more winners than its
    // prefix, [7] merge: prefix keys, [8..) scan scratch
    uint32_t *misc = reinterpret_cast<uint32_t *>(p);
    uint32_t *wsum = misc + 8;
    p += kSmallMiscWords * 4;
    uint4 *lut = reinterpret_cast<uint4 *>(p);
    p += (size_t)M * 16;
    uint64_t *bars = reinterpret_cast<uint64_t *>(p);
    const int nch = (nbc + kSmallChunk - 1) / kSmallChunk;
    p += (size_t)((nch + 2) / 2 * 2) * 8;  // one barrier per chunk
    uint8_t *region = p;  // codes + sums during the scan; keys during the merge
    const uint32_t blk_bytes = (uint32_t)M * kRowBytes;
    uint32_t *codes_s = reinterpret_cast<uint32_t *>(region);
    uint16_t *sums_s = reinterpret_cast<uint16_t *>(region + (size_t)nbc * blk_bytes);

    const int64_t nb = num_blocks(n);
    const int64_t b0 = (int64_t)cta * nbc;
    const int nblk = (int)min((int64_t)nbc, nb - b0);  // >= 1 (grid = ceil(nb / nbc))
    const int nchunks = (nblk + kSmallChunk - 1) / kSmallChunk;

    if (tid == 0) {
        for (int c = 0; c < nchunks; ++c) mbar_init(&bars[c], 1);
        fence_mbar_init();
        misc[2] = 0;
        misc[5] = 0;
        misc[6] = 0;
        misc[7] = 0;
        for (int c = 0; c < nchunks; ++c) {
            const int nbk = min(kSmallChunk, nblk - c * kSmallChunk);
            const uint32_t bytes = (uint32_t)nbk * blk_bytes;
            mbar_arrive_expect_tx(&bars[c], bytes);
            bulk_g2s(region + (size_t)c * kSmallChunk * blk_bytes,
                     codes + (size_t)(b0 + (int64_t)c * kSmallChunk) * M * kRowWords, bytes, &bars[c]);
        }
    }
    for (int i = tid; i < kBins; i += kSmallThreads) hist[i] = 0;
    // For dot the tables are complemented (255 - D is the byte complement),
    // so the lookups produce s' = 255*M - S directly.
    const uint4 *lut_g = reinterpret_cast<const uint4 *>(luts + q * M * kK);
    const uint32_t lut_x = metric == BOLT_METRIC_DOT ? 0xFFFFFFFFu : 0u;
    for (int i = tid; i < M; i += kSmallThreads) {
        const uint4 t = lut_g[i];
        lut[i] = make_uint4(t.x ^ lut_x, t.y ^ lut_x, t.z ^ lut_x, t.w ^ lut_x);
    }
    __syncthreads();

    const uint32_t smax = 255u * (uint32_t)M;
    bool failed = false;
    for (int blk = warp; blk < nblk; blk += kSmallWarps) {
        // (a completed chunk's barrier answers at once)
        const bool ok = mbar_wait_bounded(&bars[blk / kSmallChunk], 0u, kSmallWait);
        if (!__all_sync(0xFFFFFFFFu, ok)) {
            failed = true;
            break;
        }
        const uint32_t *words = codes_s + (size_t)blk * M * kRowWords;
        Acc8 acc;
        acc.zero();
        if (MT > 0) {
#pragma unroll
            for (int m = 0; m < MT; ++m) acc.add(prep_word(words[m * kRowWords + lane]), lut[m]);
        } else {
#pragma unroll 4
            for (int m = 0; m < M; ++m) acc.add(prep_word(words[m * kRowWords + lane]), lut[m]);
        }
        uint32_t e_lo, o_lo, e_hi, o_hi;
        acc.finish(e_lo, o_lo, e_hi, o_hi);
        const uint4 pk = pack_sums(e_lo, o_lo, e_hi, o_hi);
        const uint32_t w[4] = {pk.x, pk.y, pk.z, pk.w};
        const int64_t v0 = (b0 + blk) * kBlockVecs + 8 * lane;
        uint32_t out[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint32_t pair = 0;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int i = 2 * h + j;
                uint32_t sp = (w[h] >> (16 * j)) & 0xFFFFu;
                if (v0 + i >= n) sp = kPad;
                else atomicAdd(&hist[sp >> hshift], 1u);
                pair |= sp << (16 * j);
            }
            out[h] = pair;
        }
        *reinterpret_cast<uint4 *>(sums_s + (size_t)blk * kBlockVecs + 8 * lane) =
            make_uint4(out[0], out[1], out[2], out[3]);
    }
    if (failed && lane == 0) atomicOr(&misc[2], 1u);
    __syncthreads();
    BOLT_STAMP(g_stamps_small, q, cta, 1);
    const bool bad = misc[2] != 0u;
    if (bad) {
        // let copies still in flight land before shared memory is reused
        if (tid == 0)
            for (int c = 0; c < nchunks; ++c) mbar_wait_bounded(&bars[c], 0u, kSmallWait / 10);
        __syncthreads();
    }

    // ---- this CTA's exact top-k, published sorted by (s', index)
    const int L = nblk * kBlockVecs;
    const int64_t nvalid = min((int64_t)L, n - b0 * kBlockVecs);
    const uint32_t kk = (uint32_t)min((int64_t)k, nvalid);
    auto s_of = [&](int e) -> uint32_t { return sums_s[e]; };
    const int kslot = k + (k & 1);  // even: every list starts 16-byte aligned
    const int64_t qstride = (int64_t)G * kslot;
    uint64_t *mine = ws.keys + q * qstride + (int64_t)cta * kslot;
    uint64_t *kept = reinterpret_cast<uint64_t *>(
        region + small_align_dev((size_t)nbc * blk_bytes + (size_t)nbc * kBlockVecs * 2, 16));
    if (!bad) {
        uint32_t below;
        const uint32_t B = small_find(hist, kk, misc, wsum, below);
        // The query's global histogram counts every CTA's kept keys: all of
        // bins < B, and kk - below of bin B (read by the merge's exact path).
        uint32_t *gh = ws.ghist + q * kBins;
        for (int b = tid; b <= (int)B; b += kSmallThreads) {
            const uint32_t c = b < (int)B ? hist[b] : kk - below;
            if (c) atomicAdd(&gh[b], c);
        }
        uint32_t T = B, c_lt = below;
        if (hshift > 0) {  // exact value inside bin B
            __syncthreads();
            for (int i = tid; i < kBins; i += kSmallThreads) hist[i] = 0;
            __syncthreads();
            const uint32_t mask = (1u << hshift) - 1u;
            for (int e = tid; e < L; e += kSmallThreads) {
                const uint32_t v = sums_s[e];
                if (v != kPad && (v >> hshift) == B) atomicAdd(&hist[v & mask], 1u);
            }
            __syncthreads();
            uint32_t below2;
            const uint32_t f = small_find(hist, kk - below, misc, wsum, below2);
            T = (B << hshift) | f;
            c_lt = below + below2;
        }
        const int64_t base = b0 * kBlockVecs;
        BOLT_STAMP(g_stamps_small, q, cta, 2);
        // entries equal to T (the histogram still holds their count)
        const uint32_t n_le = c_lt + hist[hshift > 0 ? (T & ((1u << hshift) - 1u)) : T];
        // the code area is free now: room for nbc * M * 32 keys of 32 bits
        const uint32_t cap_le = min((uint32_t)nbc * (uint32_t)M * 32u, kk + 64u);
        if (n_le <= cap_le && L <= 65536) {
            // every entry with s' <= T (padding has s' = 0xFFFF > T) in any
            // order as (s' << 16 | e); the rank sort keeps the kk smallest
            // keys, which are the entries below T and the lowest indices
            // among those equal to T
            uint32_t *le = reinterpret_cast<uint32_t *>(region);
            small_keep_le(sums_s, L, T, le, wsum);
            BOLT_STAMP(g_stamps_small, q, cta, 3);
            BOLT_STAMP_VALUE(g_stamps_small, q, cta, 13, 1);
            small_rank_sort(le, (int)n_le, mine, (int)kk, [&](uint32_t key) {
                return ((uint64_t)(key >> 16) << 32) | (uint64_t)(base + (int64_t)(key & 0xFFFFu));
            });
        } else {
            // many entries equal to T: ordered compaction (lowest indices first)
            small_keep(L, T, kk - c_lt, s_of,
                       [&](uint32_t pos, int e) { kept[pos] = ((uint64_t)sums_s[e] << 32) | (uint64_t)(base + e); },
                       wsum);
            BOLT_STAMP(g_stamps_small, q, cta, 3);
            small_rank_sort(kept, (int)kk, mine, (int)kk);
        }
        BOLT_STAMP(g_stamps_small, q, cta, 4);
    }
    if (tid == 0) {
        ws.cnt[q * G + cta] = bad ? 0u : kk;
        if (bad) atomicOr(&ws.status[q], 1u);
    }
    __threadfence();
    __syncthreads();
    BOLT_STAMP(g_stamps_small, q, cta, 5);
    if (tid == 0) misc[3] = (atomicAdd(&ws.ticket[q], 1u) == (uint32_t)(G - 1)) ? 1u : 0u;
    __syncthreads();
    if (misc[3] == 0) return;
    __threadfence();

    // ---- last CTA: merge the G sorted lists.  Fast path: the first kp keys
    // of every list form a pool; its kout-th smallest s' is T*.  When every
    // list longer than kp has its kp-th key above T*, no key past a prefix
    // can be among the kout smallest (lists are sorted), so the pool's kout
    // smallest keys are the answer.  Otherwise (a list holds more winners
    // than its prefix) the exact path: the global histogram gives the kout-th
    // smallest s' of the union (T2) and the number below it (c2); each list
    // contributes a prefix found by binary search, ties at T2 taken in
    // vector order (lists are in CTA order = vector order).
    const int kp = min(k, kSmallPrefix) + (min(k, kSmallPrefix) & 1);
    uint32_t *cnt_s = reinterpret_cast<uint32_t *>(region);  // [G] counts; then keys below T2
    uint32_t *lt_s = cnt_s + G;                              // [G] offsets of the keys below T2
    uint32_t *eq_s = lt_s + G;                               // [G] offsets of the keys equal to T2
    // [G][kSmallPrefix]: the first kp keys of every list
    uint64_t *pre = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(region) + (size_t)G * 12 + 127) &
                                                 ~uintptr_t(127));
    uint64_t *fin = pre + (size_t)G * kSmallPrefix;
    constexpr int kPs = 4;  // log2(kSmallPrefix)
    static_assert(kSmallPrefix == 1 << kPs, "prefix stride");
    // pool entry e: key j = e mod 16 of list c = e / 16, valid while j is
    // below the list's length (which is at most kp when kp < 16)
    auto in_pool = [&](int e) { return (uint32_t)(e & (kSmallPrefix - 1)) < cnt_s[e >> kPs]; };
    int P = 1;
    while (P < k) P <<= 1;
    const uint64_t *lists = ws.keys + q * qstride;
    {
        // list lengths (G <= kSmallThreads: one per thread), their total and
        // the prefix keys' count: warp sums, then one shared add per warp
        const uint32_t v = tid < G ? __ldcg(ws.cnt + q * G + tid) : 0u;
        if (tid < G) cnt_s[tid] = v;
        uint32_t tv = v, tp = min(v, (uint32_t)kp);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tv += __shfl_xor_sync(0xFFFFFFFFu, tv, o);
            tp += __shfl_xor_sync(0xFFFFFFFFu, tp, o);
        }
        if (lane == 0 && tv) {
            atomicAdd(&misc[5], tv);
            atomicAdd(&misc[7], tp);
        }
    }
    {
        // G * kSmallPrefix <= 256 * 16 slots: at most 8 per thread, all loads
        // in flight at once (entries past a list's count are unused)
        constexpr int kPerThread = 256 * kSmallPrefix / kSmallThreads;
        uint64_t pv[kPerThread];
#pragma unroll
        for (int i = 0; i < kPerThread; ++i) {
            const int e = tid + i * kSmallThreads, c = e >> kPs, j = e & (kSmallPrefix - 1);
            pv[i] = c < G && j < kp ? __ldcg(lists + (int64_t)c * kslot + j) : 0ull;
        }
#pragma unroll
        for (int i = 0; i < kPerThread; ++i) {
            const int e = tid + i * kSmallThreads;
            if (e < G * kSmallPrefix) pre[e] = pv[i];
        }
    }
    if (tid == 0 && __ldcg(&ws.status[q]) != 0u) atomicOr(&misc[2], 4u);
    for (int i = tid; i < kBins; i += kSmallThreads) hist[i] = 0;
    __syncthreads();
    const bool qbad = (misc[2] & 4u) != 0u;
    BOLT_STAMP(g_stamps_small, q, cta, 6);
    const uint32_t total = misc[5];
    const int kout = qbad ? 0 : (int)min((uint32_t)k, total);
    bool sorted_done = false;
    if (kout > 0) {
        bool fast = misc[7] >= (uint32_t)kout;
        uint32_t Tst = 0, n_le = 0;
        if (fast) {
            for (int e = tid; e < G * kSmallPrefix; e += kSmallThreads)
                if (in_pool(e)) atomicAdd(&hist[(uint32_t)(pre[e] >> 32) >> hshift], 1u);
            __syncthreads();
            uint32_t below;
            const uint32_t B = small_find(hist, (uint32_t)kout, misc, wsum, below);
            Tst = B;
            n_le = below + hist[B];
            BOLT_STAMP(g_stamps_small, q, cta, 7);
            if (hshift > 0) {  // exact value inside bin B
                const uint32_t mask = (1u << hshift) - 1u;
                for (int i = tid; i < kBins; i += kSmallThreads) hist[i] = 0;
                __syncthreads();
                for (int e = tid; e < G * kSmallPrefix; e += kSmallThreads) {
                    const uint32_t v = (uint32_t)(pre[e] >> 32);
                    if (in_pool(e) && (v >> hshift) == B) atomicAdd(&hist[v & mask], 1u);
                }
                __syncthreads();
                uint32_t below2;
                const uint32_t f = small_find(hist, (uint32_t)kout - below, misc, wsum, below2);
                Tst = (B << hshift) | f;
                n_le = below + below2 + hist[f];
            }
            for (int c = tid; c < G; c += kSmallThreads)
                if (cnt_s[c] > (uint32_t)kp && (uint32_t)(pre[(size_t)c * kSmallPrefix + kp - 1] >> 32) <= Tst)
                    atomicOr(&misc[6], 1u);
            __syncthreads();
            fast = misc[6] == 0u && n_le <= (uint32_t)P;
            BOLT_STAMP(g_stamps_small, q, cta, 8);
            BOLT_STAMP_VALUE(g_stamps_small, q, cta, 14, fast ? 1 : 0);
        }
        if (fast) {
            // the pool's keys with s' <= T* (n_le of them), then the kout smallest
            const int npool = (G * kSmallPrefix + 255) / 256 * 256;
            small_append(
                npool,
                [&](int e) { return e < G * kSmallPrefix && in_pool(e) && (uint32_t)(pre[e] >> 32) <= Tst; },
                [&](int e) { return pre[e]; }, fin, wsum);
            BOLT_STAMP(g_stamps_small, q, cta, 9);
            if (kout <= 256) {
                small_rank_sort(fin, (int)n_le, fin + P, kout);
                __syncthreads();
                fin += P;
            } else {
                for (int i = (int)n_le + tid; i < P; i += kSmallThreads) fin[i] = ~0ull;
                __syncthreads();
                small_bitonic(fin, P);
            }
            sorted_done = true;
        } else {
            // exact path: the global histogram of every list's keys
            for (int i = tid; i < kBins; i += kSmallThreads) hist[i] = __ldcg(ws.ghist + q * kBins + i);
            __syncthreads();
            auto key_at = [&](int c, uint32_t j) -> uint64_t {
                return j < (uint32_t)kp ? pre[(size_t)c * kSmallPrefix + j] : __ldcg(lists + (int64_t)c * kslot + j);
            };
            // first position in list c whose s' >> sh is >= v (binary search; past
            // the prefix only when the prefix's last key is below v)
            auto lower = [&](int c, uint32_t v, int sh) -> uint32_t {
                const uint32_t len = cnt_s[c];
                uint32_t lo = 0, hi = min(len, (uint32_t)kp);
                if (hi == (uint32_t)kp && hi < len &&
                    ((uint32_t)(pre[(size_t)c * kSmallPrefix + kp - 1] >> 32) >> sh) < v) {
                    lo = hi;
                    hi = len;
                }
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (((uint32_t)(key_at(c, mid) >> 32) >> sh) < v) lo = mid + 1;
                    else hi = mid;
                }
                return lo;
            };
            uint32_t below;
            const uint32_t B2 = small_find(hist, (uint32_t)kout, misc, wsum, below);
            uint32_t T2 = B2, c2 = below;
            if (hshift > 0) {  // exact value inside bin B2: count the bin's keys by value
                const uint32_t mask = (1u << hshift) - 1u;
                for (int i = tid; i < kBins; i += kSmallThreads) hist[i] = 0;
                __syncthreads();
                for (int c = warp; c < G; c += kSmallWarps) {
                    const uint32_t lo = lower(c, B2, hshift), hi = lower(c, B2 + 1, hshift);
                    for (uint32_t j = lo + lane; j < hi; j += 32)
                        atomicAdd(&hist[(uint32_t)(key_at(c, j) >> 32) & mask], 1u);
                }
                __syncthreads();
                uint32_t below2;
                const uint32_t f = small_find(hist, (uint32_t)kout - below, misc, wsum, below2);
                T2 = (B2 << hshift) | f;
                c2 = below + below2;
            }
            const uint32_t r = (uint32_t)kout - c2;  // keys equal to T2 to keep, lowest index first
            uint32_t lt = 0, eq = 0;
            if (tid < G) {
                lt = lower(tid, T2, 0);
                eq = lower(tid, T2 + 1, 0) - lt;
            }
            uint32_t t1, t2;
            const uint32_t lt_off = small_scan(lt, wsum, t1);
            const uint32_t eq_off = small_scan(eq, wsum, t2);
            if (tid < G) {
                cnt_s[tid] = lt;  // the list's keys below T2 (its length is no longer needed)
                lt_s[tid] = lt_off;
                eq_s[tid] = eq_off;
            }
            __syncthreads();
            for (int c = warp; c < G; c += kSmallWarps) {
                const uint32_t nlt = cnt_s[c], lo = lt_s[c], eo = eq_s[c];
                const uint32_t neq = eo < r ? min(r - eo, (c + 1 < G ? eq_s[c + 1] : t2) - eo) : 0u;
                for (uint32_t j = lane; j < nlt; j += 32) fin[lo + j] = key_at(c, j);
                for (uint32_t j = lane; j < neq; j += 32) fin[c2 + eo + j] = key_at(c, nlt + j);
            }
            __syncthreads();
        }
    }
    if (kout > 0 && !sorted_done) {
        // order the kout survivors of the exact path by (s', index)
        if (kout <= 256) {
            small_rank_sort(fin, kout, fin + P, kout);
            __syncthreads();
            fin += P;
        } else {
            for (int i = kout + tid; i < P; i += kSmallThreads) fin[i] = ~0ull;
            __syncthreads();
            small_bitonic(fin, P);
        }
    }
    BOLT_STAMP(g_stamps_small, q, cta, 10);
    for (int r = tid; r < k; r += kSmallThreads) {
        if (r < kout) {
            const uint32_t sp = (uint32_t)(fin[r] >> 32);
            out_sums[q * k + r] = (uint16_t)(metric == BOLT_METRIC_DOT ? smax - sp : sp);
            out_idx[q * k + r] = qbad ? -2 : (int64_t)(uint32_t)fin[r];
        } else {
            out_sums[q * k + r] = 0;
            out_idx[q * k + r] = qbad ? -2 : -1;
        }
    }
    BOLT_STAMP(g_stamps_small, q, cta, 11);
}

#ifdef BOLT_PHASE_STAMPS
}  // namespace bolt
// Copies the shared-memory kernel's stamps (1024 CTAs x 16 slots) to host
// and, with clear != 0, zeroes them (diagnostic builds only).
extern "C" int bolt_debug_stamps_small(unsigned long long *host, int clear) {
    if (cudaMemcpyFromSymbol(host, bolt::g_stamps_small, sizeof(unsigned long long) * 1024 * 16) != cudaSuccess)
        return BOLT_ECUDA;
    if (clear) {
        static unsigned long long zero[1024 * 16];
        if (cudaMemcpyToSymbol(bolt::g_stamps_small, zero, sizeof(zero)) != cudaSuccess) return BOLT_ECUDA;
    }
    return BOLT_OK;
}
namespace bolt {
#endif

// ------------------------------------------------------------------ host side
static size_t small_align(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Fills the small-path fields of plan if this size class applies.
bool plan_topk_small(int64_t n, int32_t M, int32_t k, int sms, TopkPlan *plan, int64_t max_ctas) {
    const int64_t nb = num_blocks(n);
    if (nb == 0 || sms <= 0 || k > kMaxSmallK) return false;
    int64_t G = sms;
    if (max_ctas > 0 && G > max_ctas) G = max_ctas;
    if (G > nb) G = nb;
    if (G > kSmallMergeKeys / k) G = kSmallMergeKeys / k;
    if (G > 256) G = 256;  // the merge's exact path takes one list per thread
    if (G < 1) return false;
    const int64_t nbc = (nb + G - 1) / G;
    G = (nb + nbc - 1) / nbc;  // every CTA gets at least one block
    int P = 1;
    while (P < k) P <<= 1;
    const int nch = (int)((nbc + kSmallChunk - 1) / kSmallChunk);
    const size_t scan_region = small_align((size_t)nbc * M * kRowBytes + (size_t)nbc * kBlockVecs * 2, 16) +
                               (size_t)k * 8;
    const size_t merge_region = (size_t)G * 12 + 128 + (size_t)G * kSmallPrefix * 8 + (size_t)2 * P * 8;
    const size_t region = scan_region > merge_region ? scan_region : merge_region;
    const size_t smem = (size_t)kBins * 4 + kSmallMiscWords * 4 + small_align((size_t)M * 16, 16) +
                        (size_t)((nch + 2) / 2 * 2) * 8 + region;
    if (smem > kSmallMaxSmem) return false;
    int hshift = 0;
    while (((255 * M) >> hshift) >= kBins) ++hshift;
    plan->small = 1;
    plan->grid = (int)G;
    plan->nbc = (int)nbc;
    plan->hshift = hshift;
    plan->smem_bytes = smem;
    return true;
}

// ticket, status and histograms: zeroed before every launch
static size_t topk_small_header_bytes(int64_t nq) {
    return small_align((size_t)nq * 8, 256) + (size_t)nq * kBins * 4;
}

int64_t topk_small_workspace_bytes(const TopkPlan &plan, int64_t nq, int32_t k) {
    const size_t qstride = (size_t)plan.grid * (size_t)(k + (k & 1));
    return (int64_t)(topk_small_header_bytes(nq) + small_align((size_t)nq * plan.grid * 4, 256) +
                     (size_t)nq * qstride * 8);
}

template <int MT>
static int launch_small_w(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                          int32_t metric, uint16_t *out_sums, int64_t *out_idx, const SmallWS &w,
                          const TopkPlan &plan, cudaStream_t stream) {
    auto kern = topk_small_kernel<MT>;
    int rc = ensure_smem((const void *)kern, plan.smem_bytes);
    if (rc) return rc;
    dim3 grid(plan.grid, (unsigned)nq);
    kern<<<grid, kSmallThreads, plan.smem_bytes, stream>>>(reinterpret_cast<const uint32_t *>(codes), n, M, luts, k,
                                                            metric, w, plan.nbc, plan.hshift, out_sums, out_idx);
    return check_launch("topk_small_kernel");
}

int launch_topk_small(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                      int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, const TopkPlan &plan,
                      cudaStream_t stream) {
    BOLT_REQUIRE(nq <= 65535, BOLT_EUNSUPPORTED, "nq=%lld > 65535 per call", (long long)nq);
    BOLT_CUDA(cudaMemsetAsync(workspace, 0, topk_small_header_bytes(nq), stream));
    uint8_t *p = static_cast<uint8_t *>(workspace);
    SmallWS w;
    w.ticket = reinterpret_cast<uint32_t *>(p);
    w.status = w.ticket + nq;
    w.ghist = reinterpret_cast<uint32_t *>(p + small_align((size_t)nq * 8, 256));
    p += topk_small_header_bytes(nq);
    w.cnt = reinterpret_cast<uint32_t *>(p);
    p += small_align((size_t)nq * plan.grid * 4, 256);
    w.keys = reinterpret_cast<uint64_t *>(p);
#define BOLT_SMALL_ARGS codes, n, M, luts, nq, k, metric, out_sums, out_idx, w, plan, stream
    if (M == 8) return launch_small_w<8>(BOLT_SMALL_ARGS);
    if (M == 16) return launch_small_w<16>(BOLT_SMALL_ARGS);
    if (M == 32) return launch_small_w<32>(BOLT_SMALL_ARGS);
    return launch_small_w<0>(BOLT_SMALL_ARGS);
#undef BOLT_SMALL_ARGS
}

}  // namespace bolt
