// Fused Bolt scan + exact top-k (nearest neighbours for L2 sums, maximum
// inner product for dot sums; Sec. 1.2 motivates both searches).
//
// Keys.  A candidate is the 64-bit key (s' << 32 | index) with s' = S for L2
// and s' = 0xFFFF - S for dot, so "smaller key" is "better" for both metrics
// and equal sums break ties toward the lower index.
//
// Work split.  Each query is handled by `grid` CTAs, one contiguous range of
// 256-vector code blocks per CTA.  A CTA processes its blocks in rounds: in
// round r warp w takes block lo + r*WARPS + w, so every block of round r+1
// has larger indices than every block of rounds <= r.  Each warp streams its
// blocks through a private ring of shared-memory stages filled by 1-D TMA
// bulk copies (non-multicast) completing on an mbarrier.
//
// Candidates.  Lanes append sums below the CTA's threshold s_thr to a
// shared buffer.  When the buffer runs full the CTA finds s* = the k-th
// smallest s' (two 8-bit histogram passes), keeps every entry with s' <= s*
// and sets s_thr = s*: later blocks only hold larger indices, so an equal
// sum can no longer enter the top k.  The CTA then publishes s* to a
// per-query global bound (some CTA holds k entries <= s*), which every CTA
// uses to reject s' > s*.
//
// Merge.  Each CTA writes its exact top k; the last CTA to finish (atomic
// ticket) loads all lists into shared memory, selects the exact k smallest
// keys, sorts them and writes the result.
#include "scan_core.cuh"
#include "topk.cuh"

namespace bolt {

constexpr uint64_t kWaitLimit = 1000000000ull;  // 1 s bound on any mbarrier wait
constexpr int kMaxStages = 8;
constexpr size_t kStageBudget = 128 * 1024;
constexpr int kMaxK = 1024;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------------------------ block-wide selection
template <int T>
struct BlockSel {
    uint32_t *hist;  // 256 counters
    uint32_t *res;   // [0] digit, [1] count below digit, [2..2+T/32) warp counts

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
                const uint64_t key = keys[i];
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

    // Stable in-place compaction keeping keys <= bound; returns the new count.
    __device__ int keep_le(uint64_t *keys, int cnt, uint64_t bound) {
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        uint32_t *wcnt = res + 2;
        int out = 0;
        for (int base = 0; base < cnt; base += T) {
            const int i = base + tid;
            const uint64_t key = i < cnt ? keys[i] : ~0ull;
            const bool keep = i < cnt && key <= bound;
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
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1)
    topk_kernel(const uint32_t *__restrict__ codes, int64_t n, int32_t M, const uint8_t *__restrict__ luts,
                int32_t k, int32_t metric, TopkWS ws, int stages, int cap, int64_t blocks_per_cta,
                uint16_t *__restrict__ out_sums, int64_t *__restrict__ out_idx) {
    constexpr int T = WARPS * 32;
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q = blockIdx.y;
    const int G = gridDim.x, cta = blockIdx.x;
    const uint32_t stage_bytes = (uint32_t)M * kRowBytes;

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
    p += 256 * 4;
    uint32_t *misc = reinterpret_cast<uint32_t *>(p);  // [0] cnt [1] thr [2] flags [3] last [4..] sel scratch
    BlockSel<T> sel{hist, misc + 4};
    volatile uint32_t *vmisc = misc;

    const uint4 *lut_g = reinterpret_cast<const uint4 *>(luts + q * M * kK);
    for (int i = tid; i < M; i += T) lut[i] = lut_g[i];
    if (tid == 0) {
        misc[0] = 0;
        misc[1] = 0x10000u;  // insert iff s' < thr: everything passes
        misc[2] = 0;
        misc[3] = 0;
    }
    if (tid < WARPS * stages) mbar_init(&bars[tid], 1);
    fence_mbar_init();
    __syncthreads();

    const int64_t nb = num_blocks(n);
    const int64_t b_lo = (int64_t)cta * blocks_per_cta;
    const int64_t b_hi = min(nb, b_lo + blocks_per_cta);
    const int64_t nbc = b_hi > b_lo ? b_hi - b_lo : 0;
    const int64_t rounds = (nbc + WARPS - 1) / WARPS;
    uint64_t *mybars = bars + warp * stages;
    uint8_t *mystage = stage_base + (size_t)warp * stages * stage_bytes;

    // lane 0 of each warp is the producer of its ring
    uint32_t pending = 0;  // stages with a copy in flight (lane 0)
    uint32_t phase = 0;    // parity of the next completion of each stage (lane 0)
    if (lane == 0) {
        for (int s = 0; s < stages; ++s) {
            const int64_t b = b_lo + (int64_t)s * WARPS + warp;
            if (b < b_hi) {
                mbar_arrive_expect_tx(&mybars[s], stage_bytes);
                bulk_g2s(mystage + (size_t)s * stage_bytes, codes + b * M * kRowWords, stage_bytes, &mybars[s]);
                pending |= 1u << s;
            }
        }
    }

    bool failed = false;
    const uint32_t gate = (uint32_t)(cap - WARPS * kBlockVecs);  // compact above this count
    for (int64_t r = 0; r < rounds; ++r) {
        const int64_t b = b_lo + r * WARPS + warp;
        const int st = (int)(r % stages);
        const uint32_t par = (uint32_t)((r / stages) & 1);
        if (b < b_hi && !failed) {
            const bool ok = mbar_wait_bounded(&mybars[st], par, kWaitLimit);
            if (!__all_sync(0xFFFFFFFFu, ok)) {
                failed = true;
            } else {
                if (lane == 0) {
                    pending &= ~(1u << st);
                    phase ^= 1u << st;
                }
                const uint32_t *words = reinterpret_cast<const uint32_t *>(mystage + (size_t)st * stage_bytes);
                Acc8 acc;
                acc.zero();
#pragma unroll 4
                for (int m = 0; m < M; ++m) acc.add(prep_word(words[m * kRowWords + lane]), lut[m]);
                __syncwarp();
                if (lane == 0) {
                    const int64_t b2 = b + (int64_t)stages * WARPS;
                    if (b2 < b_hi) {
                        mbar_arrive_expect_tx(&mybars[st], stage_bytes);
                        bulk_g2s(mystage + (size_t)st * stage_bytes, codes + b2 * M * kRowWords, stage_bytes,
                                 &mybars[st]);
                        pending |= 1u << st;
                    }
                }
                uint32_t e_lo, o_lo, e_hi, o_hi;
                acc.finish(e_lo, o_lo, e_hi, o_hi);
                if (metric == BOLT_METRIC_DOT) {  // s' = 0xFFFF - S in each 16-bit lane
                    e_lo = ~e_lo;
                    o_lo = ~o_lo;
                    e_hi = ~e_hi;
                    o_hi = ~o_hi;
                }
                const uint32_t thr = vmisc[1];
                const uint32_t mn2 = __vminu2(__vminu2(e_lo, o_lo), __vminu2(e_hi, o_hi));
                const uint32_t mn = min(mn2 & 0xFFFFu, mn2 >> 16);
                const int64_t v0 = b * kBlockVecs + 8 * lane;
                const bool maybe = mn < thr && v0 < n;
                if (__any_sync(0xFFFFFFFFu, maybe)) {
                    const uint4 pk = pack_sums(e_lo, o_lo, e_hi, o_hi);
                    const uint32_t w4[4] = {pk.x, pk.y, pk.z, pk.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const uint32_t sp = (w4[i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
                        const bool pred = sp < thr && v0 + i < n;
                        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, pred);
                        if (bal) {
                            const int leader = __ffs(bal) - 1;
                            uint32_t base = 0;
                            if (lane == leader) base = atomicAdd(&misc[0], (uint32_t)__popc(bal));
                            base = __shfl_sync(0xFFFFFFFFu, base, leader);
                            if (pred)
                                keys[base + __popc(bal & lanemask_lt())] =
                                    ((uint64_t)sp << 32) | (uint64_t)(uint32_t)(v0 + i);
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (vmisc[0] > gate) {
            // Buffer full: keep every entry with s' <= s* (k-th smallest s').
            const int cnt = (int)vmisc[0];
            uint32_t n_less, n_eq;
            const uint32_t s_star = sel.kth_sum(keys, cnt, (uint32_t)k, n_less, n_eq);
            uint64_t bound = ((uint64_t)s_star << 32) | 0xFFFFFFFFull;
            if (n_less + n_eq > gate) bound = sel.kth_key(keys, cnt, (uint32_t)k);  // pathological ties
            const int kept = sel.keep_le(keys, cnt, bound);
            if (tid == 0) {
                misc[0] = (uint32_t)kept;
                misc[1] = min(vmisc[1], s_star);
                atomicMax(&ws.ginv[q], ~s_star);  // this CTA holds k entries with s' <= s*
            }
            __syncthreads();
        }
        if (tid == 0 && (r & 7) == 7) {
            // Fold in the global bound: entries with s' > g cannot be in the top k.
            const uint32_t g = ~*reinterpret_cast<volatile uint32_t *>(&ws.ginv[q]);
            const uint32_t gthr = g >= 0xFFFFu ? 0x10000u : g + 1u;
            if (gthr < vmisc[1]) vmisc[1] = gthr;
        }
    }
    __syncthreads();

    // Wait (bounded) for copies still in flight after a failure, so that no
    // bulk copy targets this CTA's shared memory after it exits.
    if (failed && lane == 0) {
        for (int s = 0; s < stages; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&mybars[s], (phase >> s) & 1u, kWaitLimit / 10);
    }
    if (failed) atomicOr(&misc[2], 1u);
    __syncthreads();

    // Exact top k of this CTA.
    int cnt = (int)vmisc[0];
    if (cnt > k) {
        const uint64_t kth = sel.kth_key(keys, cnt, (uint32_t)k);
        cnt = sel.keep_le(keys, cnt, kth);
    }
    uint64_t *cand = ws.cand + ((int64_t)q * G + cta) * k;
    for (int i = tid; i < cnt; i += T) cand[i] = keys[i];
    if (tid == 0) {
        ws.cnt[q * G + cta] = (uint32_t)cnt;
        if (misc[2]) atomicOr(&ws.status[q], 1u);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) misc[3] = (atomicAdd(&ws.ticket[q], 1u) == (uint32_t)(G - 1)) ? 1u : 0u;
    __syncthreads();
    if (vmisc[3] == 0) return;
    __threadfence();

    // Last CTA: merge the G lists in shared memory.
    uint64_t *mk = reinterpret_cast<uint64_t *>(smem);
    int total = 0;
    for (int c = 0; c < G; ++c) {
        const int cc = (int)__ldcg(&ws.cnt[q * G + c]);
        const uint64_t *src = ws.cand + ((int64_t)q * G + c) * k;
        for (int i = tid; i < cc; i += T) mk[total + i] = __ldcg(src + i);
        total += cc;
    }
    __syncthreads();
    int kout = total < k ? total : k;
    if (total > k) {
        const uint64_t kth = sel.kth_key(mk, total, (uint32_t)k);
        kout = sel.keep_le(mk, total, kth);
    }
    int P = 1;
    while (P < kout) P <<= 1;
    for (int i = kout + tid; i < P; i += T) mk[i] = ~0ull;
    __syncthreads();
    sel.sort_pow2(mk, P);
    const bool bad = __ldcg(&ws.status[q]) != 0u;
    for (int r = tid; r < k; r += T) {
        uint16_t s = 0;
        int64_t idx = -1;
        if (r < kout) {
            const uint64_t key = mk[r];
            const uint32_t sp = (uint32_t)(key >> 32);
            s = (uint16_t)(metric == BOLT_METRIC_DOT ? 0xFFFFu - sp : sp);
            idx = (int64_t)(uint32_t)key;
        }
        if (bad) idx = -2;
        out_sums[q * k + r] = s;
        out_idx[q * k + r] = idx;
    }
    if (tid == 0) {
        ws.ticket[q] = 0;
        ws.ginv[q] = 0;
    }
}

// ------------------------------------------------------------------ host side
static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int plan_topk(int64_t n, int32_t M, int32_t k, TopkPlan *plan) {
    BOLT_REQUIRE(k >= 1 && k <= kMaxK, BOLT_EUNSUPPORTED, "k=%d outside [1, %d]", k, kMaxK);
    const size_t stage_bytes = (size_t)M * kRowBytes;
    int warps = 16, stages = 0;
    for (warps = 16; warps >= 2; warps >>= 1) {
        stages = (int)(kStageBudget / (warps * stage_bytes));
        if (stages > kMaxStages) stages = kMaxStages;
        if (stages >= 2) break;
    }
    BOLT_REQUIRE(stages >= 2, BOLT_EUNSUPPORTED, "M=%d too large for the top-k kernel", M);
    const int cap = (k + 15) / 16 * 16 + 2 * warps * kBlockVecs;  // multiple of 16: keeps later regions aligned
    const int64_t nb = num_blocks(n);
    const size_t region = (size_t)warps * stages * stage_bytes + (size_t)cap * 8;
    const int64_t merge_keys = (int64_t)(region / 8);
    int64_t g = device_sm_count();
    if (g <= 0) g = 1;
    const int64_t by_work = (nb + warps - 1) / warps;  // at least one full round per CTA
    if (g > by_work) g = by_work;
    if (g > merge_keys / k) g = merge_keys / k;
    if (g < 1) g = 1;
    plan->warps = warps;
    plan->stages = stages;
    plan->grid = (int)g;
    plan->cap = cap;
    plan->blocks_per_cta = nb > 0 ? (nb + g - 1) / g : 0;
    plan->smem_bytes = region + align_up((size_t)M * 16, 16) + (size_t)warps * kMaxStages * 8 + 256 * 4 + 64 * 4;
    return BOLT_OK;
}

size_t topk_header_bytes(int64_t nq) { return align_up((size_t)nq * 12, 256); }

int64_t topk_workspace_bytes(const TopkPlan &plan, int64_t nq, int32_t k) {
    return (int64_t)(topk_header_bytes(nq) + align_up((size_t)nq * plan.grid * 4, 256) +
                     (size_t)nq * plan.grid * k * 8);
}

TopkWS carve_topk_ws(void *ws, const TopkPlan &plan, int64_t nq, int32_t k) {
    uint8_t *p = static_cast<uint8_t *>(ws);
    TopkWS w;
    w.ginv = reinterpret_cast<uint32_t *>(p);
    w.ticket = w.ginv + nq;
    w.status = w.ticket + nq;
    p += topk_header_bytes(nq);
    w.cnt = reinterpret_cast<uint32_t *>(p);
    p += align_up((size_t)nq * plan.grid * 4, 256);
    w.cand = reinterpret_cast<uint64_t *>(p);
    (void)k;
    return w;
}

template <int WARPS>
static int launch_w(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                    int32_t metric, uint16_t *out_sums, int64_t *out_idx, const TopkWS &w, const TopkPlan &plan,
                    cudaStream_t stream) {
    auto kern = topk_kernel<WARPS>;
    BOLT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem_bytes));
    dim3 grid(plan.grid, (unsigned)nq);
    kern<<<grid, WARPS * 32, plan.smem_bytes, stream>>>(reinterpret_cast<const uint32_t *>(codes), n, M, luts, k,
                                                         metric, w, plan.stages, plan.cap, plan.blocks_per_cta,
                                                         out_sums, out_idx);
    return check_launch("topk_kernel");
}

int launch_topk(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, const TopkPlan &plan,
                cudaStream_t stream) {
    BOLT_REQUIRE(nq <= 65535, BOLT_EUNSUPPORTED, "nq=%lld > 65535 per call", (long long)nq);
    BOLT_CUDA(cudaMemsetAsync(workspace, 0, topk_header_bytes(nq), stream));
    const TopkWS w = carve_topk_ws(workspace, plan, nq, k);
    switch (plan.warps) {
        case 16: return launch_w<16>(codes, n, M, luts, nq, k, metric, out_sums, out_idx, w, plan, stream);
        case 8: return launch_w<8>(codes, n, M, luts, nq, k, metric, out_sums, out_idx, w, plan, stream);
        case 4: return launch_w<4>(codes, n, M, luts, nq, k, metric, out_sums, out_idx, w, plan, stream);
        default: return launch_w<2>(codes, n, M, luts, nq, k, metric, out_sums, out_idx, w, plan, stream);
    }
}

}  // namespace bolt

extern "C" {

int64_t bolt_topk_workspace_bytes(int64_t n, int32_t M, int64_t nq, int32_t k) {
    bolt::clear_error();
    if (bolt::check_nm(n, M) || nq < 0) return -1;
    bolt::TopkPlan plan;
    if (bolt::plan_topk(n, M, k, &plan)) return -1;
    return bolt::topk_workspace_bytes(plan, nq, k);
}

int bolt_topk(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
              int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, int64_t workspace_bytes,
              void *stream) {
    bolt::clear_error();
    int rc = bolt::check_nm(n, M);
    if (rc) return rc;
    BOLT_REQUIRE(nq >= 0, BOLT_EINVAL, "nq=%lld < 0", (long long)nq);
    BOLT_REQUIRE(metric == BOLT_METRIC_L2 || metric == BOLT_METRIC_DOT, BOLT_EINVAL, "bad metric %d", metric);
    bolt::TopkPlan plan;
    rc = bolt::plan_topk(n, M, k, &plan);
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
