// Merge of per-shard top-k lists into the top-k of the whole database.
//
// The database is split into row ranges (shards); each shard's exact top-k
// (bolt_topk on its own codes) is a list sorted best first by the key
// (s', index) with s' = S for L2 and 255*M - S for dot (ties to the lower
// index), padded with index -1.  Vectors are independent in the scan
// (Sec. 3.1: every distance depends on one vector's codes only), so the
// global top-k is the k smallest keys of the union of the shard lists, with
// global index = shard offset + local index.  One CTA per query places each
// entry at its rank in the union: its position in its own list plus, for
// every other list, the number of keys smaller than it (binary search).
#include "common.cuh"

namespace bolt {

constexpr int kMergeThreads = 256;
constexpr int kMaxShards = 1024;

struct MergeKey {
    uint32_t s;  // s' (0x10000 for padding)
    int64_t i;   // global index
};

__device__ __forceinline__ bool key_less(const MergeKey &a, const MergeKey &b) {
    return a.s < b.s || (a.s == b.s && a.i < b.i);
}

__device__ __forceinline__ MergeKey load_key(const uint16_t *sums, const int64_t *idx, int64_t pos, int64_t off,
                                             uint32_t smax, int32_t metric) {
    MergeKey key;
    const int64_t li = idx[pos];
    if (li < 0) {
        key.s = 0x10000u;
        key.i = INT64_MAX;
    } else {
        const uint32_t S = sums[pos];
        key.s = metric == BOLT_METRIC_DOT ? smax - S : S;
        key.i = off + li;
    }
    return key;
}

__global__ void __launch_bounds__(kMergeThreads) topk_merge_kernel(const uint16_t *__restrict__ sums,
                                                                   const int64_t *__restrict__ idx,
                                                                   const int64_t *__restrict__ offsets,
                                                                   int32_t nshard, int64_t nq, int32_t k,
                                                                   int32_t M, int32_t metric,
                                                                   uint16_t *__restrict__ out_sums,
                                                                   int64_t *__restrict__ out_idx) {
    __shared__ unsigned int s_valid, s_bad;
    const int64_t q = blockIdx.x;
    const uint32_t smax = 255u * (uint32_t)M;
    if (threadIdx.x == 0) s_valid = s_bad = 0;
    __syncthreads();
    const int64_t total = (int64_t)nshard * k;
    unsigned int valid = 0;
    for (int64_t e = threadIdx.x; e < total; e += kMergeThreads) {
        const int a = (int)(e / k), p = (int)(e % k);
        const int64_t base_a = ((int64_t)a * nq + q) * k;
        if (idx[base_a + p] == -2) s_bad = 1;  // a shard's top-k reported a failed wait
        const MergeKey x = load_key(sums, idx, base_a + p, offsets[a], smax, metric);
        if (x.s > 0xFFFFu) continue;  // padding
        ++valid;
        int64_t rank = p;
        for (int b = 0; b < nshard && rank < k; ++b) {
            if (b == a) continue;
            const int64_t base_b = ((int64_t)b * nq + q) * k;
            // number of keys of list b smaller than x (lists are sorted, padding last)
            int lo = 0, hi = k;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                const MergeKey y = load_key(sums, idx, base_b + mid, offsets[b], smax, metric);
                if (key_less(y, x)) lo = mid + 1;
                else hi = mid;
            }
            rank += lo;
        }
        if (rank < k) {
            out_sums[q * k + rank] = (uint16_t)(metric == BOLT_METRIC_DOT ? smax - x.s : x.s);
            out_idx[q * k + rank] = x.i;
        }
    }
    atomicAdd(&s_valid, valid);
    __syncthreads();
    // fewer than k entries in the union: pad like bolt_topk (sum 0, index -1)
    for (int r = (int)min((int64_t)k, (int64_t)s_valid) + threadIdx.x; r < k; r += kMergeThreads) {
        out_sums[q * k + r] = 0;
        out_idx[q * k + r] = -1;
    }
    if (s_bad) {
        __syncthreads();
        for (int r = threadIdx.x; r < k; r += kMergeThreads) out_idx[q * k + r] = -2;
    }
}

}  // namespace bolt

extern "C" int bolt_topk_merge(const uint16_t *sums, const int64_t *idx, const int64_t *offsets, int32_t nshard,
                               int64_t nq, int32_t k, int32_t M, int32_t metric, uint16_t *out_sums,
                               int64_t *out_idx, void *stream) {
    bolt::clear_error();
    BOLT_REQUIRE(nshard >= 1 && nshard <= bolt::kMaxShards, BOLT_EINVAL, "nshard=%d outside [1, %d]", nshard,
                 bolt::kMaxShards);
    BOLT_REQUIRE(nq >= 0 && nq <= 0x7FFFFFFF, BOLT_EINVAL, "nq=%lld", (long long)nq);
    BOLT_REQUIRE(k >= 1 && k <= 1024, BOLT_EUNSUPPORTED, "k=%d outside [1, 1024]", k);
    BOLT_REQUIRE(M >= 1 && M <= 256, BOLT_EUNSUPPORTED, "M=%d outside [1, 256]", M);
    BOLT_REQUIRE(bolt::rank_metric_ok(metric), BOLT_EINVAL,
                 "bad metric %d", metric);
    if (nq == 0) return BOLT_OK;
    BOLT_REQUIRE(sums && idx && offsets && out_sums && out_idx, BOLT_EINVAL, "null pointer");
    bolt::topk_merge_kernel<<<(unsigned)nq, bolt::kMergeThreads, 0, (cudaStream_t)stream>>>(
        sums, idx, offsets, nshard, nq, k, M, metric, out_sums, out_idx);
    return bolt::check_launch("topk_merge_kernel");
}
