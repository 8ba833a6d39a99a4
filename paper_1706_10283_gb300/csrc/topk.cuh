// Fused scan + exact top-k: launch plan and workspace layout.
#pragma once

#include "common.cuh"

namespace bolt {

constexpr int kBins = 4096;  // histogram bins over candidate sums
// Shared-memory size class (topk_small.cu): every CTA's codes and sums fit in
// shared memory and the last CTA merges at most kSmallMergeKeys keys.
constexpr int kSmallMergeKeys = 16384;
constexpr int kMaxSmallK = 1024;
constexpr size_t kSmallMaxSmem = 220 * 1024;
constexpr int64_t kMqMinQueries = 4;

struct TopkPlan {
    int small;            // 1: shared-memory size class (topk_small.cu); the fields below
                          //    marked (s) are the ones it uses
    int nbc;              // (s) code blocks per CTA
    int mq;               // 1: sample bound + filter + select (topk_mq.cu), streaming fallback
    int mq_ns;            // sample blocks
    int64_t mq_cap;       // candidate-list capacity per query
    int mq_hshift;        // histogram bin width 2^mq_hshift
    int warps;            // warps per CTA (16, 8, 4 or 2, by stage size)
    int bpi;              // code blocks per unit of work (one bulk copy)
    int stages;           // TMA stages per warp
    int grid;             // (s) CTAs per query
    int cap;              // candidate-buffer entries per CTA
    int hshift;           // (s) histogram bin width 2^hshift
    int out_cap;          // candidates one CTA may append (k <= out_cap <= 2k)
    int list_cap;         // per-query candidate list length: grid slots of out_cap + 1 entries
    int64_t blocks_per_cta;  // units of work per CTA
    size_t smem_bytes;    // (s)
};

// Per-query device state in the workspace.
struct TopkWS {
    uint32_t *ticket;  // [nq] CTAs finished
    uint32_t *status;  // [nq] bit 0: a bounded wait gave up
    uint32_t *ghist;   // [nq][kBins] counted candidates per sum bin
    uint32_t *gcoarse; // [nq][kBins / 16] the same counts in bins 16 times wider
    uint64_t *cand;    // [nq][grid][out_cap + 1] per CTA: key count, then keys (sum' << 32 | index)
};

// Size class by database size and query count: shared-memory kernel
// (topk_small.cu), multi-query pipeline (topk_mq.cu, nq >= kMqMinQueries) or
// the fused streaming kernel (topk.cu).
int plan_topk(int64_t n, int32_t M, int32_t k, int64_t nq, TopkPlan *plan);
int64_t topk_workspace_bytes(const TopkPlan &plan, int64_t nq, int32_t k);
TopkWS carve_topk_ws(void *ws, const TopkPlan &plan, int64_t nq, int32_t k);
size_t topk_header_bytes(int64_t nq);  // ticket/status + histograms (zeroed per call)

// max_ctas > 0 caps the CTAs per query
bool plan_topk_small(int64_t n, int32_t M, int32_t k, int sms, TopkPlan *plan, int64_t max_ctas = 0);
int64_t topk_small_workspace_bytes(const TopkPlan &plan, int64_t nq, int32_t k);
int launch_topk_small(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                      int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, const TopkPlan &plan,
                      cudaStream_t stream);

int plan_topk_stream(int64_t n, int32_t M, int32_t k, TopkPlan *plan);
int64_t topk_stream_workspace_bytes(const TopkPlan &plan, int64_t nq, int32_t k);
void plan_topk_mq(int64_t n, int32_t M, int32_t k, int sms, TopkPlan *plan);
int64_t topk_mq_workspace_bytes(const TopkPlan &plan, int64_t nq, int32_t k);
int launch_topk_mq(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                   int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, const TopkPlan &plan,
                   cudaStream_t stream);
// the streaming kernel; with active != NULL only queries q with active[q] != 0 run
int launch_topk_stream(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                       int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, const TopkPlan &plan,
                       const uint32_t *active, cudaStream_t stream);

int launch_topk(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, const TopkPlan &plan,
                cudaStream_t stream);

}  // namespace bolt
