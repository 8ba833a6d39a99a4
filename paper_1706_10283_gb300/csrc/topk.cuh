// Fused scan + exact top-k: launch plan and workspace layout.
#pragma once

#include "common.cuh"

namespace bolt {

struct TopkPlan {
    int warps;            // warps per CTA (16, 8, 4 or 2, by stage size)
    int stages;           // TMA stages per warp
    int grid;             // CTAs per query
    int cap;              // candidate-buffer entries per CTA
    int64_t blocks_per_cta;
    size_t smem_bytes;
};

// Per-query device state in the workspace.
struct TopkWS {
    uint32_t *ginv;    // [nq] bitwise NOT of the best published sum threshold (0 = none)
    uint32_t *ticket;  // [nq] CTAs finished
    uint32_t *status;  // [nq] bit 0: a bounded wait gave up
    uint32_t *cnt;     // [nq][grid] candidates written by each CTA
    uint64_t *cand;    // [nq][grid][k] candidate keys (sum' << 32 | index)
};

int plan_topk(int64_t n, int32_t M, int32_t k, TopkPlan *plan);
int64_t topk_workspace_bytes(const TopkPlan &plan, int64_t nq, int32_t k);
TopkWS carve_topk_ws(void *ws, const TopkPlan &plan, int64_t nq, int32_t k);
size_t topk_header_bytes(int64_t nq);

int launch_topk(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts, int64_t nq, int32_t k,
                int32_t metric, uint16_t *out_sums, int64_t *out_idx, void *workspace, const TopkPlan &plan,
                cudaStream_t stream);

}  // namespace bolt
