// Encoder entry points shared between the fp32 and tensor-core paths.
#pragma once

#include "common.cuh"

namespace bolt {

// Staged (bulk-copied, shared-memory) kernel when J % 4 == 0, else the
// simple one-vector-per-thread kernel.
int launch_encode_simple(const float *X, int64_t n, int32_t J, int32_t M, const float *C, uint8_t *codes,
                         cudaStream_t stream);
int launch_encode_fp32(const float *X, int64_t n, int32_t J, int32_t M, const float *C, uint8_t *codes,
                       cudaStream_t stream);

// Tensor-core (tcgen05, bf16 in / fp32 accumulate) encoder with fp32 re-check.
bool encode_tc_supported(int32_t J, int32_t M);
int launch_encode_tc(const float *X, int64_t n, int32_t J, int32_t M, const float *C, uint8_t *codes,
                     int64_t *n_rechecked, cudaStream_t stream);

}  // namespace bolt
