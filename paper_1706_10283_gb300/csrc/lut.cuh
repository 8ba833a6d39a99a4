// Query-table build (Sec. 3.1 g, Sec. 3.2 beta_m), shared by the entry
// points that need tables internally (approximate matmul, quantizer fit).
#pragma once

#include "common.cuh"

namespace bolt {

// Quantizer parameters passed by value to kernels: scale a and the M
// per-table offsets b_m (M <= 256).
struct QuantParams {
    float a;
    float b[256];
};

int make_quant_params(float a, const float *b_host, int32_t M, QuantParams *qp);

// b_dev (nullable): offsets in device memory (M > 256); else qp.b is used.
// p: the exponent of BOLT_METRIC_LP tables (unused for the other metrics).
int launch_build_luts(const float *Q, int64_t nq, int32_t J, int32_t M, const float *C, int32_t metric,
                      const QuantParams &qp, uint8_t *luts, float *luts_f32, cudaStream_t stream,
                      const float *b_dev = nullptr, float p = 1.0f);

}  // namespace bolt
