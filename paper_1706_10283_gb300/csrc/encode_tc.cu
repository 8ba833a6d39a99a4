// Tensor-core encoder (tcgen05).  Not yet available: bolt_encode falls back
// to the canonical fp32 kernel, which produces the same codes.
#include "encode.cuh"

namespace bolt {

bool encode_tc_supported(int32_t, int32_t) { return false; }

int launch_encode_tc(const float *, int64_t, int32_t, int32_t, const float *, uint8_t *, int64_t *, cudaStream_t) {
    set_error("tensor-core encoder not built");
    return BOLT_EUNSUPPORTED;
}

}  // namespace bolt
