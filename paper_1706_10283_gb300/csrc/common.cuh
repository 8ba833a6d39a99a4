// Shared helpers of the Bolt CUDA library (sm_103a): status plumbing and
// small inline-PTX wrappers.  Nothing here implements Bolt arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/bolt.h"

namespace bolt {

constexpr int kK = 16;            // centroids per codebook (Sec. 3.2, change 1)
constexpr int kBlockVecs = 256;   // vectors per code block
constexpr int kRowBytes = 128;    // bytes per (block, codebook) row
constexpr int kRowWords = 32;     // 32-bit words per row: one per lane

// ------------------------------------------------------------------ status
void set_error(const char *fmt, ...);
void clear_error();
int check_launch(const char *what);  // BOLT_OK or BOLT_ECUDA with message

#define BOLT_REQUIRE(cond, code, ...)   \
    do {                                \
        if (!(cond)) {                  \
            ::bolt::set_error(__VA_ARGS__); \
            return (code);              \
        }                               \
    } while (0)

#define BOLT_CUDA(call)                                                          \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            ::bolt::set_error("%s failed: %s", #call, cudaGetErrorString(e_));   \
            return BOLT_ECUDA;                                                   \
        }                                                                        \
    } while (0)

__host__ __device__ inline bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

__host__ __device__ inline int64_t num_blocks(int64_t n) { return (n + kBlockVecs - 1) / kBlockVecs; }

int device_sm_count();  // SMs of the current device (cached per device)

// Time limit of the kernels' waits for their own data (bulk copies, MMAs):
// 1 s unless bolt_set_wait_limit_ns changed it (tests of the timeout path).
// Waits that drain copies in flight after a failure keep their own limits.
uint64_t data_wait_limit_ns();

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (device, kernel)
// and size: later launches (including ones under stream capture) make no
// attribute call.
int ensure_smem(const void *func, size_t bytes);

// Shape checks shared by the entry points.
int check_nm(int64_t n, int32_t M);
int check_jm(int32_t J, int32_t M);
// Entry points without uint16 sums (layout, encode, tables, uint32 scan)
// accept up to kMaxWideM codebooks.
constexpr int kMaxWideM = 4096;
int check_nm_wide(int64_t n, int32_t M);
int check_jm_wide(int32_t J, int32_t M);

// Metrics whose sums the top-k family ranks (L2, L1 and L_p ascending, dot
// descending).
__host__ __device__ inline bool rank_metric_ok(int32_t metric) {
    return metric == BOLT_METRIC_L2 || metric == BOLT_METRIC_DOT || metric == BOLT_METRIC_L1 ||
           metric == BOLT_METRIC_LP;
}

// ------------------------------------------------------------------ phase stamps
// Diagnostic builds only (-DBOLT_PHASE_STAMPS, libbolt_stamps.so; see
// paper_1706_10283_gb300/phases.py): a kernel's thread 0 of CTA c of query 0
// records the global timer, or a count, in slot i of its kernel's stamp
// array.  In the library itself the macros expand to nothing.
#ifdef BOLT_PHASE_STAMPS
#define BOLT_STAMP_ARRAY(name) __device__ unsigned long long name[1024 * 16]
#define BOLT_STAMP(arr, q, cta, i) \
    do {                                                                         \
        if ((q) == 0 && (cta) < 1024 && threadIdx.x == 0) arr[(cta) * 16 + (i)] = ::bolt::globaltimer_ns(); \
    } while (0)
#define BOLT_STAMP_VALUE(arr, q, cta, i, v) \
    do {                                                                          \
        if ((q) == 0 && (cta) < 1024 && threadIdx.x == 0) arr[(cta) * 16 + (i)] = (unsigned long long)(v); \
    } while (0)
#else
#define BOLT_STAMP_ARRAY(name) static_assert(true, "")
#define BOLT_STAMP(arr, q, cta, i) \
    do {                           \
    } while (0)
#define BOLT_STAMP_VALUE(arr, q, cta, i, v) \
    do {                                    \
    } while (0)
#endif

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte permute (default mode): selector nibble i picks byte (sel & 7) of
// {b:a} for output byte i; a set nibble bit 3 replicates that byte's sign bit.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of a phase (mbarrier.try_wait may itself suspend the
// thread until the phase completes).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: gives up after `limit_ns` nanoseconds of wall-clock time and
// returns false, so a copy that never lands cannot stall the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}

// Limits below kPollBelowNs (tests of the timeout path) are enforced by
// polling with the non-blocking test, so that the limit and not the
// hardware's suspend time decides when the wait gives up.
constexpr uint64_t kPollBelowNs = 1000;

__device__ __forceinline__ bool mbar_poll_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_test_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_test_wait(bar, parity))
        if (globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}

// 1-D bulk copy global -> shared (TMA engine, non-multicast), completing on
// `bar` with `bytes` transaction bytes.  dst/src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

}  // namespace bolt
