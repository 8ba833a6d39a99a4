// Status plumbing, device queries and the host-only entry points.
#include <stdarg.h>
#include <string.h>

#include <map>
#include <atomic>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "tma.cuh"

namespace bolt {

static thread_local char g_err[1024];

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: launch failed: %s", what, cudaGetErrorString(e));
        return BOLT_ECUDA;
    }
    return BOLT_OK;
}

static std::atomic<uint64_t> g_data_wait_ns{1000000000ull};

uint64_t data_wait_limit_ns() { return g_data_wait_ns.load(std::memory_order_relaxed); }

int device_sm_count() {
    static std::mutex mu;
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev] = v;
    }
    return cache[dev];
}

int ensure_smem(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> done;
    int dev = 0;
    BOLT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, func);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return BOLT_OK;
    BOLT_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done[key] = bytes;
    return BOLT_OK;
}

int check_nm(int64_t n, int32_t M) {
    BOLT_REQUIRE(n >= 0 && n < (int64_t(1) << 31), BOLT_EINVAL, "n=%lld out of range [0, 2^31)", (long long)n);
    BOLT_REQUIRE(M >= 1, BOLT_EINVAL, "M=%d must be >= 1", M);
    BOLT_REQUIRE(M <= 256, BOLT_EUNSUPPORTED, "M=%d > 256 is unsupported (uint16 sums)", M);
    return BOLT_OK;
}

int check_nm_wide(int64_t n, int32_t M) {
    BOLT_REQUIRE(n >= 0 && n < (int64_t(1) << 31), BOLT_EINVAL, "n=%lld out of range [0, 2^31)", (long long)n);
    BOLT_REQUIRE(M >= 1, BOLT_EINVAL, "M=%d must be >= 1", M);
    BOLT_REQUIRE(M <= kMaxWideM, BOLT_EUNSUPPORTED, "M=%d > %d is unsupported", M, kMaxWideM);
    return BOLT_OK;
}

int check_jm_wide(int32_t J, int32_t M) {
    BOLT_REQUIRE(J >= 1 && M >= 1, BOLT_EINVAL, "J=%d, M=%d must be >= 1", J, M);
    BOLT_REQUIRE(M <= kMaxWideM, BOLT_EUNSUPPORTED, "M=%d > %d is unsupported", M, kMaxWideM);
    BOLT_REQUIRE(J % M == 0, BOLT_EUNSUPPORTED, "J=%d is not a multiple of M=%d", J, M);
    BOLT_REQUIRE(J / M <= 256, BOLT_EUNSUPPORTED, "subspace dim J/M=%d > 256 is unsupported", J / M);
    return BOLT_OK;
}

int check_jm(int32_t J, int32_t M) {
    BOLT_REQUIRE(J >= 1 && M >= 1, BOLT_EINVAL, "J=%d, M=%d must be >= 1", J, M);
    BOLT_REQUIRE(M <= 256, BOLT_EUNSUPPORTED, "M=%d > 256 is unsupported", M);
    BOLT_REQUIRE(J % M == 0, BOLT_EUNSUPPORTED, "J=%d is not a multiple of M=%d", J, M);
    BOLT_REQUIRE(J / M <= 256, BOLT_EUNSUPPORTED, "subspace dim J/M=%d > 256 is unsupported", J / M);
    return BOLT_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

}  // namespace bolt

extern "C" {

const char *bolt_last_error(void) { return bolt::g_err; }

const char *bolt_version(void) { return "bolt-gb300 0.1 (sm_103a)"; }

int bolt_set_wait_limit_ns(uint64_t ns) {
    bolt::clear_error();
    bolt::g_data_wait_ns.store(ns == 0 ? 1000000000ull : ns, std::memory_order_relaxed);
    return BOLT_OK;
}

int64_t bolt_codes_bytes(int64_t n, int32_t M) {
    if (n < 0 || M < 1 || M > bolt::kMaxWideM) return -1;
    return bolt::num_blocks(n) * (int64_t)M * bolt::kRowBytes;
}

int bolt_dequant_params(float a, const float *b_host, int32_t M, float *inv_a_host, float *bias_host) {
    bolt::clear_error();
    BOLT_REQUIRE(b_host && inv_a_host && bias_host, BOLT_EINVAL, "null pointer");
    BOLT_REQUIRE(M >= 1 && M <= bolt::kMaxWideM, BOLT_EINVAL, "M=%d out of range", M);
    BOLT_REQUIRE(a > 0.0f, BOLT_EINVAL, "scale a=%g must be > 0", (double)a);
    double tot = 0.0;
    for (int m = 0; m < M; ++m) tot += (double)b_host[m];
    *inv_a_host = (float)(1.0 / (double)a);
    *bias_host = (float)tot;
    return BOLT_OK;
}

}  // extern "C"
