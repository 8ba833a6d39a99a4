// Measurement probes for the roofline of the scan (no Bolt results): the
// integer-ALU lane rate of the GPU, read from clock64 around a loop of
// independent byte permutes, and the time of one pass of the lookup core
// over a code array with nothing but a running minimum as output (the
// floor that any one-query fused scan + top-k built on that core meets).
#include "scan_core.cuh"

namespace bolt {

constexpr int kProbeChains = 8;
constexpr int kProbeReps = 256;

__global__ void __launch_bounds__(1024, 1) probe_prmt_kernel(const uint32_t *in, uint32_t *out,
                                                             unsigned long long *cycles) {
    uint32_t v[kProbeChains];
    const uint32_t y = in[threadIdx.x & 7], z = in[8 + (threadIdx.x & 7)];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) v[c] = in[16 + c] + threadIdx.x;
    const long long t0 = clock64();
#pragma unroll 1
    for (int r = 0; r < kProbeReps; ++r) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) {
                uint32_t d;
                asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(v[c]), "r"(y), "r"(z));
                v[c] = d;
            }
    }
    const long long t1 = clock64();
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s ^= v[c];
    if (s == 0x9E3779B9u) out[0] = s;  // keeps the chains live
    if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
}

// One pass of the lookup core (scan_core.cuh) over n vectors with M = 16,
// two blocks per unit, 16 warps with private rings of two bulk-copy stages,
// blocks split statically over the CTAs; writes the smallest sum.
constexpr int kProbeWarps = 16, kProbeM = 16, kProbeBpi = 2, kProbeStages = 2;

__global__ void __launch_bounds__(kProbeWarps * 32, 1)
    probe_core_kernel(const uint32_t *__restrict__ codes, int64_t n, const uint8_t *__restrict__ luts,
                      int64_t units_per_cta, uint32_t *out_min, uint32_t *failed) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t blk_words = kProbeM * kRowWords;
    constexpr uint32_t blk_bytes = kProbeM * kRowBytes;
    uint4 *lut = reinterpret_cast<uint4 *>(smem + kProbeWarps * kProbeStages * kProbeBpi * blk_bytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(lut + kProbeM);
    const uint32_t nb = (uint32_t)num_blocks(n);
    const uint32_t nu = (nb + kProbeBpi - 1) / kProbeBpi;
    const uint32_t u_lo = (uint32_t)min((int64_t)nu, (int64_t)blockIdx.x * units_per_cta);
    const uint32_t u_hi = (uint32_t)min((int64_t)nu, (int64_t)u_lo + units_per_cta);
    uint64_t *mybars = bars + warp * kProbeStages;
    uint8_t *mystage = smem + (size_t)warp * kProbeStages * kProbeBpi * blk_bytes;
    auto unit_bytes = [&](uint32_t u) { return min((uint32_t)kProbeBpi, nb - u * kProbeBpi) * blk_bytes; };
    uint32_t pending = 0;
    if (lane == 0) {
        for (int s = 0; s < kProbeStages; ++s) mbar_init(&mybars[s], 1);
        fence_mbar_init();
        for (int s = 0; s < kProbeStages; ++s) {
            const uint32_t u = u_lo + (uint32_t)s * kProbeWarps + warp;
            if (u < u_hi) {
                mbar_arrive_expect_tx(&mybars[s], unit_bytes(u));
                bulk_g2s(mystage + (size_t)s * kProbeBpi * blk_bytes, codes + (size_t)u * kProbeBpi * blk_words,
                         unit_bytes(u), &mybars[s]);
                pending |= 1u << s;
            }
        }
    }
    for (int i = threadIdx.x; i < kProbeM; i += kProbeWarps * 32) lut[i] = reinterpret_cast<const uint4 *>(luts)[i];
    __syncthreads();
    uint32_t best = 0xFFFFFFFFu, st = 0, par = 0;
    uint32_t phase = 0;  // lane 0: parity of the next completion of each stage
    bool bad = false;
    for (uint32_t u = u_lo + warp; u < u_hi; u += kProbeWarps) {
        const bool ok = mbar_wait_bounded(&mybars[st], par, 1000000000ull);
        if (!__all_sync(0xFFFFFFFFu, ok)) {
            bad = true;
            break;
        }
        const uint32_t *words = reinterpret_cast<const uint32_t *>(mystage + (size_t)st * kProbeBpi * blk_bytes);
        const uint32_t nblk = min((uint32_t)kProbeBpi, nb - u * kProbeBpi);
        Acc8 acc[kProbeBpi];
#pragma unroll
        for (int h = 0; h < kProbeBpi; ++h) acc[h].zero();
#pragma unroll
        for (int m = 0; m < kProbeM; ++m) {
            const uint4 t = lut[m];
#pragma unroll
            for (int h = 0; h < kProbeBpi; ++h) acc[h].add(prep_word(words[h * blk_words + m * kRowWords + lane]), t);
        }
        __syncwarp();
        if (lane == 0) {
            pending &= ~(1u << st);
            phase ^= 1u << st;
            const uint32_t u2 = u + kProbeStages * kProbeWarps;
            if (u2 < u_hi) {
                mbar_arrive_expect_tx(&mybars[st], unit_bytes(u2));
                bulk_g2s(mystage + (size_t)st * kProbeBpi * blk_bytes, codes + (size_t)u2 * kProbeBpi * blk_words,
                         unit_bytes(u2), &mybars[st]);
                pending |= 1u << st;
            }
        }
        if (++st == kProbeStages) {
            st = 0;
            par ^= 1u;
        }
#pragma unroll
        for (int h = 0; h < kProbeBpi; ++h) {
            if ((uint32_t)h >= nblk) break;  // the last unit may hold one block
            uint32_t e[4];
            acc[h].finish(e[0], e[1], e[2], e[3]);
            const uint32_t v0 = (u * kProbeBpi + h) * kBlockVecs + 8u * lane;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t s = (e[(i & 1) + 2 * (i >> 2)] >> (16 * ((i >> 1) & 1))) & 0xFFFFu;
                if (v0 + i < (uint32_t)n) best = min(best, s);
            }
        }
    }
    // after a failed wait: wait (bounded) for this warp's copies still in flight
    if (bad && lane == 0) {
        for (int s = 0; s < kProbeStages; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&mybars[s], (phase >> s) & 1u, 100000000ull);
        atomicOr(failed, 1u);
    }
    best = __reduce_min_sync(0xFFFFFFFFu, best);
    if (lane == 0) atomicMin(out_min, best);
}

}  // namespace bolt

extern "C" {

int bolt_probe_int_lanes(double *lanes_per_clk_per_sm) {
    bolt::clear_error();
    BOLT_REQUIRE(lanes_per_clk_per_sm, BOLT_EINVAL, "null pointer");
    int dev = 0;
    BOLT_CUDA(cudaGetDevice(&dev));
    uint32_t *buf = nullptr;
    unsigned long long *cyc = nullptr;
    BOLT_CUDA(cudaMalloc(&buf, 256));
    BOLT_CUDA(cudaMalloc(&cyc, 8));
    uint32_t h[64];
    for (int i = 0; i < 64; ++i) h[i] = 0x01234567u * (uint32_t)(i + 1) | 1u;
    cudaMemcpy(buf, h, 256, cudaMemcpyHostToDevice);
    int sms = bolt::device_sm_count();
    unsigned long long c = 0;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
        cudaMemset(cyc, 0, 8);
        bolt::probe_prmt_kernel<<<sms, 1024>>>(buf, buf + 48, cyc);
    }
    cudaError_t e = cudaMemcpy(&c, cyc, 8, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    cudaFree(cyc);
    BOLT_REQUIRE(e == cudaSuccess && c > 0, BOLT_ECUDA, "probe kernel failed: %s", cudaGetErrorString(e));
    // one CTA per SM: 1024 threads x reps x 8 x chains prmt in c cycles
    *lanes_per_clk_per_sm = 1024.0 * bolt::kProbeReps * 8 * bolt::kProbeChains / (double)c;
    return BOLT_OK;
}

int bolt_probe_lookup_core(const uint8_t *codes, int64_t n, const uint8_t *luts, int32_t reps, float *us_per_pass,
                           void *stream) {
    bolt::clear_error();
    BOLT_REQUIRE(codes && luts && us_per_pass && n > 0 && reps > 0, BOLT_EINVAL, "bad arguments");
    BOLT_REQUIRE(bolt::aligned(codes, 16) && bolt::aligned(luts, 16), BOLT_EINVAL, "16-byte alignment");
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = bolt::device_sm_count();
    const int64_t nb = bolt::num_blocks(n);
    const int64_t nu = (nb + bolt::kProbeBpi - 1) / bolt::kProbeBpi;
    const int64_t upc = (nu + sms - 1) / sms;
    const size_t smem = (size_t)bolt::kProbeWarps * bolt::kProbeStages * bolt::kProbeBpi * bolt::kProbeM *
                            bolt::kRowBytes + bolt::kProbeM * 16 + bolt::kProbeWarps * bolt::kProbeStages * 8;
    int rc = bolt::ensure_smem((const void *)bolt::probe_core_kernel, smem);
    if (rc) return rc;
    uint32_t *out = nullptr;
    BOLT_CUDA(cudaMallocAsync(&out, 8, s));
    BOLT_CUDA(cudaMemsetAsync(out, 0, 8, s));
    cudaEvent_t e0, e1;
    BOLT_CUDA(cudaEventCreate(&e0));
    BOLT_CUDA(cudaEventCreate(&e1));
    for (int i = 0; i < 2; ++i)
        bolt::probe_core_kernel<<<sms, bolt::kProbeWarps * 32, smem, s>>>(reinterpret_cast<const uint32_t *>(codes),
                                                                        n, luts, upc, out, out + 1);
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; ++i)
        bolt::probe_core_kernel<<<sms, bolt::kProbeWarps * 32, smem, s>>>(reinterpret_cast<const uint32_t *>(codes),
                                                                        n, luts, upc, out, out + 1);
    cudaEventRecord(e1, s);
    rc = bolt::check_launch("probe_core_kernel");
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    uint32_t hflag[2] = {0, 0};
    cudaMemcpyAsync(hflag, out, 8, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    cudaFreeAsync(out, s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    BOLT_REQUIRE(hflag[1] == 0, BOLT_ETIMEOUT, "a bounded wait of the probe gave up");
    *us_per_pass = ms * 1000.f / (float)reps;
    return BOLT_OK;
}

}  // extern "C"
