// Batched multi-collection scan: the Sec. 3.1 sums d^(q, x) = sum_m
// D_q[m][h(x)_m] for many independent collections in one persistent launch.
//
// The host turns every collection into tasks (collection, query group, code
// block range).  A task's query group is nqt tiles of qt consecutive
// queries; its units are (block, tile) pairs.  A CTA takes a task from a
// global counter, stages the group's uint8 tables in shared memory, and its
// warps take the units round-robin.  A warp scans one 256-vector block for
// qt queries at once: every code word is loaded and prepared once and looked
// up qt times, with qt sets of accumulators in registers, so the load and
// the selector preparation are shared by the tile's queries.  Collections
// with uint32 sums (any M up to 4096) sum their codebooks in groups of 256,
// each group exact in the 16-bit lanes of the lookup core, into 32-bit sums.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "scan_core.cuh"

namespace bolt {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchLutEntries = 1024;  // uint4 table rows staged per task (16 KB)

struct BatchHeader {
    unsigned int counter;       // next uint16-sum task (both counters reset before every run)
    unsigned int counter_wide;  // next uint32-sum task
    int32_t ntasks;
    int32_t ncoll;
    int64_t colls_off;  // byte offsets from the plan base
    int64_t tasks_off;
    int64_t tasks_wide_off;
    int32_t ntasks_wide;
    int32_t reserved;
    int64_t pad[2];
};
static_assert(sizeof(BatchHeader) == 64, "header size");

struct BatchColl {
    const uint32_t *codes;
    const uint4 *luts;
    uint16_t *sums;  // uint32_t * for collections with uint32 sums (their own task list)
    int64_t n;
    int64_t ld;
    int32_t M;
    int32_t pad;
};
static_assert(sizeof(BatchColl) == 48, "collection record size");

struct BatchTask {
    int32_t coll;
    int32_t q0;   // first query of the group
    int32_t b0;   // first code block
    int32_t nb;   // code blocks
    int16_t qt;   // queries per tile (1, 2, 4, 8, 16)
    int16_t nqt;  // tiles in the group
    int32_t global_luts;  // 1: the group's tables are read from global memory (too large to stage)
};
static_assert(sizeof(BatchTask) == 24, "task size");

// One unit: block b of a collection for QT queries whose tables start at lut
// (row t*M + m holds query t's table m).
template <int QT>
__device__ __forceinline__ void batch_unit(const uint32_t *__restrict__ codes, int64_t b, int M,
                                           const uint4 *lut, uint16_t *__restrict__ sums, int64_t ld, int64_t n,
                                           int lane) {
    Acc8 acc[QT];
#pragma unroll
    for (int t = 0; t < QT; ++t) acc[t].zero();
    const uint32_t *row = codes + b * M * kRowWords + lane;
    int m = 0;
    for (; m + 4 <= M; m += 4) {
        uint32_t W[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) W[u] = __ldg(row + (int64_t)(m + u) * kRowWords);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const WordSel ws = prep_word(W[u]);
#pragma unroll
            for (int t = 0; t < QT; ++t) acc[t].add(ws, lut[t * M + m + u]);
        }
    }
    for (; m < M; ++m) {
        const WordSel ws = prep_word(__ldg(row + (int64_t)m * kRowWords));
#pragma unroll
        for (int t = 0; t < QT; ++t) acc[t].add(ws, lut[t * M + m]);
    }
    const int64_t v0 = b * kBlockVecs + 8 * lane;
    if (v0 < n) {  // ld >= n rounded up to 8, so the 16-byte store stays in the row
#pragma unroll
        for (int t = 0; t < QT; ++t) {
            uint32_t e_lo, o_lo, e_hi, o_hi;
            acc[t].finish(e_lo, o_lo, e_hi, o_hi);
            __stcs(reinterpret_cast<uint4 *>(sums + t * ld + v0), pack_sums(e_lo, o_lo, e_hi, o_hi));
        }
    }
}

// The same for uint32 sums: codebooks in groups of 256 (each group's sums
// exact in the 16-bit lanes), added into 32-bit sums.  lut may point to
// shared or global memory.
template <int QT>
__device__ __forceinline__ void batch_unit_u32(const uint32_t *__restrict__ codes, int64_t b, int M, const uint4 *lut,
                                               uint32_t *__restrict__ sums, int64_t ld, int64_t n, int lane) {
    uint32_t tot[QT][8];
#pragma unroll
    for (int t = 0; t < QT; ++t)
#pragma unroll
        for (int i = 0; i < 8; ++i) tot[t][i] = 0u;
    const uint32_t *row = codes + b * M * kRowWords + lane;
    for (int m0 = 0; m0 < M; m0 += 256) {
        const int m1 = min(M, m0 + 256);
        Acc8 acc[QT];
#pragma unroll
        for (int t = 0; t < QT; ++t) acc[t].zero();
#pragma unroll 4
        for (int m = m0; m < m1; ++m) {
            const WordSel ws = prep_word(__ldg(row + (int64_t)m * kRowWords));
#pragma unroll
            for (int t = 0; t < QT; ++t) acc[t].add(ws, lut[t * M + m]);
        }
#pragma unroll
        for (int t = 0; t < QT; ++t) {
            // e = S0 | S2 << 16, o = S1 | S3 << 16 (vectors 0..3), hi: 4..7
            uint32_t e_lo, o_lo, e_hi, o_hi;
            acc[t].finish(e_lo, o_lo, e_hi, o_hi);
            tot[t][0] += e_lo & 0xFFFFu;
            tot[t][1] += o_lo & 0xFFFFu;
            tot[t][2] += e_lo >> 16;
            tot[t][3] += o_lo >> 16;
            tot[t][4] += e_hi & 0xFFFFu;
            tot[t][5] += o_hi & 0xFFFFu;
            tot[t][6] += e_hi >> 16;
            tot[t][7] += o_hi >> 16;
        }
    }
    const int64_t v0 = b * kBlockVecs + 8 * lane;
    if (v0 < n) {  // ld >= n rounded up to 8: the two 16-byte stores stay in the row
#pragma unroll
        for (int t = 0; t < QT; ++t) {
            uint4 *dst = reinterpret_cast<uint4 *>(sums + t * ld + v0);
            __stcs(dst, make_uint4(tot[t][0], tot[t][1], tot[t][2], tot[t][3]));
            __stcs(dst + 1, make_uint4(tot[t][4], tot[t][5], tot[t][6], tot[t][7]));
        }
    }
}

__global__ void __launch_bounds__(kBatchThreads, 2) batch_scan_kernel(const uint8_t *__restrict__ plan) {
    __shared__ uint4 s_lut[kBatchLutEntries];
    __shared__ int s_task;
    BatchHeader *hdr = reinterpret_cast<BatchHeader *>(const_cast<uint8_t *>(plan));
    const int ntasks = hdr->ntasks;
    const BatchColl *colls = reinterpret_cast<const BatchColl *>(plan + hdr->colls_off);
    const BatchTask *tasks = reinterpret_cast<const BatchTask *>(plan + hdr->tasks_off);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) s_task = (int)atomicAdd(&hdr->counter, 1u);
        __syncthreads();
        const int ti = s_task;
        if (ti >= ntasks) break;
        const BatchTask t = tasks[ti];
        const BatchColl c = colls[t.coll];
        const int M = c.M;
        const int nl = (int)t.qt * t.nqt * M;
        const uint4 *src = c.luts + (int64_t)t.q0 * M;
        for (int i = tid; i < nl; i += kBatchThreads) s_lut[i] = __ldg(src + i);
        __syncthreads();
        const int units = t.nb * t.nqt;
        for (int u = warp; u < units; u += kBatchWarps) {
            const int tile = u % t.nqt;
            const int64_t b = (int64_t)t.b0 + u / t.nqt;
            const uint4 *lut = s_lut + tile * t.qt * M;
            uint16_t *dst = c.sums + ((int64_t)t.q0 + (int64_t)tile * t.qt) * c.ld;
            switch (t.qt) {
                case 16: batch_unit<16>(c.codes, b, M, lut, dst, c.ld, c.n, lane); break;
                case 8: batch_unit<8>(c.codes, b, M, lut, dst, c.ld, c.n, lane); break;
                case 4: batch_unit<4>(c.codes, b, M, lut, dst, c.ld, c.n, lane); break;
                case 2: batch_unit<2>(c.codes, b, M, lut, dst, c.ld, c.n, lane); break;
                default: batch_unit<1>(c.codes, b, M, lut, dst, c.ld, c.n, lane); break;
            }
        }
        __syncthreads();  // tables and s_task are reused by the next task
    }
}

// The uint32-sum tasks (collections with sum_bits = 32) in a persistent
// kernel of their own, so that the uint16 kernel's registers stay as they
// are; tables are staged in shared memory, or read from global memory when
// the task's tables are too large to stage.
__global__ void __launch_bounds__(kBatchThreads, 2) batch_scan_u32_kernel(const uint8_t *__restrict__ plan) {
    __shared__ uint4 s_lut[kBatchLutEntries];
    __shared__ int s_task;
    BatchHeader *hdr = reinterpret_cast<BatchHeader *>(const_cast<uint8_t *>(plan));
    const int ntasks = hdr->ntasks_wide;
    const BatchColl *colls = reinterpret_cast<const BatchColl *>(plan + hdr->colls_off);
    const BatchTask *tasks = reinterpret_cast<const BatchTask *>(plan + hdr->tasks_wide_off);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) s_task = (int)atomicAdd(&hdr->counter_wide, 1u);
        __syncthreads();
        const int ti = s_task;
        if (ti >= ntasks) break;
        const BatchTask t = tasks[ti];
        const BatchColl c = colls[t.coll];
        const int M = c.M;
        const uint4 *src = c.luts + (int64_t)t.q0 * M;
        if (!t.global_luts)
            for (int i = tid; i < (int)t.qt * t.nqt * M; i += kBatchThreads) s_lut[i] = __ldg(src + i);
        __syncthreads();
        const uint4 *tab = t.global_luts ? src : s_lut;
        const int units = t.nb * t.nqt;
        for (int u = warp; u < units; u += kBatchWarps) {
            const int tile = u % t.nqt;
            const int64_t b = (int64_t)t.b0 + u / t.nqt;
            const uint4 *lut = tab + tile * t.qt * M;
            uint32_t *dst = reinterpret_cast<uint32_t *>(c.sums) + ((int64_t)t.q0 + (int64_t)tile * t.qt) * c.ld;
            if (t.qt == 2) batch_unit_u32<2>(c.codes, b, M, lut, dst, c.ld, c.n, lane);
            else batch_unit_u32<1>(c.codes, b, M, lut, dst, c.ld, c.n, lane);
        }
        __syncthreads();  // tables and s_task are reused by the next task
    }
}

// ------------------------------------------------------------------ host planning
static int check_collection(const bolt_collection &c, int i) {
    BOLT_REQUIRE(c.n >= 0 && c.nq >= 0, BOLT_EINVAL, "collection %d: n=%lld nq=%lld", i, (long long)c.n,
                 (long long)c.nq);
    BOLT_REQUIRE(c.sum_bits == 0 || c.sum_bits == 16 || c.sum_bits == 32, BOLT_EINVAL,
                 "collection %d: sum_bits=%d not in {0, 16, 32}", i, c.sum_bits);
    const int mmax = c.sum_bits == 32 ? kMaxWideM : 256;
    BOLT_REQUIRE(c.M >= 1 && c.M <= mmax, BOLT_EINVAL, "collection %d: M=%d outside [1, %d] for %s sums", i, c.M,
                 mmax, c.sum_bits == 32 ? "uint32" : "uint16");
    BOLT_REQUIRE(c.qt_max == 0 || c.qt_max == 1 || c.qt_max == 2 || c.qt_max == 4 || c.qt_max == 8 ||
                     c.qt_max == 16,
                 BOLT_EINVAL, "collection %d: qt_max=%d not in {0,1,2,4,8,16}", i, c.qt_max);
    BOLT_REQUIRE(c.units_per_warp >= 0 && c.units_per_warp <= 64, BOLT_EINVAL,
                 "collection %d: units_per_warp=%d outside [0, 64]", i, c.units_per_warp);
    BOLT_REQUIRE(num_blocks(c.n) < (int64_t)1 << 31 && c.nq < (int64_t)1 << 31, BOLT_EINVAL,
                 "collection %d too large", i);
    if (c.n == 0 || c.nq == 0) return BOLT_OK;
    BOLT_REQUIRE(c.codes && c.luts && c.sums, BOLT_EINVAL, "collection %d: null pointer", i);
    BOLT_REQUIRE(aligned(c.codes, 16) && aligned(c.luts, 16) && aligned(c.sums, 16), BOLT_EINVAL,
                 "collection %d: codes, luts and sums must be 16-byte aligned", i);
    BOLT_REQUIRE(c.ld >= c.n && c.ld % 8 == 0, BOLT_EINVAL, "collection %d: ld=%lld must be >= n=%lld and a multiple of 8",
                 i, (long long)c.ld, (long long)c.n);
    return BOLT_OK;
}

static void plan_collection(const bolt_collection &c, int32_t ci, std::vector<BatchTask> &out) {
    if (c.n == 0 || c.nq == 0) return;
    const int M = c.M;
    const bool wide = c.sum_bits == 32;
    int qmax = c.qt_max ? c.qt_max : 8;
    if (wide && qmax > 2) qmax = 2;  // 8 uint32 totals per query in registers
    // tiles shrink until their tables can be staged (tables of more than
    // kBatchLutEntries rows are read from global memory at any tile size)
    if (M <= kBatchLutEntries)
        while (qmax > 1 && qmax * M > kBatchLutEntries) qmax >>= 1;
    const int upw = c.units_per_warp ? c.units_per_warp : 4;
    const int64_t nbt = num_blocks(c.n);
    // query tiles: qmax-sized, the remainder split into powers of two
    struct Group {
        int q0, qt, nqt;
    };
    std::vector<Group> groups;
    for (int64_t q = 0; q < c.nq;) {
        int qt = qmax;
        while (qt > c.nq - q) qt >>= 1;
        const int cap = std::max(1, kBatchLutEntries / (qt * M));
        const int cnt = (int)std::min<int64_t>((c.nq - q) / qt, cap);
        groups.push_back({(int)q, qt, cnt});
        q += (int64_t)qt * cnt;
    }
    std::vector<BatchTask> mine;
    for (const Group &g : groups) {
        const int64_t want = (int64_t)kBatchWarps * upw;
        int64_t nb = std::max<int64_t>(1, (want + g.nqt - 1) / g.nqt);
        nb = std::min<int64_t>(nb, nbt);
        nb = std::min<int64_t>(nb, 32767);
        for (int64_t b0 = 0; b0 < nbt; b0 += nb) {
            BatchTask t;
            t.coll = ci;
            t.q0 = g.q0;
            t.b0 = (int32_t)b0;
            t.nb = (int32_t)std::min<int64_t>(nb, nbt - b0);
            t.qt = (int16_t)g.qt;
            t.nqt = (int16_t)g.nqt;
            t.global_luts = g.qt * g.nqt * M > kBatchLutEntries ? 1 : 0;
            mine.push_back(t);
        }
    }
    // code-block range first, so the groups of one range run back to back
    std::stable_sort(mine.begin(), mine.end(), [](const BatchTask &a, const BatchTask &b) { return a.b0 < b.b0; });
    out.insert(out.end(), mine.begin(), mine.end());
}

static int build_plan_host(const bolt_collection *colls, int32_t ncoll, std::vector<uint8_t> &blob) {
    BOLT_REQUIRE(ncoll >= 0, BOLT_EINVAL, "ncoll=%d < 0", ncoll);
    BOLT_REQUIRE(ncoll == 0 || colls, BOLT_EINVAL, "null collection array");
    for (int i = 0; i < ncoll; ++i) {
        int rc = check_collection(colls[i], i);
        if (rc) return rc;
    }
    // largest collections first (work = n * nq * M): long tasks start early
    std::vector<int> order(ncoll);
    for (int i = 0; i < ncoll; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double wa = (double)colls[a].n * (double)colls[a].nq * colls[a].M;
        const double wb = (double)colls[b].n * (double)colls[b].nq * colls[b].M;
        return wa > wb;
    });
    std::vector<BatchTask> tasks, tasks_wide;
    for (int i : order) plan_collection(colls[i], i, colls[i].sum_bits == 32 ? tasks_wide : tasks);
    BOLT_REQUIRE(tasks.size() + tasks_wide.size() < (size_t)1 << 31, BOLT_EINVAL, "too many tasks");
    const int64_t colls_off = sizeof(BatchHeader);
    const int64_t tasks_off = colls_off + (int64_t)ncoll * (int64_t)sizeof(BatchColl);
    const int64_t tasks_wide_off = tasks_off + (int64_t)tasks.size() * (int64_t)sizeof(BatchTask);
    blob.assign((size_t)(tasks_wide_off + (int64_t)tasks_wide.size() * (int64_t)sizeof(BatchTask)), 0);
    BatchHeader h{};
    h.ntasks = (int32_t)tasks.size();
    h.ncoll = ncoll;
    h.colls_off = colls_off;
    h.tasks_off = tasks_off;
    h.tasks_wide_off = tasks_wide_off;
    h.ntasks_wide = (int32_t)tasks_wide.size();
    memcpy(blob.data(), &h, sizeof(h));
    for (int i = 0; i < ncoll; ++i) {
        BatchColl r{};
        r.codes = reinterpret_cast<const uint32_t *>(colls[i].codes);
        r.luts = reinterpret_cast<const uint4 *>(colls[i].luts);
        r.sums = colls[i].sums;
        r.n = colls[i].n;
        r.ld = colls[i].ld;
        r.M = colls[i].M;
        memcpy(blob.data() + colls_off + (int64_t)i * sizeof(BatchColl), &r, sizeof(r));
    }
    if (!tasks.empty()) memcpy(blob.data() + tasks_off, tasks.data(), tasks.size() * sizeof(BatchTask));
    if (!tasks_wide.empty())
        memcpy(blob.data() + tasks_wide_off, tasks_wide.data(), tasks_wide.size() * sizeof(BatchTask));
    return BOLT_OK;
}

static int batch_grid(int *grid) {
    static std::mutex mu;
    static int cache[64] = {0};
    int dev = 0;
    BOLT_CUDA(cudaGetDevice(&dev));
    BOLT_REQUIRE(dev >= 0 && dev < 64, BOLT_EUNSUPPORTED, "device %d", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (cache[dev] == 0) {
        int per_sm = 0;
        BOLT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_scan_kernel, kBatchThreads, 0));
        cache[dev] = std::max(1, per_sm) * std::max(1, device_sm_count());
    }
    *grid = cache[dev];
    return BOLT_OK;
}

// Plans with uint32-sum tasks, recorded when a plan is uploaded (a plan not
// recorded here, e.g. one copied by the caller, runs both kernels: the wide
// one then finds no tasks).
static std::mutex g_plans_mu;
static std::map<const void *, bool> g_plan_wide;

static int run_plan(const void *plan, cudaStream_t s) {
    int grid = 0;
    int rc = batch_grid(&grid);
    if (rc) return rc;
    bool wide = true;
    {
        std::lock_guard<std::mutex> lk(g_plans_mu);
        auto it = g_plan_wide.find(plan);
        if (it != g_plan_wide.end()) wide = it->second;
    }
    BOLT_CUDA(cudaMemsetAsync(const_cast<void *>(plan), 0, 2 * sizeof(unsigned int), s));
    batch_scan_kernel<<<grid, kBatchThreads, 0, s>>>(reinterpret_cast<const uint8_t *>(plan));
    rc = check_launch("batch_scan_kernel");
    if (rc || !wide) return rc;
    batch_scan_u32_kernel<<<grid, kBatchThreads, 0, s>>>(reinterpret_cast<const uint8_t *>(plan));
    return check_launch("batch_scan_u32_kernel");
}

static int upload_plan(const std::vector<uint8_t> &blob, void *plan, int64_t plan_bytes, cudaStream_t s) {
    BOLT_REQUIRE(plan, BOLT_EINVAL, "null plan");
    BOLT_REQUIRE(aligned(plan, 256), BOLT_EINVAL, "plan must be 256-byte aligned");
    BOLT_REQUIRE(plan_bytes >= (int64_t)blob.size(), BOLT_EINVAL, "plan_bytes=%lld < %lld needed",
                 (long long)plan_bytes, (long long)blob.size());
    BOLT_CUDA(cudaMemcpyAsync(plan, blob.data(), blob.size(), cudaMemcpyHostToDevice, s));
    BOLT_CUDA(cudaStreamSynchronize(s));
    BatchHeader h;
    memcpy(&h, blob.data(), sizeof(h));
    std::lock_guard<std::mutex> lk(g_plans_mu);
    g_plan_wide[plan] = h.ntasks_wide > 0;
    return BOLT_OK;
}

}  // namespace bolt

extern "C" {

int64_t bolt_batch_plan_bytes(const bolt_collection *colls_host, int32_t ncoll) {
    bolt::clear_error();
    std::vector<uint8_t> blob;
    int rc = bolt::build_plan_host(colls_host, ncoll, blob);
    if (rc) return -(int64_t)rc;
    return (int64_t)blob.size();
}

int bolt_batch_plan(const bolt_collection *colls_host, int32_t ncoll, void *plan, int64_t plan_bytes,
                    void *stream) {
    bolt::clear_error();
    std::vector<uint8_t> blob;
    int rc = bolt::build_plan_host(colls_host, ncoll, blob);
    if (rc) return rc;
    return bolt::upload_plan(blob, plan, plan_bytes, (cudaStream_t)stream);
}

int bolt_scan_batched(const void *plan, void *stream) {
    bolt::clear_error();
    BOLT_REQUIRE(plan && bolt::aligned(plan, 256), BOLT_EINVAL, "plan must be a 256-byte aligned device pointer");
    return bolt::run_plan(plan, (cudaStream_t)stream);
}

int bolt_batch_autotune(bolt_collection *colls_host, int32_t ncoll, void *stream, float *tuning_ms_host) {
    bolt::clear_error();
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint8_t> blob;
    int rc = bolt::build_plan_host(colls_host, ncoll, blob);
    if (rc) return rc;
    static const int kQts[3] = {4, 8, 16};
    static const int kUpws[4] = {1, 2, 4, 8};
    // largest plan any mix of candidates can need: every collection at its
    // own largest task count
    int64_t max_bytes = (int64_t)blob.size();
    {
        int64_t tasks = 0;
        for (int i = 0; i < ncoll; ++i) {
            size_t most = 0;
            for (int qt : kQts)
                for (int upw : kUpws) {
                    bolt_collection c = colls_host[i];
                    c.qt_max = qt;
                    c.units_per_warp = upw;
                    std::vector<bolt::BatchTask> t;
                    bolt::plan_collection(c, i, t);
                    most = std::max(most, t.size());
                }
            tasks += (int64_t)most;
        }
        max_bytes = std::max<int64_t>(max_bytes, (int64_t)sizeof(bolt::BatchHeader) +
                                                     (int64_t)ncoll * (int64_t)sizeof(bolt::BatchColl) +
                                                     tasks * (int64_t)sizeof(bolt::BatchTask));
    }
    void *plan = nullptr;
    BOLT_CUDA(cudaMalloc(&plan, (size_t)max_bytes));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        {
            std::lock_guard<std::mutex> lk(bolt::g_plans_mu);
            bolt::g_plan_wide.erase(plan);
        }
        cudaFree(plan);
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        bolt::set_error("cudaEventCreate failed");
        return BOLT_ECUDA;
    }
    // time one configuration of the given collections: best of 3 launches
    auto time_plan = [&](const std::vector<bolt_collection> &cs, float *ms_out) -> int {
        std::vector<uint8_t> b;
        int r = bolt::build_plan_host(cs.data(), (int32_t)cs.size(), b);
        if (r) return r;
        r = bolt::upload_plan(b, plan, max_bytes, s);
        if (r) return r;
        r = bolt::run_plan(plan, s);  // warm-up
        if (r) return r;
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            BOLT_CUDA(cudaEventRecord(e0, s));
            r = bolt::run_plan(plan, s);
            if (r) return r;
            BOLT_CUDA(cudaEventRecord(e1, s));
            BOLT_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            BOLT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            best = std::min(best, ms);
        }
        *ms_out = best;
        return BOLT_OK;
    };
    // one codebook count at a time: its collections alone
    std::vector<int> Ms;
    for (int i = 0; i < ncoll; ++i)
        if (std::find(Ms.begin(), Ms.end(), colls_host[i].M) == Ms.end()) Ms.push_back(colls_host[i].M);
    for (int M : Ms) {
        std::vector<int> idx;
        for (int i = 0; i < ncoll; ++i)
            if (colls_host[i].M == M) idx.push_back(i);
        int best_qt = 8, best_upw = 4;
        float best_ms = 1e30f;
        for (int qt : kQts) {
            if (qt > 1 && qt * M > bolt::kBatchLutEntries) continue;
            for (int upw : kUpws) {
                std::vector<bolt_collection> sub;
                for (int i : idx) {
                    bolt_collection c = colls_host[i];
                    c.qt_max = qt;
                    c.units_per_warp = upw;
                    sub.push_back(c);
                }
                float ms = 0.0f;
                rc = time_plan(sub, &ms);
                if (rc) {
                    cleanup();
                    return rc;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best_qt = qt;
                    best_upw = upw;
                }
            }
        }
        for (int i : idx) {
            colls_host[i].qt_max = best_qt;
            colls_host[i].units_per_warp = best_upw;
        }
    }
    if (tuning_ms_host) {
        std::vector<bolt_collection> all(colls_host, colls_host + ncoll);
        float ms = 0.0f;
        rc = time_plan(all, &ms);
        if (rc) {
            cleanup();
            return rc;
        }
        *tuning_ms_host = ms;
    }
    cleanup();
    return BOLT_OK;
}

}  // extern "C"
