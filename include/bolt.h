/*
 * bolt.h -- C ABI of the GB300 (sm_103a) Bolt library, libbolt.so.
 *
 * Bolt (Blalock & Guttag, "Bolt: Accelerated Data Mining with Fast Vector
 * Compression", KDD'17) approximates a distance d(q, x) = f(sum_j delta(q_j,
 * x_j)) (Sec. 1.1) by
 *   h(x): M 4-bit codes, the nearest of K = 16 centroids per subspace
 *         (Sec. 3.1 encoding function h; K = 16 from Sec. 3.2, change 1),
 *   g(q): an M x 16 table of subvector-to-centroid distances quantized to
 *         uint8 by beta_m(y) = clamp(floor(a (y - b_m)), 0, 255) (Sec. 3.2),
 *   d^ :  the sum over m of the table entries the codes pick (Sec. 3.1,
 *         approximate distance as a sum of table entries).
 *
 * Conventions for every entry point
 *  - Array arguments are DEVICE pointers owned by the caller unless the
 *    parameter name ends in _host.  The library never frees or keeps them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless stated.
 *  - Every call returns BOLT_OK (0) or an error code; no exception crosses
 *    the ABI.  bolt_last_error() returns this thread's last message.
 *  - Sizes: n database vectors, J dims, M codebooks (J % M == 0,
 *    1 <= M <= 256, s = J/M dims per subspace, subspace m owning dims
 *    [m*s, (m+1)*s), Sec. 3.1 "consecutive indices"), nq queries.  The
 *    entry points that need no uint16 sum -- layout, encode, bolt_build_luts,
 *    bolt_scan_u32, bolt_dequantize_u32 -- accept 1 <= M <= 4096; the rest
 *    return BOLT_EUNSUPPORTED for M > 256.
 *  - Dense float inputs are row-major fp32 (X: n x J, Q: nq x J).
 *  - centroids: fp32 [M][16][s].
 *  - Codes use the BLOCKED layout: vectors are grouped in blocks of 256; block
 *    b stores M rows of 128 bytes, row m holding the 4-bit codes of codebook m
 *    for vectors 256b .. 256b+255; within a row, little-endian 32-bit word w
 *    holds vectors 256b + 8w + i in bits [4i, 4i+4), i = 0..7.  Vectors past
 *    n in the last block are code 0 and never reported.  Size:
 *    bolt_codes_bytes(n, M) = ceil(n/256) * M * 128 bytes (16-byte aligned
 *    base required).
 *  - luts: uint8 [nq][M][16] (16 contiguous entries per query and codebook).
 *  - Scan sums are exact integers stored as uint16 (255*M <= 65280), or
 *    as uint32 by bolt_scan_u32 for any M up to 4096.
 *  - Top-k order: L2 ascending sum, dot descending sum, ties to the lower
 *    vector index; rows with k > n are padded with index -1 and sum 0.
 */
#ifndef BOLT_H_
#define BOLT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BOLT_OK 0
#define BOLT_EINVAL 1       /* bad pointer, shape, alignment or argument */
#define BOLT_EUNSUPPORTED 2 /* J % M != 0, M > 256, k too large, ... */
#define BOLT_ENOMEM 3       /* workspace too small or allocation failed */
#define BOLT_ECUDA 4        /* a CUDA runtime call or launch failed */
#define BOLT_ETIMEOUT 5     /* a bounded device wait gave up */

#define BOLT_METRIC_L2 0  /* delta = squared difference, f = sqrt (Sec. 1.1) */
#define BOLT_METRIC_DOT 1 /* delta = product, f = identity (Sec. 1.1) */
#define BOLT_METRIC_L1 2  /* delta = absolute difference, f = identity: the L_p family of
                             Sec. 1.1 with p = 1 (f = r^(1/p) is monotone, so top-k ranks
                             by the sum, ascending, as for L2) */
#define BOLT_METRIC_LP 3  /* delta = |difference|^p for a real p > 0 (tables built by
                             bolt_build_luts_lp): the L_p family of Sec. 1.1; top-k ranks by
                             the sum, ascending.  Accepted by the top-k, merge and filter
                             calls; the tables come from the _lp entry points */

#define BOLT_PREC_FP32 0         /* canonical fp32 encoder */
#define BOLT_PREC_BF16_RECHECK 1 /* tensor-core bf16 scores + fp32 re-check */

/* Thread-local message for the last failing call on this thread ("" if none).
 * Valid until the next call on the same thread. */
const char *bolt_last_error(void);

/* Library version string. */
const char *bolt_version(void);

/* ---------------------------------------------------------------- layout
 * Size in bytes of the blocked code array for n vectors and M codebooks
 * (ceil(n/256) * M * 128); -1 for invalid arguments.  Host only. */
int64_t bolt_codes_bytes(int64_t n, int32_t M);

/* Convert row-major codes (n x M bytes, each 0..15) to the blocked layout.
 * Codes are not range-checked on the device: only the low nibble of each
 * byte is stored.  blocked: bolt_codes_bytes(n, M) bytes, fully written
 * (padding codes are 0). */
int bolt_pack_codes(const uint8_t *rowmajor, int64_t n, int32_t M,
                    uint8_t *blocked, void *stream);

/* Inverse of bolt_pack_codes: blocked -> row-major n x M bytes (0..15). */
int bolt_unpack_codes(const uint8_t *blocked, int64_t n, int32_t M,
                      uint8_t *rowmajor, void *stream);

/* ---------------------------------------------------------------- encode h
 * Sec. 3.1, h(x)_m = argmin_i d(c_i^(m), x^(m)) over K = 16 centroids.
 * The canonical distance of (x, m, k) is the fp32 sum over the subspace's
 * dims, in dim order, of acc = fmaf(t, t, acc), t = x_j - c_j, from 0; ties
 * go to the lowest k.
 * precision BOLT_PREC_FP32 computes exactly that.  BOLT_PREC_BF16_RECHECK
 * scores ||c||^2 - 2 x.c on tcgen05 tensor cores: x and c are each split
 * into a bf16 high part and a bf16 residual, three bf16 MMAs (hi.hi, hi.lo,
 * lo.hi) accumulate in fp32, and every centroid whose score lies within a
 * rigorous error margin of the best is re-evaluated with the canonical fp32
 * distance, so its codes equal BOLT_PREC_FP32's.  It needs J % 32 == 0 and
 * s = J / M in {4, 8, 16, 32}; other shapes run the fp32 kernel instead.
 * X: n x J fp32 (16-byte aligned); codes: blocked, bolt_codes_bytes(n, M).
 * n_rechecked (nullable, device int64): set to the number of (vector,
 * subspace) pairs that took the fp32 re-check (0 for BOLT_PREC_FP32), or
 * to -1 if the tensor-core kernel gave up waiting on its own copies; the
 * codes are then invalid (the launch itself is asynchronous, so this is
 * the only report of that failure). */
int bolt_encode(const float *X, int64_t n, int32_t J, int32_t M,
                const float *centroids, int32_t precision, uint8_t *codes,
                int64_t *n_rechecked, void *stream);

/* ---------------------------------------------------------------- LUT g
 * Sec. 3.1 query encoding D_im = delta(q^(m), c_i^(m)), then Sec. 3.2
 * quantization beta_m.  L2: fp32 acc = fmaf(t, t, acc), t = q_j - c_j; dot:
 * acc = fmaf(q_j, c_j, acc), both in dim order from 0.  Quantization: t =
 * (y - b_m) then t * a, two fp32 roundings, floor, clamp to [0, 255], NaN to
 * 0.  a: scale (host value); b_host: M offsets in HOST memory (read before
 * the call returns; for M > 256 they are copied to a stream-ordered device
 * buffer, so such a call cannot be captured in a CUDA graph).
 * luts: nq x M x 16 uint8.  luts_f32 (nullable): the unquantized table
 * nq x M x 16 fp32 ("Bolt No Quantize", Sec. 4.2). */
int bolt_build_luts(const float *Q, int64_t nq, int32_t J, int32_t M,
                    const float *centroids, int32_t metric, float a,
                    const float *b_host, uint8_t *luts, float *luts_f32,
                    void *stream);

/* L_p tables for a real exponent p > 0 (the d = f(sum delta) family of
 * Sec. 1.1 with delta = |q_j - c_j|^p): D[q][m][k] = sum over the dims of
 * subspace m, in order from the first, of powf(|q_j - c_kj|, p) (CUDA's
 * powf, fp32 adds), then quantized by beta_m exactly as bolt_build_luts
 * does.  The fp32 entries follow the library powf, whose results can differ
 * from another implementation's in the last bits.  Same arguments as
 * bolt_build_luts otherwise (M up to 4096); rank the sums with
 * BOLT_METRIC_LP.  BOLT_EINVAL unless p > 0 and finite. */
int bolt_build_luts_lp(const float *Q, int64_t nq, int32_t J, int32_t M,
                       const float *centroids, float p, float a,
                       const float *b_host, uint8_t *luts, float *luts_f32,
                       void *stream);

/* ---------------------------------------------------------------- scan d^
 * Sec. 3.1 approximate distance: sums[q][i] = sum_m luts[q][m][code_m(x_i)],
 * exact, as uint16.  sums: nq x n.  The two names compute the same integer
 * sums; they differ only in how top-k and dequantization read them. */
int bolt_scan_l2(const uint8_t *codes, int64_t n, int32_t M,
                 const uint8_t *luts, int64_t nq, uint16_t *sums, void *stream);
int bolt_scan_dot(const uint8_t *codes, int64_t n, int32_t M,
                  const uint8_t *luts, int64_t nq, uint16_t *sums, void *stream);

/* The same exact sums for 1 <= M <= 4096 codebooks, as uint32 (the uint16
 * form holds them only while 255 * M <= 65535).  The codebooks are summed in
 * chunks of 256 in the uint16 form and the chunk sums added in 32 bits.
 * sums: nq x n uint32, device; codes and luts 16-byte aligned. */
int bolt_scan_u32(const uint8_t *codes, int64_t n, int32_t M,
                  const uint8_t *luts, int64_t nq, uint32_t *sums, void *stream);

/* "Bolt No Quantize" (the Sec. 4.2 ablation that skips the 8-bit tables):
 * out[q][i] = sum over m = 0..M-1 of luts_f32[q][m][code_m(x_i)], summed in
 * codebook order from 0.0f with one fp32 add (round to nearest) per
 * codebook.  luts_f32: nq x M x 16 fp32 (the `luts_f32` output of
 * bolt_build_luts); out: nq x n fp32.  Device pointers, codes 16-byte
 * aligned. */
int bolt_scan_float(const uint8_t *codes, int64_t n, int32_t M, const float *luts_f32,
                    int64_t nq, float *out, void *stream);

/* ---------------------------------------------------------------- top-k
 * Fused scan + exact top-k (nearest neighbours for L2, maximum inner product
 * for dot; Sec. 1.2 and Sec. 4.5 use these searches).  out_sums: nq x k
 * uint16, out_idx: nq x k int64, best first.  1 <= k <= 1024.
 * workspace: device scratch of at least bolt_topk_workspace_bytes(n, M, nq,
 * k) bytes, 256-byte aligned, or NULL to let the library allocate and free
 * it stream-ordered (cudaMallocAsync/cudaFreeAsync) inside the call.
 * Calls sharing one workspace must not overlap on the GPU.
 * Timed-out waits: every wait of the kernel on its own bulk copies is bounded
 * (1 s).  If one gives up (only on a GPU stalled or preempted for that
 * long), the query's row comes back with every index -2 (sums undefined).
 * The call has already returned BOLT_OK by then, since the failure happens
 * on the GPU after the launch: callers that read results check for index -2
 * in column 0 and treat the row as failed (the Python binding's
 * check_topk() and its serving loop do). */
int64_t bolt_topk_workspace_bytes(int64_t n, int32_t M, int64_t nq, int32_t k);
int bolt_topk(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts,
              int64_t nq, int32_t k, int32_t metric, uint16_t *out_sums,
              int64_t *out_idx, void *workspace, int64_t workspace_bytes,
              void *stream);

/* Fused scan + exact top-k for 1 <= M <= 4096 codebooks over uint32 sums
 * (Sec. 3.1: the approximate distance sums all M tables; bolt_topk's uint16
 * sums hold it only up to M = 256).  Same order as bolt_topk -- L2 and L1
 * ascending, dot descending, ties to the lower vector index, k > n padded
 * with index -1 and sum 0 -- with the sums of the best k as uint32.
 * out_sums: nq x k uint32, out_idx: nq x k int64, 1 <= k <= 1024,
 * n < 2^31, nq <= 65535.  workspace: device scratch of at least
 * bolt_topk_u32_workspace_bytes(n, M, nq, k) bytes (it holds every sum,
 * 4 n nq bytes, plus histograms and k candidates per query), 256-byte
 * aligned, or NULL to allocate and free it stream-ordered inside the call.
 * Calls sharing one workspace must not overlap on the GPU.  The kernels
 * have no device waits. */
int64_t bolt_topk_u32_workspace_bytes(int64_t n, int32_t M, int64_t nq, int32_t k);
int bolt_topk_u32(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts,
                  int64_t nq, int32_t k, int32_t metric, uint32_t *out_sums,
                  int64_t *out_idx, void *workspace, int64_t workspace_bytes,
                  void *stream);

/* Allocation-free variant of bolt_topk (the paper has no counterpart: this is
 * an interface for callers that may not allocate device memory during the
 * call -- e.g. code issuing work while a CUDA graph is being captured under a
 * strict capture mode, latency-critical serving loops that keep allocator
 * calls off the request path, or embedders whose own allocator owns the GPU
 * heap).  Same arguments, results and order as bolt_topk, without the
 * workspace: the scratch space is a 4 MiB array compiled into libbolt.so,
 * which every GPU that loads the library keeps until the process exits.
 *  - The call makes no cudaMalloc/cudaFree or other allocation; it zeroes the
 *    parts of the array that must start at zero with cudaMemsetAsync.
 *  - Requests whose scratch need (bolt_topk_workspace_bytes(n, M, nq, k))
 *    exceeds 4 MiB fail with BOLT_ENOMEM and a message; split the queries.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture on that device.
 *  - The address is cached per device for the life of the process; it is
 *    invalid after cudaDeviceReset or anything else that destroys the
 *    device's primary context, so do not call this entry point after that.
 *  - All calls share the one array: calls that may overlap on the GPU (other
 *    streams, other host threads) race and give wrong results; serialize them
 *    (one stream, or events).
 *  - A timed-out wait marks the query's row with index -2, as in bolt_topk. */
int bolt_topk_noalloc(const uint8_t *codes, int64_t n, int32_t M, const uint8_t *luts,
                      int64_t nq, int32_t k, int32_t metric, uint16_t *out_sums,
                      int64_t *out_idx, void *stream);

/* ---------------------------------------------------------------- batched scan
 * The Sec. 3.1 scan of many independent collections -- each with its own
 * encoded database, codebook count and query tables -- in ONE persistent
 * launch.  (The paper scans one database at a time; batching collections is
 * a serving form of the same sums.)  Results are exactly those of
 * bolt_scan_l2 on each collection alone.
 *
 * One bolt_collection per collection; all pointers are device memory:
 *   codes : blocked layout of n vectors and M codebooks (16-byte aligned)
 *   luts  : nq x M x 16 uint8 tables (16-byte aligned)
 *   sums  : nq rows of ld sums, sums[q * ld + i] for i < n (16-byte
 *           aligned; ld >= n and a multiple of 8), uint16 or, with
 *           sum_bits = 32, uint32 (pass the uint32 buffer cast to uint16_t*).
 *           Entries i in [n, ld) of each row may be overwritten with padding
 *           sums.
 *   n, nq : sizes (either may be 0: the collection then has no work)
 *   M     : 1 <= M <= 256 with uint16 sums; up to 4096 with uint32 sums
 *           (codebooks summed in groups of 256, each group exact in 16 bits)
 *   qt_max: queries one warp accumulates in registers per pass over a code
 *           block: 1, 2, 4, 8 or 16; 0 = library default (8)
 *   units_per_warp: (block, query-tile) units each warp of a CTA takes per
 *           task, 1..64; 0 = library default (4)
 *   sum_bits: 0 or 16 = uint16 sums, 32 = uint32 sums (any M; required for
 *           M > 256, where a uint16 sum could overflow); uint32 collections
 *           take at most 2 queries per pass, and above 1024 codebooks read
 *           their tables from global memory instead of staging them
 * qt_max and units_per_warp change speed only, never results;
 * bolt_batch_autotune chooses them by timing. */
typedef struct bolt_collection {
    const uint8_t *codes;
    const uint8_t *luts;
    uint16_t *sums;
    int64_t n;
    int64_t nq;
    int64_t ld;
    int32_t M;
    int32_t qt_max;
    int32_t units_per_warp;
    int32_t sum_bits; /* 0 or 16: uint16 sums; 32: uint32 sums */
} bolt_collection;

/* Bytes of device memory the plan for these collections needs (host only;
 * < 0 with bolt_last_error set on invalid input). */
int64_t bolt_batch_plan_bytes(const bolt_collection *colls_host, int32_t ncoll);

/* Build the task list for colls_host[0..ncoll) on the host and copy it into
 * `plan` (device, 256-byte aligned, plan_bytes >= bolt_batch_plan_bytes).
 * Tasks are ordered largest collection first, and within a collection by
 * code-block range, so that the query tiles of one range run close together
 * and re-read its codes from L2.  Synchronizes `stream` (the copy comes from
 * pageable host memory): build plans before any stream capture.  The plan
 * holds the collections' pointers; it stays valid while they do. */
int bolt_batch_plan(const bolt_collection *colls_host, int32_t ncoll, void *plan,
                    int64_t plan_bytes, void *stream);

/* Run a plan: one stream-ordered memset of its task counter and one
 * persistent launch (one CTA per resident slot on every SM; CTAs take tasks
 * from the counter).  Capturable in a CUDA graph.  Launches of one plan must
 * not overlap on the GPU (they share the counter). */
int bolt_scan_batched(const void *plan, void *stream);

/* Choose qt_max and units_per_warp for every collection by timing
 * bolt_scan_batched on the collections themselves, one codebook count M at
 * a time, over the candidates qt_max in {4, 8, 16} (capped by the table
 * space) x units_per_warp in {1, 2, 4, 8}; writes the fastest into
 * colls_host.  Overwrites the collections' sums; allocates and frees a
 * scratch plan and synchronizes `stream`.  tuning_ms_host (nullable)
 * receives the best time of the whole batch with the chosen settings. */
int bolt_batch_autotune(bolt_collection *colls_host, int32_t ncoll, void *stream,
                        float *tuning_ms_host);

/* ---------------------------------------------------------------- shard merge
 * Top-k of a database split into disjoint row ranges (shards): every
 * distance depends on one vector's codes only (Sec. 3.1), so the global
 * top-k is the best k of the union of the shards' own top-k lists.
 * sums, idx: nshard x nq x k, shard-major; list (a, q) is bolt_topk's output
 * for query q on shard a (best first, local indices, padding index -1;
 * index -2 marks a failed wait and makes the merged row -2).
 * offsets: nshard int64 (device), global index of each shard's row 0.
 * out_sums / out_idx: nq x k, the same order and padding as bolt_topk over
 * the whole database, so the merge is bit-identical to the unsharded
 * result.  All pointers are device memory.  M and metric as in bolt_topk
 * (dot lists are merged by largest sum). */
int bolt_topk_merge(const uint16_t *sums, const int64_t *idx, const int64_t *offsets,
                    int32_t nshard, int64_t nq, int32_t k, int32_t M, int32_t metric,
                    uint16_t *out_sums, int64_t *out_idx, void *stream);

/* ---------------------------------------------------------------- online changes
 * Databases that change while in use (Sec. 1.3: vectors are added and
 * changed online).  bolt_write_codes writes the codes of `count` vectors --
 * rowmajor: count x M bytes, each 0..15 (e.g. bolt_unpack_codes of a
 * bolt_encode result) -- into rows[i] of a blocked code array with room for
 * n_cap vectors (bolt_codes_bytes(n_cap, M) bytes).  rows: count distinct
 * int64 (device).  A row outside [0, n_cap) or a code above 15 is not
 * written and the call returns BOLT_EINVAL.  Synchronizes `stream` (to
 * report bad rows).  Calls that scan the array must not overlap it. */
int bolt_write_codes(const uint8_t *rowmajor, int64_t count, int32_t M, const int64_t *rows,
                     uint8_t *blocked, int64_t n_cap, void *stream);

/* Drop deleted vectors from top-k lists: for each of nq lists (in_sums /
 * in_idx: nq x k_in, best first, as from bolt_topk), the first k_out
 * entries whose index i is live (bit i of dead_bits clear; indices at or
 * past n_bits are live), in list order, padded with index -1 and sum 0.
 * If at most D rows are dead, the top k_out of the live rows is the
 * filtered top (k_out + D) of all rows.  A list holding index -2 (a failed
 * wait) comes out all -2.  Device pointers. */
int bolt_topk_filter(const uint16_t *in_sums, const int64_t *in_idx, int64_t nq, int32_t k_in,
                     const uint32_t *dead_bits, int64_t n_bits, int32_t k_out, uint16_t *out_sums,
                     int64_t *out_idx, void *stream);

/* ---------------------------------------------------------------- dequantize
 * Sec. 3.2: the per-table reconstructions beta_m/a + b_m sum to
 * S * (1/a) + sum_m b_m.  Host helper (fp64, no GPU): inv_a =
 * (float)(1/(double)a), bias = (float)(sum_m (double)b_host[m]). */
int bolt_dequant_params(float a, const float *b_host, int32_t M, float *inv_a_host,
                        float *bias_host);

/* out[i] = fp32(fp32((float)S[i] * inv_a) + bias), count values. */
int bolt_dequantize(const uint16_t *S, int64_t count, float inv_a, float bias,
                    float *out, void *stream);

/* The same for uint32 sums (bolt_scan_u32; S < 2^24 converts exactly). */
int bolt_dequantize_u32(const uint32_t *S, int64_t count, float inv_a, float bias,
                        float *out, void *stream);

/* ---------------------------------------------------------------- matmul
 * Sec. 4.4 approximate matrix product: rows of A are queries with dot
 * tables, codesB is the encoded database; out[i][j] is the dequantized
 * approximate A_i . B_j.  A: rows x J fp32, codesB: blocked (n vectors),
 * out: rows x n fp32. */
int bolt_approx_matmul(const float *A, int64_t rows, int32_t J,
                       const uint8_t *codesB, int64_t n, int32_t M,
                       const float *centroids, float a, const float *b_host,
                       float *out, void *stream);

/* ---------------------------------------------------------------- fit
 * Offline phase (Sec. 1.3).  k-means (Sec. 3.1 background) with exactly
 * `iters` Lloyd iterations: assignment by the canonical fp32 encoder, means
 * accumulated in fp64 and rounded to fp32, an empty cluster keeps its
 * centroid; init_rows_host: 16 row indices whose subvectors seed every
 * codebook.  If Qtrain != NULL the quantizer for `metric` is fitted as in
 * bolt_fit_quantizer.  Blocking: returns after the work is done.
 * centroids: output M x 16 x s fp32 (device).  a_host, b_host: outputs
 * (ignored when Qtrain is NULL). */
int bolt_fit_codebooks(const float *X, int64_t n, int32_t J, int32_t M,
                       int32_t iters, const int64_t *init_rows_host,
                       const float *Qtrain, int64_t nqt, int32_t metric,
                       float *centroids, float *a_host, float *b_host,
                       void *stream);

/* Sec. 3.2 quantizer fit over the tables of nqt training queries, in fp64 on
 * the GPU: b_m = lower-rank empirical alpha-quantile of table m (entry
 * floor(alpha*(16*nqt-1)) of the sorted table), a = 255 / (entry
 * floor((1-alpha)*(16*nqt*M-1)) of the sorted pooled offsets y - b_m) (a = 1
 * if that is <= 0); alpha in {0,.001,.002,.005,.01,.02,.05,.1} minimizing the
 * mean squared reconstruction error, ties to the smaller alpha.  Outputs
 * rounded to fp32.  alpha_idx_host (nullable).  Blocking. */
int bolt_fit_quantizer(const float *Qtrain, int64_t nqt, int32_t J, int32_t M,
                       const float *centroids, int32_t metric, float *a_host,
                       float *b_host, int32_t *alpha_idx_host, void *stream);

/* The same fit over the L_p tables of bolt_build_luts_lp (exponent p > 0). */
int bolt_fit_quantizer_lp(const float *Qtrain, int64_t nqt, int32_t J, int32_t M,
                          const float *centroids, float p, float *a_host,
                          float *b_host, int32_t *alpha_idx_host, void *stream);

/* ---------------------------------------------------------------- timeout-path tests
 * Sets the time limit, in nanoseconds, of the waits of the streaming top-k
 * kernel and of the tensor-core encoder for their own data (bulk copies of
 * codes, the encoder's ring of copies, conversions and MMAs); ns = 0
 * restores the default of 1 s.  With a limit of a few nanoseconds those waits
 * give up at once (limits below 1 us are enforced by non-blocking polls, as
 * a blocking wait may itself outlast them) and the calls take their failure
 * path -- top-k rows of
 * index -2, the encoder's n_rechecked = -1 -- while the waits that drain
 * copies and MMAs in flight before a CTA exits keep their own 0.1 s bound.
 * For tests of that path; process-wide, not thread-safe with concurrent
 * calls.  (The paper has no counterpart.) */
int bolt_set_wait_limit_ns(uint64_t ns);

/* ---------------------------------------------------------------- measurement probes
 * Roofline denominators for the scan, measured on the device that is
 * current (the paper has no counterpart; these compute no Bolt result).
 *
 * bolt_probe_int_lanes: integer-ALU lanes per clock per SM, from clock64()
 * around a loop of independent byte permutes (prmt, the scan's lookup
 * instruction) on one CTA of 1024 threads per SM.  Synchronous; allocates
 * and frees 264 bytes of device memory.
 *
 * bolt_probe_lookup_core: microseconds per pass of the scan's lookup core
 * (M = 16, blocked layout, the streaming kernel's bulk-copy rings) over n
 * vectors of codes with the 16 x 16 uint8 tables luts, keeping only the
 * smallest sum: the time below which no one-query fused scan + top-k on
 * this core can go.  codes and luts are device pointers, 16-byte aligned;
 * reps timed passes after two warm-up passes, on `stream`, synchronized
 * before return.  BOLT_ETIMEOUT if a bounded wait gave up. */
int bolt_probe_int_lanes(double *lanes_per_clk_per_sm);
int bolt_probe_lookup_core(const uint8_t *codes, int64_t n, const uint8_t *luts, int32_t reps,
                           float *us_per_pass, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BOLT_H_ */
