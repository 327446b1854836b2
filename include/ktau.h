/*
 * ktau.h -- C ABI of the GB300 all-pairs Kendall tau-b library (libktau.so).
 *
 * Method: Liu, Pan, Green, Aluru, "Parallelized Kendall's Tau Coefficient Computation via
 * SIMD Vectorized Sorting On Many-Integrated-Core Processors" (arXiv 1704.03767).
 *   - tau-b definition: Sec. 1, Eq. 3 and Table 1 (n_0, n_1, n_2, n_3).
 *   - per-variable rank transform done once: Sec. 3 (opening paragraph).
 *   - Knight counting with exact tie handling: Sec. 3.2, Steps 1-5 and Algorithm 2.
 *   - sign form of the concordance count (naive kernel): Sec. 3.1, Algorithm 1.
 *   - job-id <-> (y, x) bijection and tiling of the upper triangle: Sec. 4.1-4.2, Eq. 4-14.
 *   - result sub-ranges processed pass by pass: Sec. 4.3.1.
 *   - query-based co-expression search (motivation for the query form): Sec. 1.
 *
 * Conventions shared by every entry point
 *   - Every function returns a ktau_status; nothing throws across the ABI. On failure
 *     ktau_last_error() returns a thread-local, human-readable message for the calling thread.
 *   - "device pointer" means memory of the current CUDA device, allocated by the caller
 *     (cudaMalloc, a torch tensor's data_ptr(), ...). The library never frees caller memory.
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream). Work is
 *     enqueued on it asynchronously unless a function says it synchronises.
 *   - A matrix of m variables by n samples is row-major: variable i occupies
 *     values[i*ld .. i*ld + n), with ld >= n (elements, not bytes).
 *   - Pairs are the strict upper triangle of the m x m job matrix: pair (i, j) with i < j has the
 *     packed index p = i*(2m-i-1)/2 + (j-i-1), i.e. rows are numbered left-to-right,
 *     top-to-bottom as in the paper's Eq. 4-5 applied to the (m-1) x (m-1) triangle that
 *     excludes the diagonal. u = variable i, v = variable j. All outputs are symmetric in (u, v).
 *   - Counts per pair: S = n_c - n_d and n_3 (joint ties). The per-variable tie counts
 *     n_1 (of u) and n_2 (of v) are T[i] and T[j] from ktau_tie_counts().
 *   - tau-b = (double)S / sqrt((double)(n_0-T_u) * (double)(n_0-T_v)) in IEEE FP64
 *     (round-to-nearest sqrt and divide); NaN when either factor is 0 (a constant variable).
 *     The FP32 output is the FP64 value rounded to nearest-even.
 *   - Limits: 2 <= n <= KTAU_MAX_N, 1 <= m <= KTAU_MAX_M (a single variable has no pairs); the
 *     batched and allocation-free forms take n <= KTAU_BATCH_MAX_N. Rows longer than 16384 samples
 *     are ranked and counted (merge path) with library scratch in global memory. Rows longer than
 *     KTAU_NARROW_MAX_N samples keep 32-bit ranks and sample indices (the 64-bit key packing the
 *     paper's Sec. 6 anticipates): such handles serve the merge path of ktau_allpairs and
 *     ktau_allpairs_host only, with 64-bit counts; every other form returns KTAU_EINVAL or
 *     KTAU_ETOOLARGE for them. Values may be +-Inf; -0.0 equals +0.0; a NaN anywhere fails
 *     the call with KTAU_ENAN.
 */
#ifndef KTAU_H
#define KTAU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KTAU_ABI_VERSION 2
#define KTAU_MAX_N 4194304    /* samples per variable */
#define KTAU_NARROW_MAX_N 65535 /* longest rows kept with uint16 ranks and sample indices */
#define KTAU_BATCH_MAX_N 16384 /* samples per variable in the batched and allocation-free forms */
#define KTAU_MAX_M 4194304    /* variables per matrix */

typedef enum {
  KTAU_OK = 0,
  KTAU_EINVAL = 1,     /* bad argument: NULL where required, sizes out of range, mismatch */
  KTAU_ENAN = 2,       /* a NaN value was found in the input */
  KTAU_ETOOLARGE = 3,  /* n > KTAU_MAX_N, m > KTAU_MAX_M, or a count does not fit count_bits */
  KTAU_ENOMEM = 4,     /* a device allocation made by the library failed */
  KTAU_ECUDA = 5,      /* a CUDA runtime call failed; ktau_last_error() has the CUDA message */
  KTAU_ETIMEOUT = 6,   /* a bounded device-side wait gave up (reported through a status word) */
  KTAU_EBUSY = 7       /* the object is in use by a captured graph or another call */
} ktau_status;

typedef enum { KTAU_F32 = 0, KTAU_I32 = 1 } ktau_dtype;

/* Which pairwise kernel computes the counts. */
typedef enum {
  KTAU_PATH_AUTO = 0,      /* pick by shape and measured timings (autotuner table) */
  KTAU_PATH_MERGE = 1,     /* Knight merge-sort swap counting, Sec. 3.2 Steps 1-5 */
  KTAU_PATH_SIGNGEMM = 2,  /* exact sign-matrix contraction on tensor cores, Sec. 3.1 Alg. 1;
                              n <= 5792 (n_0 < 2^24). n_3 from the tied sample pairs' lists, or,
                              for tie-heavy matrices and rows above 3000 samples (FP4 operands,
                              ktau_allpairs only), from a second contraction of the magnitudes */
  KTAU_PATH_BITS = 3       /* bit-parallel dominance count: the sign form of Sec. 3.1 Alg. 1 over
                              per-sample masks of larger / smaller ranks, 32 sample pairs per
                              AND + popcount; ktau_allpairs(_host) only, n <= KTAU_BITS_MAX_N */
} ktau_path;
#define KTAU_BITS_MAX_N 256

/* Tuning knobs; any field left 0 means "library default / autotuned". */
typedef struct {
  int32_t path;         /* ktau_path */
  int32_t tile_q;       /* variables per side of a square tile of the job matrix (Sec. 4.2 q) */
  int32_t mapping;      /* merge path: 1 = one warp per pair, 2 = one CTA per pair */
  int32_t schedule;     /* 1 = static stride over tile ids (Sec. 4.3.2), 2 = dynamic counter */
  int32_t ctas_per_sm;  /* persistent grid = ctas_per_sm * SM count */
  int32_t operand_bits; /* contraction operands: 4 = FP4 e2m1 (the triangle's pair kernel reads
                           them with the block-scaled FP4 MMA, scale factors 1), 8 = FP8 e4m3,
                           16 = BF16, all exact for n <= 5792 (n_0 < 2^24); 0 = FP4 */
  int32_t statistic;    /* 0 = tau-b (Eq. 3, default); 1 = tau-a = (n_c - n_d) / n_0 (Sec. 2, no
                           tie correction): tau64 = S / n_0 in IEEE FP64, tau32 = S / n_0
                           correctly rounded to FP32. ktau_allpairs, ktau_allpairs_path and
                           ktau_allpairs_host only; ktau_query and ktau_batch_create reject it */
  int32_t reserved[1];
} ktau_options;

/* Opaque, library-owned, device-resident ranked matrix (Sec. 3: each variable ranked once):
 * stable sort permutation, dense ranks, per-variable tie counts, and (lazily) the sign
 * expansion used by the tensor-core path. */
typedef struct ktau_ranked ktau_ranked;

/* Thread-local message describing the last failure of this thread (never NULL). */
const char* ktau_last_error(void);
/* Static name of a status code. */
const char* ktau_status_string(ktau_status s);
/* KTAU_ABI_VERSION of the loaded library. */
int32_t ktau_abi_version(void);

/*
 * ktau_rank_prepare -- rank transform of every variable (Sec. 3, opening paragraph; the scans
 * of Steps 2 and 4 for n_1 and n_2 are hoisted here because they depend on one variable only).
 *   values : caller-owned device pointer, m x n row-major with row stride ld (elements),
 *            dtype dt (KTAU_F32 or KTAU_I32). Read only; may be freed once the call returns.
 *   out    : receives a new handle owned by the caller; release with ktau_ranked_free().
 * Per variable u the handle holds the stable argsort pi_u (ties keep sample order), the dense
 * rank r_u (equal values share a rank, -0.0 == +0.0), and T_u = sum over tie groups t(t-1)/2.
 * Synchronises `stream` once (to read the NaN flag). On any error no handle is returned.
 * Errors: EINVAL (NULL, m < 1, n < 2, ld < n, bad dtype), ETOOLARGE, ENAN, ENOMEM, ECUDA.
 */
ktau_status ktau_rank_prepare(const void* values, ktau_dtype dt, int64_t m, int64_t n, int64_t ld,
                              void* stream, ktau_ranked** out);

/* ktau_rank_prepare without the synchronisation: the NaN flag and the tie statistics are copied
 * to pinned host memory behind an event on `stream`, and the first call that needs them
 * (ktau_allpairs, ktau_allpairs_host, ktau_allpairs_path, ktau_query, ktau_permutation_exceed)
 * waits for that copy, so work enqueued in between (ktau_prepare_signs) overlaps the rank
 * transform's completion. A NaN is reported by that first call (KTAU_ENAN, and again by every
 * later call on the handle). `values` must stay valid until the rank transform has run on
 * `stream`. The first use must not race with another call on the same handle. Errors as
 * ktau_rank_prepare except ENAN. */
ktau_status ktau_rank_prepare_async(const void* values, ktau_dtype dt, int64_t m, int64_t n,
                                    int64_t ld, void* stream, ktau_ranked** out);

/* ktau_rank_prepare from HOST values: values_h is a host pointer (page-locked memory gives full
 * copy bandwidth), m x n row-major with row stride ld elements, dtype dt. The values are copied
 * into a library-owned device staging buffer on `stream` and ranked from there; the staging
 * buffer goes back to the library's cache before the call returns, so values_h may be reused at
 * once. Synchronises `stream`. Errors as ktau_rank_prepare. */
ktau_status ktau_rank_prepare_host(const void* values_h, ktau_dtype dt, int64_t m, int64_t n,
                                   int64_t ld, void* stream, ktau_ranked** out);

/* Releases a handle (NULL is accepted). Synchronises the device before freeing. */
ktau_status ktau_ranked_free(ktau_ranked* R);
/* Releases a handle whose every use was enqueued on `stream`: synchronises that stream only
 * (other streams keep running), then returns its memory to the library's cache. */
ktau_status ktau_ranked_free_on(ktau_ranked* R, void* stream);

/* Shape of a handle (either output pointer may be NULL). Host only, no synchronisation. */
ktau_status ktau_ranked_shape(const ktau_ranked* R, int64_t* m, int64_t* n);

/* Copies T_u (n_1 / n_2 of Table 1) for every variable into the caller's device buffer
 * T_dev[m] (int64). Asynchronous on `stream`. */
ktau_status ktau_tie_counts(const ktau_ranked* R, int64_t* T_dev, void* stream);

/* Copies the permutation pi (perm[m*n]) and dense ranks r (rank[m*n]) into caller device
 * buffers, packed m x n (uint16). Either pointer may be NULL. Asynchronous on `stream`.
 * EINVAL for a handle with n > KTAU_NARROW_MAX_N (use ktau_ranked_export32). */
ktau_status ktau_ranked_export(const ktau_ranked* R, uint16_t* perm, uint16_t* rank, void* stream);
/* The same as uint32 (any n): perm[m*n] and rank[m*n] packed m x n. Asynchronous on `stream`. */
ktau_status ktau_ranked_export32(const ktau_ranked* R, uint32_t* perm, uint32_t* rank,
                                 void* stream);

/*
 * ktau_allpairs -- exact tau-b for every pair with packed index in [p_begin, p_end)
 * (Sec. 4.1-4.3: the upper triangle walked through the job-id bijection, tile by tile, in
 * result sub-ranges so the output of one pass fits the caller's buffers).
 *   [p_begin, p_end) : subrange of [0, m(m-1)/2); empty ranges are accepted and do nothing.
 *   tau64, tau32, S, n3 : caller-owned device buffers of p_end - p_begin elements, element k
 *            for pair p_begin + k. Any of them may be NULL (that output is not stored).
 *            S and n3 are int32 when count_bits == 32, int64 when count_bits == 64.
 *   count_bits : 32 or 64. 32 requires n_0 = n(n-1)/2 < 2^31, else ETOOLARGE.
 *   opt    : NULL or options (path, tile, mapping, schedule); NULL = autotuned.
 * Asynchronous on `stream`; the handle must stay alive until the work completes.
 * The first tensor-core call on a handle allocates and fills its sign expansion (library
 * memory, m * n_0 bytes rounded up) and is therefore not graph-capturable.
 * Errors: EINVAL (NULL handle, range outside the triangle, bad count_bits/options), ETOOLARGE,
 * ENOMEM, ECUDA.
 */
ktau_status ktau_allpairs(const ktau_ranked* R, uint64_t p_begin, uint64_t p_end, double* tau64,
                          float* tau32, void* S, void* n3, int32_t count_bits,
                          const ktau_options* opt, void* stream);

/*
 * ktau_allpairs_noalloc -- ktau_allpairs (merge path) for one matrix straight from its values,
 * allocating nothing. The paper has no counterpart. It serves callers that cannot allocate device
 * memory where they need the result: plug-ins of a host framework that owns the device memory
 * through its own allocator and budget (a cudaMalloc behind its back can fail or break its
 * accounting), and real-time loops that forbid cudaMalloc/cudaFree because those calls can
 * synchronise the device and stall.
 *   values, dt, m, n, ld : as ktau_rank_prepare. [p_begin, p_end), tau64, tau32, S, n3,
 *            count_bits : as ktau_allpairs. All caller-owned; the library allocates nothing.
 * Working memory is a fixed array of KTAU_NOALLOC_SCRATCH_BYTES compiled into the library (every
 * GPU that loads the library holds it until the process exits). It must hold the ranked matrix,
 * 3*m*ld16*2 + 32*m bytes (ld16 = n rounded up to 16, arrays padded to 256 bytes) plus 256; larger
 * inputs fail with KTAU_ETOOLARGE (m <= 16384 at n = 128 fits). The first call on a device looks
 * up the array's device address (set-up, once per device), so make that first call before any
 * stream capture. Every call uses the same array, which keeps the previous call's contents: calls
 * whose GPU work overlaps (other streams, other threads) race and must be serialised by the
 * caller. Synchronises `stream` once, after the rank transform, to read the NaN flag (KTAU_ENAN).
 * Errors: EINVAL, ETOOLARGE, ENAN, ECUDA.
 */
#define KTAU_NOALLOC_SCRATCH_BYTES (16u << 20)
ktau_status ktau_allpairs_noalloc(const void* values, ktau_dtype dt, int64_t m, int64_t n,
                                  int64_t ld, uint64_t p_begin, uint64_t p_end, double* tau64,
                                  float* tau32, void* S, void* n3, int32_t count_bits,
                                  void* stream);

/*
 * ktau_allpairs_host -- ktau_allpairs with HOST output buffers, in passes (Sec. 4.3.1: the range is
 * split into sub-ranges computed one after another, and each pass's results are copied to the host
 * while the next pass computes). Device staging is two library-owned buffers per output.
 *   tau64_h, tau32_h, S_h, n3_h : host buffers of p_end - p_begin elements (any may be NULL);
 *            page-locked memory (cudaHostAlloc / pinned tensors) gives full copy bandwidth.
 *   pass_pairs : pairs per pass; 0 picks about a quarter of the range, aligned to 256-row blocks.
 * Synchronises `stream` before returning (the host buffers are complete on return). Other
 * arguments and errors as ktau_allpairs.
 */
ktau_status ktau_allpairs_host(const ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                               double* tau64_h, float* tau32_h, void* S_h, void* n3_h,
                               int32_t count_bits, const ktau_options* opt, uint64_t pass_pairs,
                               void* stream);

/* Which path ktau_allpairs would take for this handle and options (KTAU_PATH_MERGE or
 * KTAU_PATH_SIGNGEMM) -- the autotuner's choice when opt is NULL or opt->path is AUTO. */
ktau_status ktau_allpairs_path(const ktau_ranked* R, const ktau_options* opt, int32_t* path);

/* Builds the tensor-core operands of a handle now instead of on first use: the sign expansion
 * A_u[k] = sign(u_b - u_a) over all sample pairs (Sec. 3.1, Algorithm 1; the pairs in an internal
 * order shared by every variable), stored as packed FP4 e2m1 (library memory, m * n_0 / 2 bytes
 * with n_0 rounded up to 256 per variable). The lists of tied
 * sample pairs that n_3 needs are built by the first ktau_allpairs call that stores n_3, beside
 * its contraction. Asynchronous on `stream` (allocates on first use). EINVAL when n > 5792
 * (path unsupported). */
ktau_status ktau_prepare_signs(ktau_ranked* R, void* stream);

/* Synchronises `stream` and reports device-side status words raised since the last call, then
 * clears them: KTAU_ETIMEOUT when a bounded wait of a tensor-core kernel gave up (that launch's
 * results are invalid), KTAU_ETOOLARGE when a top-k selection met more than 2048 rows tied at
 * its boundary without exact keys (n > 300; that query's top-k order is not exact). */
ktau_status ktau_device_status(void* stream);

/* Permutation test of every pair (Sec. 2: the significance of tau under random relabelling of one
 * variable's samples). For each of the B permutations sigma_b (perms: device uint16 [B][n], row b
 * a permutation of 0..n-1 drawn by the caller) and each pair (u, v), u < v, with packed index p
 * in [p_begin, p_end), adds 1 to exceed[p - p_begin] when |S(u, v o sigma_b)| >= |S(u, v)|, where
 * S(u, v o sigma) = n_c - n_d between u and v with v's samples reordered by sigma. T_u and T_v do
 * not change under the relabelling, so this is |tau_b| (and |tau_a|) exceedance exactly. The
 * two-sided permutation p-value of pair p is (exceed + 1) / (B + 1).
 *   S_obs  : int32 device array, the observed S of the same range (ktau_allpairs, count_bits 32)
 *   exceed : uint32 device array of p_end - p_begin counts, accumulated (the caller zeroes it)
 * Runs on the sign contraction (EINVAL when n > 5792): per permutation one relabelled copy of
 * the ranks, its sign expansion and one pass of the pair contraction. Entries of perms outside
 * 0..n-1 give meaningless counts but no out-of-range access. Allocates scratch of one rank and one
 * operand matrix and returns after the work has finished on `stream`. */
ktau_status ktau_permutation_exceed(const ktau_ranked* R, const uint16_t* perms, int32_t B,
                                    uint64_t p_begin, uint64_t p_end, const int32_t* S_obs,
                                    uint32_t* exceed, void* stream);

/* Two-sided permutation p-values of the pairs whose exceedance counts ktau_permutation_exceed
 * accumulated over B permutations: pvalue[i] = (exceed[i] + 1) / (B + 1) in IEEE FP64 (the
 * observed labelling counted as one of B + 1 equally likely ones; Sec. 2 motivates tau as a
 * test statistic). exceed: uint32 device array of `count` counts; pvalue: FP64 device array of
 * `count`. Asynchronous on `stream`. Errors: EINVAL (NULL arrays with count > 0, B < 0), ECUDA. */
ktau_status ktau_permutation_pvalues(const uint32_t* exceed, int32_t B, uint64_t count,
                                     double* pvalue, void* stream);

/* Failure injection for tests of error handling (no GPU fault involved):
 * ktau_debug_fail_alloc(k): the next k library allocations succeed, every later one fails as if
 * the device were out of memory (KTAU_ENOMEM); k < 0 switches the injection off.
 * ktau_debug_wait_timeout(limit_ns, stream): launches one small kernel whose bounded wait (the
 * same wait the tensor-core kernels use) watches an mbarrier nothing arrives on; after limit_ns it
 * raises the device status word and returns, so ktau_device_status then reports KTAU_ETIMEOUT and
 * the context stays usable. */
ktau_status ktau_debug_fail_alloc(int32_t k);
ktau_status ktau_debug_wait_timeout(int64_t limit_ns, void* stream);

/* Kernel trace: when enabled, every kernel the library launches is bracketed by CUDA events on
 * its stream (no extra synchronisation). ktau_trace_collect waits for the recorded launches,
 * copies up to `cap` records (kernel name, milliseconds, in launch order) and clears the list.
 * Tracing must be off while a stream is being captured into a CUDA graph. */
typedef struct {
  char name[48];
  float ms;
} ktau_trace_record;
ktau_status ktau_trace_enable(int32_t on);
ktau_status ktau_trace_collect(ktau_trace_record* out, int32_t cap, int32_t* count);
/* Restricts the trace to launches named `name` (the record names, e.g. "contract_kernel"); NULL
 * or "" traces every launch. Each traced launch adds two event records to its stream, so a
 * filter keeps the trace from adding to the time of the steps it measures. */
ktau_status ktau_trace_filter(const char* name);

/*
 * Batched form: many independent matrices of uneven m and n processed by one persistent
 * launch per kernel family (generalises the pass/tile scheduling of Sec. 4.2-4.3 to a list of
 * datasets). A plan owns all scratch; ktau_batch_run allocates nothing and never synchronises,
 * so it can be captured into a CUDA graph (ktau_batch_graph_launch does that itself).
 */
typedef struct {
  const void* values;  /* device, m x n row-major, row stride ld, dtype */
  int32_t dtype;       /* ktau_dtype */
  int32_t count_bits;  /* 32 or 64, as in ktau_allpairs */
  int64_t m, n, ld;
  double* tau64;       /* m(m-1)/2 outputs each, any may be NULL */
  float* tau32;
  void* S;
  void* n3;
  int32_t path;        /* ktau_path for this dataset; AUTO = opt->path, else by n (autotuner) */
  int32_t mapping;     /* merge path: 1 = one warp per pair, 2 = one CTA per pair, 0 = by n
                          (a warp up to n = 1024); datasets of both kinds form separate groups */
} ktau_batch_desc;

typedef struct ktau_batch ktau_batch;

/* Validates the descriptors (host-side only; the contents of `values` are read at run time),
 * chooses a path per dataset (opt->path, or the autotuner table when AUTO), allocates device
 * scratch and descriptor tables. The descriptors are copied; the pointed-to buffers must stay
 * valid for the plan's lifetime. Errors: EINVAL, ETOOLARGE, ENOMEM, ECUDA. */
ktau_status ktau_batch_create(const ktau_batch_desc* descs, int32_t count, const ktau_options* opt,
                              ktau_batch** out);
/* Enqueues rank transform + all pairs of every dataset on `stream` (no allocation, no sync). */
ktau_status ktau_batch_run(ktau_batch* B, void* stream);
/* Same work through a CUDA graph captured on first use (on `stream`, which must not be the
 * legacy default stream) and replayed after. */
ktau_status ktau_batch_graph_launch(ktau_batch* B, void* stream);
/* Synchronises `stream` and reports a NaN found in any dataset since the last check (ENAN). */
ktau_status ktau_batch_check(ktau_batch* B, void* stream);
/* Number of datasets routed to each path (either pointer may be NULL). */
ktau_status ktau_batch_paths(const ktau_batch* B, int32_t* n_merge, int32_t* n_signgemm);
/* Total pairs over all datasets. */
ktau_status ktau_batch_pairs(const ktau_batch* B, uint64_t* pairs);
ktau_status ktau_batch_free(ktau_batch* B);

/*
 * ktau_allpairs_batched -- the batched form as one call, with all scratch in a workspace the caller
 * owns (the pass and tile scheduling of Sec. 4.2-4.3 generalised to a list of job matrices):
 * rank transform and every pair of every dataset, exactly as ktau_batch_create + ktau_batch_run
 * would compute them, bit for bit.
 *   descs, count, opt : as ktau_batch_create (the descriptors are read during the call only).
 *   workspace : caller-owned device memory, 256-byte aligned, of at least ktau_workspace_size()
 *            bytes for the same descriptors and options. It holds the ranked datasets, their
 *            operands and the plan's tables, and must stay untouched until the work has finished
 *            on `stream`. Its contents need no initialisation.
 *   nan_flag : NULL or a device uint32 that receives this call's NaN flag (nonzero when some
 *            dataset holds a NaN; that dataset's outputs are then meaningless).
 * Allocates nothing, creates no stream and never synchronises: the plan's tables reach the device
 * as parameters of small kernel launches on `stream` (no memcpy, no staging), and every group runs
 * on `stream`, one after another, so the call can also be captured into a CUDA graph. For repeated
 * launches of the same datasets, ktau_batch_create + ktau_batch_graph_launch spread the groups over
 * several streams and replay them as one CUDA graph.
 * Errors: EINVAL (as ktau_batch_create; workspace NULL, unaligned or too small), ETOOLARGE, ECUDA.
 */
ktau_status ktau_allpairs_batched(const ktau_batch_desc* descs, int32_t count,
                                  const ktau_options* opt, void* workspace, size_t workspace_bytes,
                                  uint32_t* nan_flag, void* stream);
/* Bytes of workspace ktau_allpairs_batched needs for these descriptors and options (host only; no
 * device work, nothing allocated). */
ktau_status ktau_workspace_size(const ktau_batch_desc* descs, int32_t count,
                                const ktau_options* opt, size_t* bytes);

/*
 * ktau_query -- query-based search (Sec. 1): exact tau-b of every query profile against every
 * database variable, plus the k database rows with the largest |tau-b| per query.
 *   db      : ranked database (m_db x n). queries: ranked queries (b x n, same n, else EINVAL).
 *   tau     : device FP64 [b][m_db] or NULL.  S, n3: device [b][m_db] of count_bits, or NULL.
 *   k       : 0 <= k <= min(m_db, 1024). topk_idx (int32 [b][k]) and topk_tau (FP64 [b][k]) are
 *             required when k > 0. Order: |tau| descending by exact rational comparison of
 *             S^2/(D_u D_v); equal values by smaller row index; NaN (constant rows) last.
 *   opt     : as for ktau_allpairs (path choice). The database's sign expansion, when the
 *             tensor-core path is chosen, is built on first use and kept in the handle; with an
 *             n3 output the contraction is used for n <= 3000 only (longer rows: merge path).
 * The top-k is selected in passes over 4096-row chunks (their candidate lists in scratch from
 * a stream-ordered memory pool the library owns per device, which keeps its memory once
 * reserved; released on `stream`). n <= KTAU_NARROW_MAX_N (the exact
 * comparison of S^2 / D_v uses 64- and 128-bit integers), else ETOOLARGE.
 * Asynchronous on `stream`. Errors: EINVAL, ETOOLARGE, ENOMEM, ECUDA.
 */
ktau_status ktau_query(const ktau_ranked* db, const ktau_ranked* queries, double* tau, void* S,
                       void* n3, int32_t count_bits, int32_t k, int32_t* topk_idx, double* topk_tau,
                       const ktau_options* opt, void* stream);

/* Device memory (bytes) that ktau_query needs beyond its outputs for b queries against db;
 * used by servers to admit work by free memory. */
ktau_status ktau_query_scratch_bytes(const ktau_ranked* db, int64_t b, int32_t k, size_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* KTAU_H */
