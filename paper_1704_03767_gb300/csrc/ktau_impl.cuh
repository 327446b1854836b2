// Internal definitions shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ktau.h"

// ---------------------------------------------------------------------------------------------
// Ranked matrix (Sec. 3: every variable is rank transformed once, before any pair is counted).
// Layout in HBM, row-major with row stride `ld` elements (ld = n rounded up to 16, so every row
// starts on a 32-byte boundary and can be moved with 16-byte vector loads):
//   perm [m][ld] uint16  stable argsort pi_u: perm[k] = sample index of the k-th smallest value
//   rank [m][ld] uint16  dense rank r_u of each sample (equal values share a rank)
//   srank[m][ld] uint16  rank in sorted order, srank[k] = rank[perm[k]] (tie-group id at k)
//   T    [m]     int64   tie pairs of the variable, sum over groups t(t-1)/2 (n_1 / n_2)
//   ndist[m]     int32   number of distinct values; maxg[m] int32 largest tie group
//   rs64 [m]     double  1/sqrt(n_0 - T): the variable's factor of the tau-b denominator (Eq. 3),
//                        NaN for a constant variable
//   rsff [m]     float2  rs64 split into a float-float pair (hi, lo), hi + lo == rs64 to 2^-48
// Padding entries (k >= n) hold 0xFFFF.
// Rows longer than 65535 samples ("wide" handles) hold the same three arrays as uint32 (perm32,
// rank32, srank32; padding 0xFFFFFFFF) and leave the uint16 pointers null: only the merge path
// reads them.
// ---------------------------------------------------------------------------------------------
struct ktau_stats {
  unsigned long long T_sum;
  unsigned long long T_max;
  unsigned int maxg;
  unsigned int nan_flag;
  unsigned int pad[2];
};

// Rows longer than this are ranked in chunks of this many keys merged in global scratch, and
// their pairs are counted with the merge buffers in global scratch (shared memory holds rows of up
// to this length).
#define KTAU_RANK_CHUNK 16384

struct ktau_ranked {
  int64_t m, n, ld;
  int device;
  void* block;  // single allocation holding every array below
  size_t block_bytes;
  uint16_t* perm;
  uint16_t* rank;
  uint16_t* srank;
  int wide;  // n > KTAU_NARROW_MAX_N: 32-bit arrays below instead of the 16-bit ones above
  uint32_t* perm32;
  uint32_t* rank32;
  uint32_t* srank32;
  int64_t* T;
  int32_t* ndist;
  int32_t* maxg;
  double* rs64;
  float2* rsff;
  ktau_stats* stats_dev;
  ktau_stats stats;  // host copy, filled by ktau_rank_prepare (see ktau_ranked_stats)
  // ktau_rank_prepare_async: the statistics are copied into a pinned host slot behind stats_ev
  // and read on first use; stats_pin is null once `stats` holds them.
  ktau_stats* stats_pin;
  cudaEvent_t stats_ev;
  // Scratch of the long-row rank transform (n > KTAU_RANK_CHUNK), released once the statistics
  // copy (which follows the rank transform on its stream) has completed.
  void* tmp_block;
  size_t tmp_bytes;
  // Sign expansion for the tensor-core path, built on first use (library-owned):
  // sgn[m][K_pad] of values in {-1, 0, +1} as FP4 e2m1 (obits 4, two per byte), FP8 e4m3
  // (obits 8) or BF16 (obits 16), K = n(n-1)/2, K_pad = K rounded up to 128; esize is the
  // operand's bytes per element in shared memory (1, or 2 for BF16); tmap is its TMA descriptor.
  void* sgn;
  int64_t K, K_pad;
  int esize, obits;
  int sg_ready;
  alignas(64) unsigned char tmap[128];
  // FP4 only: the same rows as plain bytes, for the block-scaled (kind::mxf4) pair contraction,
  // which reads the packed e2m1 elements directly (tmap expands them to one byte each): boxes of
  // 128 rows (column operand) and of 120 rows (row operand).
  alignas(64) unsigned char tmap_mx[128];
  alignas(64) unsigned char tmap_mxb[128];
  size_t sgn_bytes;
  // |A| operand (FP4 only, built on first use by an n_3 output of a tie-heavy matrix): the same
  // rows with 1 where the sample pair is not tied in the variable and 0 where it is, so that
  // |A_u| . |A_v| = n_c + n_d = n_0 - T_u - T_v + n_3 (Table 1). Tensor maps as tmap_mx/_mxb.
  void* sgn_abs;
  size_t sgn_abs_bytes;
  alignas(64) unsigned char tmap_mx_abs[128];
  alignas(64) unsigned char tmap_mxb_abs[128];
  int abs_ready;
  // Lists of tied sample pairs for n_3 (tie_off[m+1] = prefix of T, tie_pairs[(a << 16) | b]);
  // a variable is listed when its list ends within tie_cap entries.
  int64_t* tie_off;
  uint32_t* tie_pairs;
  int64_t tie_cap;
  size_t tie_bytes;
  // Inverted index of the tied sample pairs (triangular n_3): bucket k (the k-th sample pair in
  // the Eq. 4 order) lists the variables tied on it; bkt_off[K + 1] prefix, bkt_var[T_sum].
  // bkt_stat = {sum of s(s-1)/2 over buckets, largest s(s-1)/2, use flag} (device words).
  int32_t* bkt_off;
  int32_t* bkt_var;
  unsigned long long* bkt_stat;
  size_t bkt_var_bytes;
  int ties_ready;  // tie lists and index built (on first use by an n_3 output)
  // Bit-parallel path: per-sample dominance masks of every variable (built on first use).
  uint32_t* bits;
  size_t bits_bytes;
};

// The handle's rank statistics on the host: waits for the copy of an asynchronously prepared
// handle on its first use (one thread at a time); ENAN when the matrix held a NaN.
ktau_status ktau_ranked_stats(const ktau_ranked* R);

// ---------------------------------------------------------------------------------------------
// Error reporting (thread-local message, see ktau_last_error).
// ---------------------------------------------------------------------------------------------
ktau_status ktau_fail(ktau_status s, const char* fmt, ...);
ktau_status ktau_cuda_fail(cudaError_t e, const char* what);
int ktau_sm_count();
// Library allocations go through a per-device cache of freed blocks (exact-size reuse), so
// handles created and released every step do not pay cudaMalloc/cudaFree (which synchronises).
ktau_status ktau_dmalloc(void** p, size_t bytes);
void ktau_dfree(void* p, size_t bytes);

// Kernel trace (ktau_trace_enable): events around each launch when enabled.
struct ktau_trace_scope {
  int slot;
  cudaStream_t st;
  ktau_trace_scope(const char* name, cudaStream_t s);
  ~ktau_trace_scope();
};
#define KTAU_TRACE(name, stream) ktau_trace_scope ktau_trace_scope_##__LINE__(name, stream)

#define KTAU_CUDA(call)                                                   \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return ktau_cuda_fail(e_, #call);              \
  } while (0)

#include "bijection.cuh"

// ---------------------------------------------------------------------------------------------
// Step 5 of Sec. 3.2 and Eq. 3: S = n_0 - n_1 - n_2 + n_3 - 2 n_d, tau-b from the exact counts.
//
// FP64 runs at a small fraction of the FP32 rate on GB300, so the per-pair division and square
// root of Eq. 3 are replaced by the product of per-variable factors r_u = 1/sqrt(n_0 - T_u)
// (computed once per variable in IEEE FP64 by the rank kernel):
//   tau64 = ((double)S * r_u) * r_v                    two FP64 products, error <= 4 ulp
//   tau32 = RN_f32 of the FP64 formula S / sqrt(D_u D_v), decided from a float-float product
//           S * r_u * r_v (relative error < 2^-43); when that value lies within 2^-40 of a float
//           rounding boundary, the FP64 formula itself is evaluated, so the result is always
//           exactly the round-to-nearest float of the FP64 formula.
// Every kernel (merge, sign contraction, query, batched) stores through this one function, so
// all paths give bit-identical outputs for the same pair.
// ---------------------------------------------------------------------------------------------
struct ktau_out {
  double* tau64;
  float* tau32;
  void* S;
  void* n3;
  int count_bits;
  int stat;  // 0 = tau-b, 1 = tau-a
};

__device__ __forceinline__ double ktau_nan() { return __longlong_as_double(0x7ff8000000000000LL); }

// The FP64 formula of Eq. 3 (slow on this part; only for the rare boundary cases).
static __device__ __noinline__ double ktau_tau_b_formula(int64_t S, int64_t du, int64_t dv) {
  if (du == 0 || dv == 0) return ktau_nan();
  return __ddiv_rn((double)S, __dsqrt_rn(__dmul_rn((double)du, (double)dv)));
}

__device__ __forceinline__ double ktau_tau64(int64_t S, double ru, double rv) {
  return __dmul_rn(__dmul_rn((double)S, ru), rv);
}

// RN_f32 of tau-b: the float-float product S * r_u * r_v approximates tau within 2^-43 relative
// (and the FP64 formula is within 2^-51 of tau), so when rounding the approximation 2^-40 |tau|
// lower and higher gives the same float, every value in between -- the FP64 formula's included --
// rounds to that float (round-to-nearest is monotone). Otherwise (rare) the FP64 formula decides.
// A constant variable has NaN factors: the test fails and the formula returns NaN.
__device__ __forceinline__ bool ktau_tau32_fast(int S, float2 fu, float2 fv, float& out) {
  const float sh = __int2float_rn(S);
  const float sl = __int2float_rn(S - __float2int_rn(sh));  // S == sh + sl exactly
  const float th = __fmul_rn(sh, fu.x);
  const float tl = __fadd_rn(__fmaf_rn(sh, fu.x, -th), __fmaf_rn(sh, fu.y, __fmul_rn(sl, fu.x)));
  const float ph = __fmul_rn(th, fv.x);
  const float pl = __fadd_rn(__fmaf_rn(th, fv.x, -ph), __fmaf_rn(th, fv.y, __fmul_rn(tl, fv.x)));
  const float d = __fmul_rn(fabsf(ph), 0x1p-40f);
  const float lo = __fadd_rn(ph, __fsub_rn(pl, d));
  const float hi = __fadd_rn(ph, __fadd_rn(pl, d));
  out = lo;
  return lo == hi;
}

__device__ __forceinline__ float ktau_tau32(int64_t S, float2 fu, float2 fv, int64_t n0,
                                            int64_t Tu, int64_t Tv) {
  float f;
  // The float-float split of S assumes |S| < 2^31 (always so for n <= 65535); longer rows whose
  // S is larger take the FP64 formula.
  if (S > -(1ll << 31) && S < (1ll << 31) && ktau_tau32_fast((int)S, fu, fv, f)) return f;
  return __double2float_rn(ktau_tau_b_formula(S, n0 - Tu, n0 - Tv));
}

struct ktau_fac {
  const double* rs64;
  const float2* rsff;
  const int64_t* T;
};

// tau-a = S / n_0 (no tie correction). FP64: the IEEE quotient of two exact integers. FP32: the
// quotient correctly rounded to FP32. With S and n_0 below 2^24 that is one IEEE division; above,
// the FP64 quotient q is rounded to FP32, which can mislead only when q lies exactly on the
// midpoint m of two floats; then the sign of S - m * n_0 decides. That difference is formed
// exactly: p = RN(m * n_0) and its rounding error e = fma(m, n_0, -p) are exact doubles, S - p is
// exact (S and p are within a factor of two of each other), and the sign of (S - p) - e is the
// sign of the exact difference (S, n_0 < 2^53).
__device__ __forceinline__ double ktau_taua64(int64_t S, int64_t n0) {
  return __ddiv_rn((double)S, (double)n0);
}
__device__ __forceinline__ float ktau_taua32(int64_t S, int64_t n0) {
  if (n0 < (1ll << 24)) return __fdiv_rn((float)S, (float)n0);
  const double q = __ddiv_rn((double)S, (double)n0);
  const float f = __double2float_rn(q);
  const double fd = (double)f;
  if (fd == q) return f;
  const float g = nextafterf(f, q > fd ? INFINITY : -INFINITY);
  const double mid = 0.5 * (fd + (double)g);
  if (q != mid) return f;
  const double prod = __dmul_rn(mid, (double)n0);
  const double err = __fma_rn(mid, (double)n0, -prod);
  const double diff = __dsub_rn(__dsub_rn((double)S, prod), err);
  if (diff == 0.0) return f;  // exact tie: already rounded to even
  return diff > 0.0 ? fmaxf(f, g) : fminf(f, g);
}

__device__ __forceinline__ void ktau_store(const ktau_out& o, uint64_t k, int64_t S, int64_t n3,
                                           int64_t n0, const ktau_fac& f, int64_t u, int64_t v) {
  if (o.tau64) o.tau64[k] = o.stat ? ktau_taua64(S, n0) : ktau_tau64(S, f.rs64[u], f.rs64[v]);
  if (o.tau32)
    o.tau32[k] = o.stat ? ktau_taua32(S, n0)
                        : ktau_tau32(S, f.rsff[u], f.rsff[v], n0, f.T[u], f.T[v]);
  if (o.count_bits == 64) {
    if (o.S) ((long long*)o.S)[k] = S;
    if (o.n3) ((long long*)o.n3)[k] = n3;
  } else {
    if (o.S) ((int*)o.S)[k] = (int)S;
    if (o.n3) ((int*)o.n3)[k] = (int)n3;
  }
}

// ---------------------------------------------------------------------------------------------
// One dataset of a batch (device-resident copy; see batch.cu). Arrays point into the batch's
// workspace; outputs are the caller's.
// ---------------------------------------------------------------------------------------------
struct ktau_bds {
  const void* values;
  int32_t dtype, count_bits;
  int64_t m, n, ld_in;
  int64_t ld;  // row stride (elements) of perm / rank / srank
  uint16_t* perm;
  uint16_t* rank;
  uint16_t* srank;
  int64_t* T;
  double* rs64;
  float2* rsff;
  int32_t* ndist;
  int32_t* maxg;
  ktau_out out;
  int32_t path, esize;
  // merge path: tile side and tiles per side
  int32_t tq;
  int64_t w;
  // tensor-core path: first row in the group's stacked operand, K blocks, super-tiles per side,
  // tie lists (group-wide arrays indexed by the dataset's own rows)
  int64_t srow, num_kb, wS;
  int64_t* tie_off;
  uint32_t* tie_pairs;
  int64_t tie_cap;
};

// ---------------------------------------------------------------------------------------------
// Launchers implemented in the kernel translation units.
// ---------------------------------------------------------------------------------------------
ktau_status ktau_launch_rank(const void* values, int dtype, int64_t m, int64_t n, int64_t ld_in,
                             ktau_ranked* R, cudaStream_t st);
// perm / rank of a 16-bit handle widened to uint32, packed m x n (either pointer may be null).
ktau_status ktau_launch_widen(const ktau_ranked* R, uint32_t* perm, uint32_t* rank,
                              cudaStream_t st);

struct ktau_merge_plan {
  int tile_q;     // tile side
  int mapping;    // 1 warp per pair, 2 CTA per pair
  int schedule;   // 1 static, 2 dynamic
  int ctas_per_sm;
};
void ktau_merge_default_plan(int64_t n, ktau_merge_plan* plan);
// Bit-parallel dominance count over the triangle's pairs [p_begin, p_end) (n <= KTAU_BITS_MAX_N).
ktau_status ktau_bits_allpairs(ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                               const ktau_out& out, cudaStream_t st);
void ktau_bits_release(ktau_ranked* R);
ktau_status ktau_launch_batch_rank(const ktau_bds* ds, int count, const int64_t* row_prefix,
                                   int64_t total_rows, int64_t max_n, ktau_stats* stats,
                                   cudaStream_t st);
// Merge path over the tiles of several datasets (ids[] index ds[]; tile_prefix over ids).
ktau_status ktau_launch_batch_merge(const ktau_bds* ds, const int32_t* ids, int nids,
                                    const int64_t* tile_prefix, int64_t total_tiles, int64_t max_n,
                                    int cta_team, cudaStream_t st);
ktau_status ktau_launch_merge(const ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                              const ktau_out& out, const ktau_merge_plan& plan, cudaStream_t st);
// Every row of Q against every row of D (outputs [Q.m][ldo]).
ktau_status ktau_launch_merge_rect(const ktau_ranked* Q, const ktau_ranked* D, int64_t ldo,
                                   const ktau_out& out, const ktau_merge_plan& plan,
                                   cudaStream_t st);
