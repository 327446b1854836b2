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
// Padding entries (k >= n) hold 0xFFFF.
// ---------------------------------------------------------------------------------------------
struct ktau_stats {
  unsigned long long T_sum;
  unsigned long long T_max;
  unsigned int maxg;
  unsigned int nan_flag;
  unsigned int pad[2];
};

struct ktau_ranked {
  int64_t m, n, ld;
  int device;
  void* block;  // single allocation holding every array below
  uint16_t* perm;
  uint16_t* rank;
  uint16_t* srank;
  int64_t* T;
  int32_t* ndist;
  int32_t* maxg;
  ktau_stats* stats_dev;
  ktau_stats stats;  // host copy, filled by ktau_rank_prepare
  // Sign expansion for the tensor-core path, built on first use (library-owned).
  int8_t* sgn;
  int64_t K, K_pad;
  // Tie-pair lists for n_3 in the tensor-core path, built with the expansion.
  uint32_t* tie_pairs;
  int64_t* tie_off;
  int64_t tie_total;
};

// ---------------------------------------------------------------------------------------------
// Error reporting (thread-local message, see ktau_last_error).
// ---------------------------------------------------------------------------------------------
ktau_status ktau_fail(ktau_status s, const char* fmt, ...);
ktau_status ktau_cuda_fail(cudaError_t e, const char* what);
int ktau_sm_count();

#define KTAU_CUDA(call)                                                   \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return ktau_cuda_fail(e_, #call);              \
  } while (0)

// ---------------------------------------------------------------------------------------------
// Job-id <-> coordinate bijection (Sec. 4.1, Eq. 4-10), applied to a w x w matrix of tiles
// (Sec. 4.2, Eq. 11-14) with the diagonal included.
// ---------------------------------------------------------------------------------------------
__host__ __device__ inline int64_t ktau_rowstart(int64_t w, int64_t y) {  // Eq. 5 / Eq. 12
  return y * (2 * w - y + 1) / 2;
}

// Eq. 13-14: y = ceil(w - 1/2 - sqrt(w^2 + w + 1/4 - 2(J+1))), x = J + y - F(y). The FP64
// square root can land the ceiling one row off when z is (nearly) an integer, so the result is
// checked against F(y) <= J < F(y+1) (Eq. 6) and moved by one row if needed.
__host__ __device__ inline void ktau_tile_coord(int64_t w, int64_t J, int64_t& y, int64_t& x) {
  double wd = (double)w;
  double z = wd - 0.5 - sqrt(wd * wd + wd + 0.25 - 2.0 * ((double)J + 1.0));
  int64_t yy = (int64_t)ceil(z);
  if (yy < 0) yy = 0;
  if (yy > w - 1) yy = w - 1;
  while (yy > 0 && ktau_rowstart(w, yy) > J) --yy;
  while (yy < w - 1 && ktau_rowstart(w, yy + 1) <= J) ++yy;
  y = yy;
  x = J + yy - ktau_rowstart(w, yy);
}

// Packed index of pair (i, j), i < j, in the strict upper triangle of an m x m job matrix
// (Eq. 4 applied to the (m-1)-triangle: p = J_{m-1}(i, j-1)).
__host__ __device__ inline uint64_t ktau_pair_index(int64_t m, int64_t i, int64_t j) {
  return (uint64_t)(i * (2 * m - i - 1) / 2 + (j - i - 1));
}

// ---------------------------------------------------------------------------------------------
// Step 5 of Sec. 3.2 and Eq. 3: S = n_0 - n_1 - n_2 + n_3 - 2 n_d, tau-b in FP64.
// ---------------------------------------------------------------------------------------------
struct ktau_out {
  double* tau64;
  float* tau32;
  void* S;
  void* n3;
  int count_bits;
};

__device__ __forceinline__ double ktau_tau_b(int64_t S, int64_t n0, int64_t Tu, int64_t Tv) {
  int64_t du = n0 - Tu, dv = n0 - Tv;
  if (du == 0 || dv == 0) return __longlong_as_double(0x7ff8000000000000LL);
  return __ddiv_rn((double)S, __dsqrt_rn(__dmul_rn((double)du, (double)dv)));
}

__device__ __forceinline__ void ktau_store(const ktau_out& o, uint64_t k, int64_t S, int64_t n3,
                                           int64_t n0, int64_t Tu, int64_t Tv) {
  if (o.tau64 || o.tau32) {
    double t = ktau_tau_b(S, n0, Tu, Tv);
    if (o.tau64) o.tau64[k] = t;
    if (o.tau32) o.tau32[k] = __double2float_rn(t);
  }
  if (o.count_bits == 64) {
    if (o.S) ((long long*)o.S)[k] = S;
    if (o.n3) ((long long*)o.n3)[k] = n3;
  } else {
    if (o.S) ((int*)o.S)[k] = (int)S;
    if (o.n3) ((int*)o.n3)[k] = (int)n3;
  }
}

// ---------------------------------------------------------------------------------------------
// Launchers implemented in the kernel translation units.
// ---------------------------------------------------------------------------------------------
ktau_status ktau_launch_rank(const void* values, int dtype, int64_t m, int64_t n, int64_t ld_in,
                             ktau_ranked* R, cudaStream_t st);

struct ktau_merge_plan {
  int tile_q;     // tile side
  int mapping;    // 1 warp per pair, 2 CTA per pair
  int schedule;   // 1 static, 2 dynamic
  int ctas_per_sm;
};
void ktau_merge_default_plan(int64_t n, ktau_merge_plan* plan);
ktau_status ktau_launch_merge(const ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                              const ktau_out& out, const ktau_merge_plan& plan, cudaStream_t st);
