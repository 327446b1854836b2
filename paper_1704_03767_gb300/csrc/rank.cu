// K-a: per-variable rank transform (Sec. 3, opening paragraph: values are replaced by ranks
// once per vector before any pair is counted). One CTA per variable sorts the row in shared
// memory and emits the stable permutation pi_u, the dense ranks r_u, the ranks in sorted order,
// and the tie statistics that Steps 2 and 4 of Sec. 3.2 would otherwise rescan for every pair
// (n_1 and n_2 depend on one variable only).
#include <algorithm>
#include <cstdarg>
#include <cstdio>

#include "ktau_impl.cuh"

namespace {

// Order-preserving map of a float to uint32 (IEEE total order on non-NaN values), with -0.0
// folded onto +0.0 so that they compare equal, as the definition's comparisons do.
__device__ __forceinline__ uint32_t orderable_f32(uint32_t b) {
  if (b == 0x80000000u) b = 0u;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Sort key: (orderable value << 32) | sample index, so that a plain ascending sort is a
// stable argsort. Padding keys are all-ones and sort last.
template <int DT>
__device__ __forceinline__ unsigned long long load_key(const void* values, int64_t off, int i,
                                                       unsigned int* nan_seen) {
  uint32_t b = ((const uint32_t*)values)[off + i];
  uint32_t k;
  if (DT == KTAU_F32) {
    if ((b & 0x7fffffffu) > 0x7f800000u) *nan_seen = 1u;
    k = orderable_f32(b);
  } else {
    k = b ^ 0x80000000u;
  }
  return ((unsigned long long)k << 32) | (unsigned)i;
}

// Rank transform of one variable (row `row` of the outputs) by one CTA; `off` is the element
// offset of its values. Shared memory: np2 keys + 2 x np2 uint16.
template <int EPL>
__device__ __forceinline__ void cta_bitonic_hybrid(unsigned long long* sm_keys, int np2);

// Ascending sort of sm_keys[0, np2) (shared memory) by the whole CTA: bitonic network, warp
// blocks in registers where np2 = blockDim * EPL for EPL in 2..8, all through shared memory
// otherwise.
__device__ void cta_sort_keys(unsigned long long* sm_keys, int np2) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int epl = np2 / nt;
  if (epl * nt == np2 && epl >= 2 && epl <= 8) {
    switch (epl) {
      case 2: cta_bitonic_hybrid<2>(sm_keys, np2); break;
      case 4: cta_bitonic_hybrid<4>(sm_keys, np2); break;
      default: cta_bitonic_hybrid<8>(sm_keys, np2); break;
    }
  } else {
    for (int k = 2; k <= np2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < np2 / 2; i += nt) {
          int lo = 2 * i - (i & (j - 1));  // index with bit j clear
          int hi = lo + j;
          bool up = (lo & k) == 0;
          unsigned long long a = sm_keys[lo], b = sm_keys[hi];
          if ((a > b) == up) {
            sm_keys[lo] = b;
            sm_keys[hi] = a;
          }
        }
        __syncthreads();
      }
    }
  }

}

// Outputs of one variable from its keys sorted ascending in keys[0, n) (shared or global memory):
// group heads and dense ranks by a block-wide scan, pi_u, r_u, ranks in sorted order, T_u, the
// number of distinct values, the largest tie group and the denominator factors. first[] and
// dense[] are n-entry work arrays (shared or global). nan_seen: this thread's NaN flag. RT is the
// rank type: uint16_t, or uint32_t for rows longer than 65535 samples.
template <typename RT>
__device__ void rank_finish(const unsigned long long* keys, RT* sm_first, RT* sm_dense, int n,
                            int64_t ld, int64_t row, RT* perm, RT* rank, RT* srank, int64_t* T,
                            int32_t* ndist, int32_t* maxg, double* rs64, float2* rsff,
                            ktau_stats* stats, unsigned int nan_seen) {
  __shared__ int warp_tot[32];
  __shared__ unsigned long long red_T[32];
  __shared__ int red_g[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const unsigned long long* sm_keys = keys;
  // Group heads and dense ranks: a block-wide inclusive scan of head flags over positions,
  // each thread owning a contiguous chunk.
  const int per = (n + nt - 1) / nt;
  const int beg = min(n, tid * per), end = min(n, beg + per);
  int local = 0;
  for (int k = beg; k < end; ++k)
    local += (k == 0) || ((sm_keys[k] >> 32) != (sm_keys[k - 1] >> 32));
  // warp inclusive scan of chunk totals
  const int lane = tid & 31, wid = tid >> 5;
  int incl = local;
  for (int d = 1; d < 32; d <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int nw = (nt + 31) >> 5;
    int v = lane < nw ? warp_tot[lane] : 0;
    for (int d = 1; d < 32; d <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += t;
    }
    if (lane < nw) warp_tot[lane] = v;  // inclusive per-warp prefix
  }
  __syncthreads();
  int run = incl - local + (wid > 0 ? warp_tot[wid - 1] : 0);  // heads before this chunk
  for (int k = beg; k < end; ++k) {
    bool head = (k == 0) || ((sm_keys[k] >> 32) != (sm_keys[k - 1] >> 32));
    run += head;
    sm_dense[k] = (RT)(run - 1);
    if (head) sm_first[run - 1] = (RT)k;
  }
  __syncthreads();

  // Outputs and tie statistics: position k has k - first(group) earlier equal values, so
  // the sum over k is the number of tied pairs, sum t(t-1)/2.
  RT* prow = perm + row * ld;
  RT* rrow = rank + row * ld;
  RT* srow = srank + row * ld;
  constexpr RT kPad = (RT)~(RT)0;
  unsigned long long tsum = 0;
  int gmax = 0;
  for (int k = tid; k < (int)ld; k += nt) {
    if (k < n) {
      int idx = (int)(sm_keys[k] & 0xffffffffu);
      int d = (int)sm_dense[k];
      int before = k - (int)sm_first[d];
      prow[k] = (RT)idx;
      srow[k] = (RT)d;
      rrow[idx] = (RT)d;
      tsum += (unsigned long long)before;
      gmax = max(gmax, before + 1);
    } else {
      prow[k] = kPad;
      srow[k] = kPad;
      rrow[k] = kPad;
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    tsum += __shfl_down_sync(0xffffffffu, tsum, d);
    gmax = max(gmax, __shfl_down_sync(0xffffffffu, gmax, d));
  }
  unsigned int nan_any = __syncthreads_or(nan_seen);
  if (lane == 0) {
    red_T[wid] = tsum;
    red_g[wid] = gmax;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long t = 0;
    int g = 0;
    for (int w = 0; w < (nt + 31) / 32; ++w) {
      t += red_T[w];
      g = max(g, red_g[w]);
    }
    T[row] = (int64_t)t;
    // Factor of the tau-b denominator (Eq. 3): 1/sqrt(n_0 - n_1), IEEE FP64.
    const long long D = (long long)n * (n - 1) / 2 - (long long)t;
    const double r = D > 0 ? __ddiv_rn(1.0, __dsqrt_rn((double)D))
                           : __longlong_as_double(0x7ff8000000000000LL);
    const float hi = __double2float_rn(r);
    rs64[row] = r;
    rsff[row] = make_float2(hi, D > 0 ? __double2float_rn(r - (double)hi) : hi);
    ndist[row] = (int32_t)sm_dense[n - 1] + 1;
    maxg[row] = g;
    atomicAdd(&stats->T_sum, t);
    atomicMax(&stats->T_max, t);
    atomicMax(&stats->maxg, (unsigned)g);
    if (nan_any) atomicOr(&stats->nan_flag, 1u);
  }
}

template <int DT>
__device__ void rank_row(const void* __restrict__ values, int64_t off, int n, int np2,
                         int64_t ld, int64_t row, uint16_t* perm, uint16_t* rank, uint16_t* srank,
                         int64_t* T, int32_t* ndist, int32_t* maxg, double* rs64, float2* rsff,
                         ktau_stats* stats) {
  extern __shared__ unsigned long long sm_keys[];                  // [np2]
  uint16_t* sm_first = reinterpret_cast<uint16_t*>(sm_keys + np2);  // [np2] group start
  uint16_t* sm_dense = sm_first + np2;                             // [np2] dense rank at k
  unsigned int nan_seen = 0;
  for (int i = threadIdx.x; i < np2; i += blockDim.x)
    sm_keys[i] = i < n ? load_key<DT>(values, off, i, &nan_seen) : ~0ull;
  __syncthreads();
  cta_sort_keys(sm_keys, np2);
  rank_finish<uint16_t>(sm_keys, sm_first, sm_dense, n, ld, row, perm, rank, srank, T, ndist,
                        maxg, rs64, rsff, stats, nan_seen);
}

// Short rows (n <= 256): one warp per variable, EPL = np2/32 keys per lane in registers, blocked
// (lane l holds sorted positions l*EPL .. l*EPL+EPL-1). Same outputs, bit for bit, as rank_row.
constexpr int RANK_WARPS = 8;

template <int EPL>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&v)[EPL], int lane) {
#pragma unroll
  for (int k = 2; k <= 32 * EPL; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= EPL) {  // partner in lane ^ (j / EPL), same slot
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int i = lane * EPL + e;
          const unsigned long long y = __shfl_xor_sync(0xffffffffu, v[e], j / EPL);
          const bool take_min = ((i & k) == 0) == ((i & j) == 0);
          v[e] = take_min ? (y < v[e] ? y : v[e]) : (y > v[e] ? y : v[e]);
        }
      } else {  // partner in this lane
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int p = e ^ j;
          if (p > e) {
            const bool up = ((lane * EPL + e) & k) == 0;
            const unsigned long long a = v[e], b = v[p];
            if ((a > b) == up) {
              v[e] = b;
              v[p] = a;
            }
          }
        }
      }
    }
  }
}

// Bitonic merge of a bitonic sequence of 32 * EPL keys held by a warp (position lane * EPL + e)
// into ascending (up) or descending order: the steps j = 16 EPL .. 1 of one phase.
template <int EPL>
__device__ __forceinline__ void warp_merge(unsigned long long (&v)[EPL], int lane, bool up) {
#pragma unroll
  for (int j = 16 * EPL; j > 0; j >>= 1) {
    if (j >= EPL) {
      const bool lower = (lane & (j / EPL)) == 0;  // this lane holds the lower position
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, v[e], j / EPL);
        v[e] = (lower == up) ? (y < v[e] ? y : v[e]) : (y > v[e] ? y : v[e]);
      }
    } else {
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        const int p = e ^ j;
        if (p > e) {
          const unsigned long long a = v[e], b = v[p];
          if ((a > b) == up) {
            v[e] = b;
            v[p] = a;
          }
        }
      }
    }
  }
}

// Reverses the order of the warp's 32 * EPL keys (position p -> 32 EPL - 1 - p).
template <int EPL>
__device__ __forceinline__ void warp_reverse(unsigned long long (&v)[EPL], int lane) {
  unsigned long long r[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) r[e] = __shfl_sync(0xffffffffu, v[EPL - 1 - e], 31 - lane);
#pragma unroll
  for (int e = 0; e < EPL; ++e) v[e] = r[e];
}

// Bitonic sort of sm_keys[0, np2) ascending by a CTA whose warps each own one block of 32 * EPL
// consecutive keys (np2 = blockDim.x * EPL): the phases up to the block size and, in later
// phases, the steps inside a block run in registers with shuffles; only the steps across blocks
// go through shared memory, with one barrier each. The compare-exchange network is the standard
// one (position i pairs with i ^ j, ascending where i & k == 0), so the result is the same.
template <int EPL>
__device__ __forceinline__ void cta_bitonic_hybrid(unsigned long long* sm_keys, int np2) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int B = 32 * EPL;
  const int base = wid * B;
  unsigned long long v[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) v[e] = sm_keys[base + lane * EPL + e];
  warp_bitonic<EPL>(v, lane);               // block ascending
  if (base & B) warp_reverse<EPL>(v, lane);  // odd blocks descending, as the network leaves them
#pragma unroll
  for (int e = 0; e < EPL; ++e) sm_keys[base + lane * EPL + e] = v[e];
  __syncthreads();
  for (int k = 2 * B; k <= np2; k <<= 1) {
    for (int j = k >> 1; j >= B; j >>= 1) {
      for (int i = threadIdx.x; i < np2 / 2; i += blockDim.x) {
        const int lo = 2 * i - (i & (j - 1));  // index with bit j clear
        const int hi = lo + j;
        const bool up = (lo & k) == 0;
        const unsigned long long a = sm_keys[lo], b = sm_keys[hi];
        if ((a > b) == up) {
          sm_keys[lo] = b;
          sm_keys[hi] = a;
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int e = 0; e < EPL; ++e) v[e] = sm_keys[base + lane * EPL + e];
    warp_merge<EPL>(v, lane, (base & k) == 0);
#pragma unroll
    for (int e = 0; e < EPL; ++e) sm_keys[base + lane * EPL + e] = v[e];
    __syncthreads();
  }
}

template <int EPL>
__device__ __forceinline__ void store_u16s(uint16_t* dst, const uint16_t (&x)[EPL]) {
  if (EPL == 1) {
    dst[0] = x[0];
  } else if (EPL == 2) {
    *reinterpret_cast<uint32_t*>(dst) = (uint32_t)x[0] | ((uint32_t)x[1] << 16);
  } else if (EPL == 4) {
    *reinterpret_cast<uint2*>(dst) = make_uint2((uint32_t)x[0] | ((uint32_t)x[1] << 16),
                                                (uint32_t)x[2] | ((uint32_t)x[3] << 16));
  } else {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      w[q] = (uint32_t)x[(2 * q) % EPL] | ((uint32_t)x[(2 * q + 1) % EPL] << 16);
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Rank transform of one variable by one warp (see rank_warp_kernel); `off` is the element offset
// of its values, `row` its row in the outputs. Accumulates the warp's statistics.
template <int DT, int EPL>
__device__ __forceinline__ void rank_warp_row(const void* __restrict__ values, int64_t off, int n,
                                              int64_t ld, int64_t row, uint16_t* __restrict__ perm,
                                              uint16_t* __restrict__ rank,
                                              uint16_t* __restrict__ srank, int64_t* __restrict__ T,
                                              int32_t* __restrict__ ndist,
                                              int32_t* __restrict__ maxg, double* __restrict__ rs64,
                                              float2* __restrict__ rsff, unsigned long long& tsum,
                                              int& gmax, unsigned& nan_seen, int lane) {
  unsigned long long v[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int i = lane * EPL + e;
    v[e] = i < n ? load_key<DT>(values, off, i, &nan_seen) : ~0ull;
  }
  warp_bitonic<EPL>(v, lane);
  // Group heads over sorted positions k < n; dense rank = heads up to k, minus one;
  // first(k) = position of the last head <= k.
  const unsigned long long prev_last = __shfl_up_sync(0xffffffffu, v[EPL - 1], 1);
  int heads = 0, last_head = -1;
  bool head[EPL];
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int k = lane * EPL + e;
    const unsigned long long pv = e == 0 ? prev_last : v[e - 1];
    head[e] = k < n && (k == 0 || (v[e] >> 32) != (pv >> 32));
    heads += head[e];
    if (head[e]) last_head = k;
  }
  int incl = heads, lmax = last_head;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    const int u = __shfl_up_sync(0xffffffffu, lmax, d);
    if (lane >= d) {
      incl += t;
      lmax = u > lmax ? u : lmax;
    }
  }
  int run = incl - heads;                                  // heads before this lane
  int first = __shfl_up_sync(0xffffffffu, lmax, 1);        // last head before this lane
  if (lane == 0) first = -1;
  uint16_t pk[EPL], sk[EPL], pad[EPL];
  uint16_t* rrow = rank + row * ld;
#pragma unroll
  for (int e = 0; e < EPL; ++e) {
    const int k = lane * EPL + e;
    pad[e] = 0xffff;
    if (k < n) {
      run += head[e];
      if (head[e]) first = k;
      const int idx = (int)(v[e] & 0xffffffffu);
      const int d = run - 1;
      const int before = k - first;
      pk[e] = (uint16_t)idx;
      sk[e] = (uint16_t)d;
      rrow[idx] = (uint16_t)d;
      tsum += (unsigned long long)before;
      gmax = before + 1 > gmax ? before + 1 : gmax;
    } else {
      pk[e] = sk[e] = 0xffff;
    }
  }
  // ld is a multiple of 16 and EPL divides 16: a lane's positions are all inside or all
  // outside the padded row.
  if (lane * EPL < ld) {
    store_u16s<EPL>(perm + row * ld + lane * EPL, pk);
    store_u16s<EPL>(srank + row * ld + lane * EPL, sk);
    if (lane * EPL >= n) store_u16s<EPL>(rrow + lane * EPL, pad);
    else if (lane * EPL + EPL > n)
      for (int e = n - lane * EPL; e < EPL; ++e) rrow[lane * EPL + e] = 0xffff;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    tsum += __shfl_xor_sync(0xffffffffu, tsum, d);
    const int o = __shfl_xor_sync(0xffffffffu, gmax, d);
    gmax = o > gmax ? o : gmax;
  }
  const int total_heads = __shfl_sync(0xffffffffu, incl, 31);
  nan_seen = __any_sync(0xffffffffu, nan_seen != 0);
  if (lane == 0) {
    T[row] = (int64_t)tsum;
    // Factor of the tau-b denominator (Eq. 3): 1/sqrt(n_0 - n_1), IEEE FP64.
    const long long D = (long long)n * (n - 1) / 2 - (long long)tsum;
    const double r = D > 0 ? __ddiv_rn(1.0, __dsqrt_rn((double)D))
                           : __longlong_as_double(0x7ff8000000000000LL);
    const float hi = __double2float_rn(r);
    rs64[row] = r;
    rsff[row] = make_float2(hi, D > 0 ? __double2float_rn(r - (double)hi) : hi);
    ndist[row] = total_heads;
    maxg[row] = gmax;
  }
}

// Per-CTA statistics: one set of atomics for the CTA's warps.
__device__ __forceinline__ void rank_warp_stats(unsigned long long tsum, int gmax, unsigned nan_seen,
                                                ktau_stats* stats) {
  __shared__ unsigned long long s_T[RANK_WARPS];
  __shared__ unsigned s_g[RANK_WARPS], s_nan[RANK_WARPS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_T[wid] = tsum;
    s_g[wid] = (unsigned)gmax;
    s_nan[wid] = nan_seen;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0, tm = 0;
    unsigned g = 0, nn = 0;
    for (int w = 0; w < RANK_WARPS; ++w) {
      t += s_T[w];
      tm = s_T[w] > tm ? s_T[w] : tm;
      g = s_g[w] > g ? s_g[w] : g;
      nn |= s_nan[w];
    }
    atomicAdd(&stats->T_sum, t);
    atomicMax(&stats->T_max, tm);
    atomicMax(&stats->maxg, g);
    if (nn) atomicOr(&stats->nan_flag, 1u);
  }
}

template <int DT, int EPL>
__global__ void __launch_bounds__(32 * RANK_WARPS) rank_warp_kernel(
    const void* __restrict__ values, int64_t ld_in, int n, int64_t m, int64_t ld,
    uint16_t* __restrict__ perm, uint16_t* __restrict__ rank, uint16_t* __restrict__ srank,
    int64_t* __restrict__ T, int32_t* __restrict__ ndist, int32_t* __restrict__ maxg,
    double* __restrict__ rs64, float2* __restrict__ rsff, ktau_stats* __restrict__ stats) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row = (int64_t)blockIdx.x * RANK_WARPS + wid;
  unsigned long long tsum = 0;
  int gmax = 0;
  unsigned nan_seen = 0;
  if (row < m)
    rank_warp_row<DT, EPL>(values, row * ld_in, n, ld, row, perm, rank, srank, T, ndist, maxg,
                           rs64, rsff, tsum, gmax, nan_seen, lane);
  rank_warp_stats(tsum, gmax, nan_seen, stats);
}

// Batched form for the variables of datasets with n <= 256: one warp per variable, the dataset
// found from the prefix of row counts; variables of longer datasets are left to batch_rank_kernel.
__global__ void __launch_bounds__(32 * RANK_WARPS) batch_rank_warp_kernel(
    const ktau_bds* __restrict__ ds, int count, const int64_t* __restrict__ row_prefix,
    int64_t total_rows, ktau_stats* __restrict__ stats) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t r = (int64_t)blockIdx.x * RANK_WARPS + wid;
  unsigned long long tsum = 0;
  int gmax = 0;
  unsigned nan_seen = 0;
  if (r < total_rows) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // largest d with row_prefix[d] <= r
      const int mid = (lo + hi + 1) >> 1;
      if (row_prefix[mid] <= r)
        lo = mid;
      else
        hi = mid - 1;
    }
    const ktau_bds& D = ds[lo];
    const int64_t row = r - row_prefix[lo];
    const int n = (int)D.n;
    if (n <= 256) {
      const bool f32 = D.dtype == KTAU_F32;
#define KTAU_BATCH_WARP_ROW(EPL)                                                                 \
  if (f32)                                                                                       \
    rank_warp_row<KTAU_F32, EPL>(D.values, row * D.ld_in, n, D.ld, row, D.perm, D.rank, D.srank, \
                                 D.T, D.ndist, D.maxg, D.rs64, D.rsff, tsum, gmax, nan_seen,     \
                                 lane);                                                          \
  else                                                                                           \
    rank_warp_row<KTAU_I32, EPL>(D.values, row * D.ld_in, n, D.ld, row, D.perm, D.rank, D.srank, \
                                 D.T, D.ndist, D.maxg, D.rs64, D.rsff, tsum, gmax, nan_seen,     \
                                 lane);
      if (n <= 32) {
        KTAU_BATCH_WARP_ROW(1)
      } else if (n <= 64) {
        KTAU_BATCH_WARP_ROW(2)
      } else if (n <= 128) {
        KTAU_BATCH_WARP_ROW(4)
      } else {
        KTAU_BATCH_WARP_ROW(8)
      }
#undef KTAU_BATCH_WARP_ROW
    }
  }
  rank_warp_stats(tsum, gmax, nan_seen, stats);
}

template <int DT>
__global__ void __launch_bounds__(512) rank_kernel(const void* __restrict__ values, int64_t ld_in,
                                                   int n, int np2, int64_t ld, uint16_t* perm,
                                                   uint16_t* rank, uint16_t* srank, int64_t* T,
                                                   int32_t* ndist, int32_t* maxg,
                                                   double* rs64, float2* rsff,
                                                   ktau_stats* stats) {
  const int64_t row = blockIdx.x;
  rank_row<DT>(values, row * ld_in, n, np2, ld, row, perm, rank, srank, T, ndist, maxg, rs64, rsff,
               stats);
}

// Long rows (n > KTAU_RANK_CHUNK), a pass over up to kLongRows variables at a time, in four small
// kernels over global scratch: sort keys of every element (long_keys_kernel), chunks of
// KTAU_RANK_CHUNK keys sorted in shared memory (long_chunk_kernel), the sorted chunks merged level
// by level (long_merge_kernel, one launch per level), and the outputs of each variable
// (long_finish_kernel). Scratch per variable: two key arrays of np2 and two work arrays of the
// rank type (uint16, or uint32 above 65535 samples). A pass holds at most kLongRows variables and
// at most kLongBudget bytes of scratch (at least one variable).
constexpr int kLongRows = 256;
constexpr size_t kLongBudget = (size_t)1 << 30;
constexpr int LONG_THREADS = 512;
__host__ __device__ inline size_t long_rank_scratch(int64_t np2, size_t rank_bytes) {
  return (size_t)np2 * (2 * sizeof(unsigned long long) + 2 * rank_bytes);
}

template <int DT>
__global__ void __launch_bounds__(256) long_keys_kernel(const void* __restrict__ values,
                                                        int64_t ld_in, int n, int np2,
                                                        int64_t row0, int rows,
                                                        unsigned long long* __restrict__ keys,
                                                        ktau_stats* stats) {
  unsigned int nan_seen = 0;
  const int64_t total = (int64_t)rows * np2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / np2;
    const int k = (int)(i - r * np2);
    keys[i] = k < n ? load_key<DT>(values, (row0 + r) * ld_in, k, &nan_seen) : ~0ull;
  }
  if (__any_sync(0xffffffffu, nan_seen != 0) && (threadIdx.x & 31) == 0)
    atomicOr(&stats->nan_flag, 1u);
}

// One CTA per chunk of KTAU_RANK_CHUNK keys (chunks of a variable are consecutive).
__global__ void __launch_bounds__(LONG_THREADS) long_chunk_kernel(unsigned long long* keys) {
  extern __shared__ unsigned long long sm_keys[];  // [KTAU_RANK_CHUNK]
  unsigned long long* g = keys + (size_t)blockIdx.x * KTAU_RANK_CHUNK;
  for (int i = threadIdx.x; i < KTAU_RANK_CHUNK; i += blockDim.x) sm_keys[i] = g[i];
  __syncthreads();
  cta_sort_keys(sm_keys, KTAU_RANK_CHUNK);
  for (int i = threadIdx.x; i < KTAU_RANK_CHUNK; i += blockDim.x) g[i] = sm_keys[i];
}

// One merge level: runs of s sorted keys, pairs of runs merged into `out`. Each thread writes
// `per` consecutive outputs of one pair of runs: it finds how many come from the left run by
// binary search along its diagonal (merge path), then merges them serially. Keys are unique
// (the sample index is their low word) except the all-ones padding, which sorts last.
__global__ void __launch_bounds__(256) long_merge_kernel(const unsigned long long* __restrict__ in,
                                                         unsigned long long* __restrict__ out,
                                                         int64_t total, int s, int per) {
  const int64_t o = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * per;
  if (o >= total) return;
  const int64_t A = (o / (2 * (int64_t)s)) * (2 * (int64_t)s), B = A + s;
  const int diag = (int)(o - A);
  int lo = max(0, diag - s), hi = min(diag, s);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (in[A + mid] <= in[B + diag - 1 - mid])
      lo = mid + 1;
    else
      hi = mid;
  }
  int ai = lo, bi = diag - lo;
  for (int k = 0; k < per; ++k) {
    const unsigned long long va = ai < s ? in[A + ai] : ~0ull;
    const unsigned long long vb = bi < s ? in[B + bi] : ~0ull;
    if (bi < s && (ai >= s || vb < va)) {
      out[o + k] = vb;
      ++bi;
    } else {
      out[o + k] = va;
      ++ai;
    }
  }
}

// Outputs of each variable of the pass from its sorted keys (one CTA per variable).
template <typename RT>
__global__ void __launch_bounds__(LONG_THREADS) long_finish_kernel(
    const unsigned long long* __restrict__ keys, RT* work, int n, int np2, int64_t row0,
    int64_t ld, RT* perm, RT* rank, RT* srank, int64_t* T, int32_t* ndist, int32_t* maxg,
    double* rs64, float2* rsff, ktau_stats* stats) {
  const int r = blockIdx.x;
  RT* first = work + (size_t)r * 2 * np2;
  rank_finish<RT>(keys + (size_t)r * np2, first, first + np2, n, ld, row0 + r, perm, rank, srank,
                  T, ndist, maxg, rs64, rsff, stats, 0u);
}

// uint16 perm / rank rows widened to packed uint32 rows (one thread per element).
__global__ void widen_kernel(const uint16_t* __restrict__ src, int64_t ld, int64_t m, int64_t n,
                             uint32_t* __restrict__ dst) {
  const int64_t total = m * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n;
    dst[i] = src[r * ld + (i - r * n)];
  }
}

// Batched form: one CTA per variable of every dataset; the dataset is found from the prefix of
// row counts (rows of a batch are numbered dataset by dataset).
__global__ void __launch_bounds__(256) batch_rank_kernel(const ktau_bds* __restrict__ ds, int count,
                                                         const int64_t* __restrict__ row_prefix,
                                                         ktau_stats* stats) {
  const int64_t r = blockIdx.x;
  int lo = 0, hi = count - 1;
  while (lo < hi) {  // largest d with row_prefix[d] <= r
    const int mid = (lo + hi + 1) >> 1;
    if (row_prefix[mid] <= r)
      lo = mid;
    else
      hi = mid - 1;
  }
  const ktau_bds& D = ds[lo];
  if (D.n <= 256) return;  // ranked by batch_rank_warp_kernel
  const int64_t row = r - row_prefix[lo];
  int np2 = 32;
  while (np2 < D.n) np2 <<= 1;
  if (D.dtype == KTAU_F32)
    rank_row<KTAU_F32>(D.values, row * D.ld_in, (int)D.n, np2, D.ld, row, D.perm, D.rank, D.srank,
                       D.T, D.ndist, D.maxg, D.rs64, D.rsff, stats);
  else
    rank_row<KTAU_I32>(D.values, row * D.ld_in, (int)D.n, np2, D.ld, row, D.perm, D.rank, D.srank,
                       D.T, D.ndist, D.maxg, D.rs64, D.rsff, stats);
}

}  // namespace

ktau_status ktau_launch_batch_rank(const ktau_bds* ds, int count, const int64_t* row_prefix,
                                   int64_t total_rows, int64_t max_n, ktau_stats* stats,
                                   cudaStream_t st) {
  int np2 = 32;
  while (np2 < max_n) np2 <<= 1;
  const size_t smem = (size_t)np2 * (sizeof(unsigned long long) + 2 * sizeof(uint16_t));
  KTAU_CUDA(cudaFuncSetAttribute(batch_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  if (total_rows > 0x7fffffffLL) return ktau_fail(KTAU_ETOOLARGE, "too many rows in one batch");
  {
    KTAU_TRACE("batch_rank_warp_kernel", st);
    batch_rank_warp_kernel<<<(unsigned)((total_rows + RANK_WARPS - 1) / RANK_WARPS),
                             32 * RANK_WARPS, 0, st>>>(ds, count, row_prefix, total_rows, stats);
  }
  KTAU_CUDA(cudaGetLastError());
  if (max_n > 256) {
    KTAU_TRACE("batch_rank_kernel", st);
    batch_rank_kernel<<<(unsigned)total_rows, 256, smem, st>>>(ds, count, row_prefix, stats);
  }
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

ktau_status ktau_launch_rank(const void* values, int dtype, int64_t m, int64_t n, int64_t ld_in,
                             ktau_ranked* R, cudaStream_t st) {
  int np2 = 32;
  while (np2 < n) np2 <<= 1;
  if (m > 0x7fffffffLL) return ktau_fail(KTAU_ETOOLARGE, "m too large for one launch");
  if (np2 <= 256) {
    const unsigned blocks = (unsigned)((m + RANK_WARPS - 1) / RANK_WARPS);
    const bool f32 = dtype == KTAU_F32;
    KTAU_TRACE("rank_kernel", st);
#define KTAU_RANK_WARP(EPL)                                                                    \
  (f32 ? rank_warp_kernel<KTAU_F32, EPL> : rank_warp_kernel<KTAU_I32, EPL>)<<<               \
      blocks, 32 * RANK_WARPS, 0, st>>>(values, ld_in, (int)n, m, R->ld, R->perm, R->rank,     \
                                        R->srank, R->T, R->ndist, R->maxg, R->rs64, R->rsff, \
                                        R->stats_dev)
    switch (np2) {
      case 32: KTAU_RANK_WARP(1); break;
      case 64: KTAU_RANK_WARP(2); break;
      case 128: KTAU_RANK_WARP(4); break;
      default: KTAU_RANK_WARP(8); break;
    }
#undef KTAU_RANK_WARP
    KTAU_CUDA(cudaGetLastError());
    return KTAU_OK;
  }
  if (np2 > KTAU_RANK_CHUNK) {
    // Long rows: global scratch for up to kLongRows variables per pass, released by the handle
    // once the rank transform has run (ktau_ranked_stats).
    if (!R->block) return ktau_fail(KTAU_EINVAL, "rows longer than %d need a library handle",
                                    KTAU_RANK_CHUNK);
    const size_t rb = R->wide ? sizeof(uint32_t) : sizeof(uint16_t);
    int64_t pass = m < kLongRows ? m : kLongRows;
    while (pass > 1 && (size_t)pass * long_rank_scratch(np2, rb) > kLongBudget) pass >>= 1;
    const size_t kbytes = (size_t)pass * np2 * sizeof(unsigned long long);
    R->tmp_bytes = (size_t)pass * long_rank_scratch(np2, rb);
    if (ktau_dmalloc(&R->tmp_block, R->tmp_bytes) != KTAU_OK) {
      R->tmp_block = nullptr;
      return KTAU_ENOMEM;
    }
    unsigned long long* ka = (unsigned long long*)R->tmp_block;
    unsigned long long* kb = (unsigned long long*)((char*)R->tmp_block + kbytes);
    void* work = (char*)R->tmp_block + 2 * kbytes;
    const size_t smem_c = (size_t)KTAU_RANK_CHUNK * sizeof(unsigned long long);
    KTAU_CUDA(cudaFuncSetAttribute(long_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_c));
    auto kk = dtype == KTAU_F32 ? long_keys_kernel<KTAU_F32> : long_keys_kernel<KTAU_I32>;
    const int per = 16;  // merge outputs per thread (divides every run length)
    for (int64_t row0 = 0; row0 < m; row0 += pass) {
      const int rows = (int)(m - row0 < pass ? m - row0 : pass);
      const int64_t total = (int64_t)rows * np2;
      {
        KTAU_TRACE("long_keys_kernel", st);
        kk<<<(unsigned)std::min<int64_t>((total + 255) / 256, 8LL * ktau_sm_count()), 256, 0, st>>>(
            values, ld_in, (int)n, np2, row0, rows, ka, R->stats_dev);
      }
      KTAU_CUDA(cudaGetLastError());
      {
        KTAU_TRACE("long_chunk_kernel", st);
        long_chunk_kernel<<<(unsigned)(total / KTAU_RANK_CHUNK), LONG_THREADS, smem_c, st>>>(ka);
      }
      KTAU_CUDA(cudaGetLastError());
      unsigned long long* in = ka;
      unsigned long long* out = kb;
      for (int s = KTAU_RANK_CHUNK; s < np2; s <<= 1) {
        KTAU_TRACE("long_merge_kernel", st);
        const int64_t threads_total = total / per;
        long_merge_kernel<<<(unsigned)((threads_total + 255) / 256), 256, 0, st>>>(in, out, total, s,
                                                                                  per);
        KTAU_CUDA(cudaGetLastError());
        unsigned long long* t = in;
        in = out;
        out = t;
      }
      {
        KTAU_TRACE("long_finish_kernel", st);
        if (R->wide)
          long_finish_kernel<uint32_t><<<(unsigned)rows, LONG_THREADS, 0, st>>>(
              in, (uint32_t*)work, (int)n, np2, row0, R->ld, R->perm32, R->rank32, R->srank32,
              R->T, R->ndist, R->maxg, R->rs64, R->rsff, R->stats_dev);
        else
          long_finish_kernel<uint16_t><<<(unsigned)rows, LONG_THREADS, 0, st>>>(
              in, (uint16_t*)work, (int)n, np2, row0, R->ld, R->perm, R->rank, R->srank, R->T,
              R->ndist, R->maxg, R->rs64, R->rsff, R->stats_dev);
      }
      KTAU_CUDA(cudaGetLastError());
    }
    return KTAU_OK;
  }
  int threads = np2 / 2 < 32 ? 32 : (np2 / 2 > 512 ? 512 : np2 / 2);
  size_t smem = (size_t)np2 * (sizeof(unsigned long long) + 2 * sizeof(uint16_t));
  if (m > 0x7fffffffLL) return ktau_fail(KTAU_ETOOLARGE, "m too large for one launch");
  auto kern = dtype == KTAU_F32 ? rank_kernel<KTAU_F32> : rank_kernel<KTAU_I32>;
  KTAU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  KTAU_TRACE("rank_kernel", st);
  kern<<<(unsigned)m, threads, smem, st>>>(values, ld_in, (int)n, np2, R->ld, R->perm, R->rank,
                                            R->srank, R->T, R->ndist, R->maxg, R->rs64, R->rsff,
                                            R->stats_dev);
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

ktau_status ktau_launch_widen(const ktau_ranked* R, uint32_t* perm, uint32_t* rank,
                              cudaStream_t st) {
  const int64_t total = R->m * R->n;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 8LL * ktau_sm_count());
  if (total == 0) return KTAU_OK;
  if (perm) {
    KTAU_TRACE("widen_kernel", st);
    widen_kernel<<<blocks, 256, 0, st>>>(R->perm, R->ld, R->m, R->n, perm);
    KTAU_CUDA(cudaGetLastError());
  }
  if (rank) {
    KTAU_TRACE("widen_kernel", st);
    widen_kernel<<<blocks, 256, 0, st>>>(R->rank, R->ld, R->m, R->n, rank);
    KTAU_CUDA(cudaGetLastError());
  }
  return KTAU_OK;
}
