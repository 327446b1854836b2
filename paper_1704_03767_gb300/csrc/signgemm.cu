// K-c: exact sign-matrix contraction on the GB300 tensor cores (see signgemm.cuh).
//
// Kernels
//   sign_expand_kernel : A_u[k] = sign(r_u[(i + d) mod n] - r_u[i]) for the k-th sample pair
//                        (i, d) in circulant order (below), encoded as FP8 e4m3, FP4 e2m1 or
//                        BF16, zero padded to K_pad.
//   contract_kernel    : persistent, warp-specialised tcgen05 GEMM over the upper triangle (or
//                        the query rectangle). The accumulator is computed transposed, S^T =
//                        A_cols A_rows^T: TMEM lanes are 128 output columns v and TMEM columns
//                        are up to 256 output rows u, so a tcgen05.ld register is one row and a
//                        store across the 32 lanes is contiguous along the packed output row.
//                        Super-tiles of 256 x 256 are walked through the job-id bijection of
//                        Sec. 4.1 (Eq. 13-14) and split into two 128-column halves.
//                        warp 0: TMA producer (cp.async.bulk.tensor, 128B swizzle, 4-stage ring)
//                        warp 1: TMEM allocation + single-thread tcgen05.mma issue
//                        warps 2-9: epilogue, tcgen05.ld of the FP32 accumulator (exact integers),
//                                   tau-b, coalesced stores straight from registers.
//   joint_ties_kernel  : n_3 for every pair from the variables' tie groups (see below).
//                        Two TMEM accumulators (2 x 256 columns) let the epilogue of one tile run
//                        under the MMAs of the next. Every mbarrier wait is bounded (about 2 s);
//                        on timeout the kernel raises an error word and every role winds down.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "signgemm.cuh"

namespace {

constexpr int BM = 128;            // output columns of a unit (TMEM lanes, MMA M)
constexpr int BN = 256;            // output rows of a unit, at most (TMEM columns, MMA N)
constexpr int BKB = 128;           // bytes of K per stage row (one 128B swizzle atom row)
constexpr int STAGES = 4;
// Rectangular kernel with at most 128 output rows per unit (one 128-row box of the row operand):
// 32 KB stages, so six fit where four 48 KB ones do (more operand bytes in flight).
constexpr int STAGES_MAX = 6;
constexpr int A_BYTES = BM * BKB;  // 16 KB
constexpr int B_BYTES = BN * BKB;  // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 8;       // two warps per TMEM lane quarter, each half of the rows
constexpr int GROUP = 8;           // super-tiles per side of a traversal group (L2 locality)
constexpr int THREADS = 64 + 32 * EPI_WARPS;
// Per-row data of the 32 rows an epilogue warp is storing (broadcast reads from shared memory).
struct RowInfo {
  float rhi, rlo;   // float-float 1/sqrt(n_0 - T_u)
  long long base;   // packed index of (u, 0) (triangle) or u * ldo (rectangle)
};
constexpr int RI_ROWS = BN / 2;  // rows of one epilogue warp's half of a unit
constexpr size_t SMEM_BYTES = 1024 /*align*/ + (size_t)STAGES * STAGE_BYTES +
                              (size_t)EPI_WARPS * RI_ROWS * sizeof(RowInfo) + 256 /*barriers*/;
// Pair form (two CTAs of a cluster share one tcgen05.mma.cta_group::2 of M = 256): each CTA
// holds its 128 column variables (A) and half of the 256 row variables (B) per stage.
constexpr int STAGES2 = 7;
constexpr int STAGE2_BYTES = A_BYTES + BM * BKB;  // 32 KB
constexpr size_t SMEM2_BYTES = 1024 /*align*/ + (size_t)STAGES2 * STAGE2_BYTES + 256 /*barriers*/;
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded waits: 2 s
constexpr int kMxFmt = 9;  // ContractArgs::afmt of block-scaled FP4 operands
// Block-scaled FP4 pair kernel: TMEM holds two accumulators and the scale factors, so its MMA is
// N = 240 rows (accumulators at columns 0 and 256, scale factors at columns 496..511) and its
// super-tiles are 240 x 240. The column operand is still loaded as 256 rows (M = 256 of the pair);
// the 16 columns past the super-tile are the next super-tile's first columns, whose counts (and
// hence outputs) are identical, so storing them again is harmless.
constexpr int MXT = 240;       // super-tile side
constexpr int MXB = MXT / 2;   // row-operand rows per CTA
constexpr uint32_t kSfCol = 496;
// Pair kernel with block-scaled FP4: stages of 16 KB (column operand) + 15 KB (120 rows), and a
// 32-row slot of row data per epilogue warp (broadcast reads instead of shuffles).
constexpr int STAGE2_MX_BYTES = 128 * 128 + MXB * 128;
// Epilogue warps of the pair kernel: four per TMEM lane quarter, each a quarter of the unit's rows
// (more warps in flight hide the latency of the per-output arithmetic and stores).
constexpr int PAIR_EW = 8;
constexpr int PAIR_THREADS = 64 + 32 * PAIR_EW;
constexpr size_t SMEM2_MX_BYTES = 1024 + (size_t)7 * STAGE2_MX_BYTES +
                                  (size_t)PAIR_EW * 32 * 16 /*row slots*/ + 256 /*barriers*/;
static_assert(SMEM2_MX_BYTES <= 232448, "shared memory of the block-scaled pair kernel");
static_assert(STAGE2_MX_BYTES % 1024 == 0, "stages start on 1024-byte swizzle atoms");

__device__ unsigned int g_sg_error;  // set when a bounded wait gives up

// ---------------------------------------------------------------------------------------------
// Sign expansion
// ---------------------------------------------------------------------------------------------
// Order of the sample pairs in the operands (circulant order): position k < K holds the pair
// (i, (i + d) mod n) with d = k / n + 1 and i = k mod n. Offsets d = 1 .. floor((n - 1) / 2) take
// every i; for even n the offset n / 2 takes i < n / 2 only, which is exactly k < K = n (n - 1) / 2.
// Every unordered sample pair appears once, and the sign is taken in the same direction for every
// variable, so A_u . A_v is n_c - n_d (Algorithm 1 sums over the pairs in any order). In this order
// eight consecutive positions read two contiguous runs of ranks, r[i0 ..] and r[i0 + d ..], except
// where i passes n - 1 inside the eight (then d advances and the partner run skips one sample).
//
// A CTA expands up to ktau_expand_rows(n) variables. Each variable's ranks sit in shared memory
// as eight copies of the ranks repeated past n, copy c holding r[(x + c) mod n] at x, so a run that
// starts anywhere is one aligned 16-byte load from copy (start mod 8). A thread takes eight
// positions at a time for every variable of the CTA: b - a for the two runs in packed 16-bit lanes
// gives the signs of eight pairs in eight adds (ranks are below 2^15, so no lane borrows: bit 15
// of each lane of b - a + 0x7fff is b > a, of b - a + 0x8000 is b >= a), then packed into the operand
// encoding: FP8 e4m3 (+1 = 0x38, -1 = 0xB8), BF16 (0x3F80 / 0xBF80) or FP4 e2m1 (+1 = 0x2,
// -1 = 0xA, element b of the eight in the high nibble of byte b, element 4 + b in the low nibble).
// Positions K <= k < K_pad are zero.
__host__ __device__ __forceinline__ int expand_copy_len(int n) { return (n + 24 + 7) & ~7; }
// 16 warps per CTA: at n > 1024 a CTA holds 66 KB of rank copies, three CTAs per SM, and the
// shared-memory load latency needs the 48 resident warps that gives.
constexpr int kExpandThreads = 512;
__host__ __device__ __forceinline__ size_t expand_smem(int64_t max_n) {
  return (size_t)ktau_expand_rows(max_n) * 8 * expand_copy_len((int)max_n) * sizeof(uint16_t);
}

// prmt.b32 in its default mode: a selector nibble with bit 3 set fills the result byte with the
// sign bit of the selected byte (0xFF or 0x00).
__device__ __forceinline__ uint32_t prmt_sx(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

// Operand bytes of eight signs from the flag words: bit 15 / 31 of G[t] = (b > a) for elements
// 2t / 2t + 1, of E[t] = (b >= a). The flags become byte masks (sign-filling byte permutes), and
// two logic ops per word give the codes: ne = gt | !ge selects the magnitude bits, !ge the sign.
// ABS (FP4 only): the magnitudes |sign| instead, 1.0 (0x2) where the pair is not tied, else 0.
template <int OB, bool ABS = false>
__device__ __forceinline__ void encode_store(const uint32_t (&G)[4], const uint32_t (&E)[4],
                                             uint8_t* __restrict__ dst) {
  if (OB == 4) {
    const uint32_t mg0 = prmt_sx(G[0], G[1], 0xFDB9u), mg1 = prmt_sx(G[2], G[3], 0xFDB9u);
    const uint32_t me0 = prmt_sx(E[0], E[1], 0xFDB9u), me1 = prmt_sx(E[2], E[3], 0xFDB9u);
    // nibble masks: element b in the high nibble of byte b, element 4 + b in the low nibble
    const uint32_t hg = (mg0 & 0xF0F0F0F0u) | (mg1 & 0x0F0F0F0Fu);
    const uint32_t he = (me0 & 0xF0F0F0F0u) | (me1 & 0x0F0F0F0Fu);
    *reinterpret_cast<uint32_t*>(dst) =
        ABS ? ((hg | ~he) & 0x22222222u) : (((hg | ~he) & 0x22222222u) | (~he & 0x88888888u));
  } else if (OB == 8) {
    uint32_t w[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t mg = prmt_sx(G[2 * h], G[2 * h + 1], 0xFDB9u);
      const uint32_t me = prmt_sx(E[2 * h], E[2 * h + 1], 0xFDB9u);
      w[h] = ((mg | ~me) & 0x38383838u) | (~me & 0x80808080u);
    }
    *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
  } else {
    uint32_t w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const uint32_t mg = prmt_sx(G[t], G[t], 0xBB99u), me = prmt_sx(E[t], E[t], 0xBB99u);
      w[t] = ((mg | ~me) & 0x3F803F80u) | (~me & 0x80008000u);
    }
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Eight ranks r[(x0 + e) mod n], e < 8, of one variable as four packed words: one 16-byte load
// where they are an aligned run of the row, else one by one.
__device__ __forceinline__ void load_rank_run(const uint16_t* __restrict__ src, int n, int x0,
                                              uint32_t* w) {
  int x = x0;
  while (x >= n) x -= n;
  if ((x & 7) == 0 && x + 8 <= n) {
    const uint4 v = *reinterpret_cast<const uint4*>(src + x);
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
    return;
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    uint32_t h[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      int xe = x + 2 * t + e;
      while (xe >= n) xe -= n;
      h[e] = src[xe];
    }
    w[t] = h[0] | (h[1] << 16);
  }
}

// Signs of `rows` <= RR variables (ranks rank[r * ld + x]) into out[r * row_bytes + ...],
// positions [0, K_pad). s_r: 8 * expand_copy_len(n) uint16 per variable, 16-byte aligned.
template <int OB, int RR, bool ABS = false>
__device__ __forceinline__ void expand_block(const uint16_t* __restrict__ rank, int64_t ld,
                                             int rows, int n, int K, int K_pad,
                                             uint8_t* __restrict__ out, int64_t row_bytes,
                                             uint16_t* __restrict__ s_r) {
  const int LS = expand_copy_len(n);
  const int RS = 8 * LS;   // elements per variable
  const int CH = LS / 8 - 1;  // 8-element chunks of every copy that are read (x < LS - 8)
  // the eight copies, chunk by chunk: chunk y of copy c = r[(8y + c + e) mod n], e < 8
  for (int idx = threadIdx.x; idx < rows * CH; idx += blockDim.x) {
    const int r = idx / CH, y = idx - r * CH;
    const uint16_t* src = rank + (int64_t)r * ld;
    uint32_t w[8];
    load_rank_run(src, n, 8 * y, w);
    load_rank_run(src, n, 8 * y + 8, w + 4);
    uint16_t* dst = s_r + r * RS + 8 * y;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      uint32_t o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int u = j + (c >> 1);
        o[j] = (c & 1) ? __funnelshift_r(w[u], w[u + 1], 16) : w[u];
      }
      *reinterpret_cast<uint4*>(dst + c * LS) = make_uint4(o[0], o[1], o[2], o[3]);
    }
  }
  __syncthreads();

  constexpr int UB = OB;  // bytes of eight elements
  const int units = K_pad >> 3;
  // (d, i0) = (k0 / n, k0 % n) of this thread's first position, then advanced by the loop's
  // stride of 8 * blockDim positions with one conditional wrap (no division per iteration).
  const int kstep = 8 * (int)blockDim.x;
  const int dstep = kstep / n, istep = kstep - dstep * n;
  int dq = (8 * (int)threadIdx.x) / n;
  int iq = 8 * (int)threadIdx.x - dq * n;
  for (int q = threadIdx.x; q < units;
       q += blockDim.x, dq += dstep, iq += istep, dq += iq >= n ? 1 : 0, iq -= iq >= n ? n : 0) {
    const int k0 = q << 3;
    uint8_t* dst = out + (int64_t)q * UB;
    if (k0 >= K) {  // padding
      for (int r = 0; r < rows; ++r) {
        if (OB == 4)
          *reinterpret_cast<uint32_t*>(dst + r * row_bytes) = 0u;
        else if (OB == 8)
          *reinterpret_cast<uint2*>(dst + r * row_bytes) = make_uint2(0u, 0u);
        else
          *reinterpret_cast<uint4*>(dst + r * row_bytes) = make_uint4(0u, 0u, 0u, 0u);
      }
      continue;
    }
    if (n < 8 || K - k0 < 8) {
      // short rows (the eight positions may span several offsets) and the last, partly valid
      // eight of a row: pairs one by one from copy 0, positions k >= K compare equal (sign 0)
      for (int r = 0; r < rows; ++r) {
        const uint16_t* row = s_r + r * RS;
        uint32_t A[4] = {0u, 0u, 0u, 0u}, B[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = k0 + e;
          if (k < K) {
            const int i = k % n, j = (i + k / n + 1) % n;
            A[e >> 1] |= (uint32_t)row[i] << (16 * (e & 1));
            B[e >> 1] |= (uint32_t)row[j] << (16 * (e & 1));
          }
        }
        uint32_t G[4], E[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          G[t] = B[t] - A[t] + 0x7FFF7FFFu;
          E[t] = B[t] - A[t] + 0x80008000u;
        }
        encode_store<OB, ABS>(G, E, dst + r * row_bytes);
      }
      continue;
    }
    const int d = dq, i0 = iq;  // k0 = d * n + i0
    int s = i0 + d + 1;  // partner run r[s ..], reduced mod n
    if (s >= n) s -= n;
    const int c = n - i0;  // elements 0 .. c-1 take offset d + 1, the rest d + 2 (one sample on)
    const int offA = (i0 & 7) * LS + (i0 & ~7);
    const int offX = (s & 7) * LS + (s & ~7);
    if (c >= 8) {
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        if (r >= rows) break;
        const uint16_t* row = s_r + r * RS;
        const uint4 a4 = *reinterpret_cast<const uint4*>(row + offA);
        const uint4 b4 = *reinterpret_cast<const uint4*>(row + offX);
        const uint32_t G[4] = {b4.x - a4.x + 0x7FFF7FFFu, b4.y - a4.y + 0x7FFF7FFFu,
                               b4.z - a4.z + 0x7FFF7FFFu, b4.w - a4.w + 0x7FFF7FFFu};
        const uint32_t E[4] = {b4.x - a4.x + 0x80008000u, b4.y - a4.y + 0x80008000u,
                               b4.z - a4.z + 0x80008000u, b4.w - a4.w + 0x80008000u};
        encode_store<OB, ABS>(G, E, dst + r * row_bytes);
      }
    } else {
      const int offY = ((s + 1) & 7) * LS + ((s + 1) & ~7);
      uint32_t sel[4];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        sel[t] = 0x3210u + (2 * t + 1 >= c ? 0x4400u : 0u) + (2 * t >= c ? 0x0044u : 0u);
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        if (r >= rows) break;
        const uint16_t* row = s_r + r * RS;
        const uint4 a4 = *reinterpret_cast<const uint4*>(row + offA);
        const uint4 x4 = *reinterpret_cast<const uint4*>(row + offX);
        const uint4 y4 = *reinterpret_cast<const uint4*>(row + offY);
        const uint32_t A[4] = {a4.x, a4.y, a4.z, a4.w};
        const uint32_t B[4] = {__byte_perm(x4.x, y4.x, sel[0]), __byte_perm(x4.y, y4.y, sel[1]),
                               __byte_perm(x4.z, y4.z, sel[2]), __byte_perm(x4.w, y4.w, sel[3])};
        uint32_t G[4], E[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          G[t] = B[t] - A[t] + 0x7FFF7FFFu;
          E[t] = B[t] - A[t] + 0x80008000u;
        }
        encode_store<OB, ABS>(G, E, dst + r * row_bytes);
      }
    }
  }
}

template <int OB, int RR, bool ABS = false>
__global__ void __launch_bounds__(kExpandThreads) sign_expand_kernel(const uint16_t* __restrict__ rank,
                                                          int64_t ld, int n, int64_t m, int K,
                                                          int K_pad, uint8_t* __restrict__ out) {
  extern __shared__ __align__(16) uint16_t s_r[];
  const int64_t row0 = (int64_t)blockIdx.x * RR;
  const int rows = (int)min((int64_t)RR, m - row0);
  const int64_t row_bytes = (int64_t)K_pad * OB / 8;
  expand_block<OB, RR, ABS>(rank + row0 * ld, ld, rows, n, K, K_pad, out + row0 * row_bytes,
                            row_bytes, s_r);
}

// Batched: blocks of up to RR variables of one dataset (numbered dataset by dataset, prefix
// blk_prefix over bids), written into the group's stacked operand (row stride `stride` bytes,
// dataset rows from srow). Each row is written up to its own dataset's K_pad.
template <int OB, int RR>
__global__ void __launch_bounds__(kExpandThreads) batch_sign_expand_kernel(
    const ktau_bds* __restrict__ ds, const int32_t* __restrict__ bids, int nb,
    const int64_t* __restrict__ blk_prefix, int64_t stride, uint8_t* __restrict__ out) {
  extern __shared__ __align__(16) uint16_t s_r[];
  const int64_t blk = blockIdx.x;
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (blk_prefix[mid] <= blk)
      lo = mid;
    else
      hi = mid - 1;
  }
  const ktau_bds& D = ds[bids[lo]];
  const int64_t row0 = (blk - blk_prefix[lo]) * RR;
  const int rows = (int)min((int64_t)RR, D.m - row0);
  const int n = (int)D.n;
  const int K = n * (n - 1) / 2;
  const int K_pad = (int)ktau_kpad(K, OB);
  expand_block<OB, RR>(D.rank + row0 * D.ld, D.ld, rows, n, K, K_pad, out + (D.srow + row0) * stride,
                   stride, s_r);
}

// Ranks of every variable with its samples relabelled: out[v][k] = rank[v][sigma[k]] for k < n,
// the padding slots (k >= n) 0xffff as in a ranked handle.
__global__ void permute_ranks_kernel(const uint16_t* __restrict__ rank, int64_t ld, int n,
                                     int64_t m, const uint16_t* __restrict__ sigma,
                                     uint16_t* __restrict__ out) {
  const int64_t total = m * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / ld;
    const int k = (int)(i - v * ld);
    const int src = min((int)sigma[k], n - 1);  // entries outside 0..n-1 cannot read out of the row
    out[i] = k < n ? rank[v * ld + src] : (uint16_t)0xffffu;
  }
}

// ---------------------------------------------------------------------------------------------
// PTX wrappers (tcgen05, TMA, mbarrier)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.b32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the error word is already set or the wait exceeded kWaitNs.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 256; ++i)
      if (mbar_try(bar, parity)) return true;
    if (*(volatile unsigned int*)&g_sg_error) return false;
    if (gtimer() - t0 > kWaitNs) {
      atomicExch(&g_sg_error, 1u);
      return false;
    }
  }
}
__device__ __forceinline__ bool sg_failed() { return *(volatile unsigned int*)&g_sg_error != 0; }

// The same bounded wait with a caller-chosen limit; used to exercise the timeout path.
__device__ __noinline__ bool mbar_wait_limit(uint32_t bar, uint32_t parity,
                                             unsigned long long limit_ns) {
  const unsigned long long t0 = gtimer();
  while (!mbar_try(bar, parity)) {
    __nanosleep(1000);
    if (gtimer() - t0 > limit_ns) {
      atomicExch(&g_sg_error, 1u);
      return false;
    }
  }
  return true;
}

// One thread waits on an mbarrier that nothing arrives on until the limit runs out.
__global__ void wait_timeout_kernel(unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait_limit(smem_u32(&bar), 0u, limit_ns);
  }
}

// Operand tiles are re-read by many CTAs: keep them in L2 ahead of the streamed outputs.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y,
                                            uint32_t bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(tmap), "r"(x), "r"(y), "r"(bar), "l"(pol)
      : "memory");
}

// Pair (2-CTA) forms. A TMA load whose completion is signalled on the mbarrier of the leader CTA
// of the pair (shared::cluster address from mapa).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const void* tmap, int x, int y,
                                                 uint32_t cluster_bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(tmap), "r"(x), "r"(y), "r"(cluster_bar), "l"(pol)
      : "memory");
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
// Arrive on a barrier of the leader CTA without release semantics: used to hand an accumulator
// back, where the only ordering needed is that of the TMEM reads, which tcgen05.wait::ld has
// already completed; a release arrive would also wait for the warp's global stores.
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar)
               : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the canonical 128-byte-swizzle layout
// (8-row x 128-byte atoms, 1024 bytes apart along M/N).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

template <int ESIZE>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
  if (ESIZE == 1) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  }
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
template <int ESIZE>
__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  if (ESIZE == 1) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  }
}
// Block-scaled FP4 pair MMA (kind::mxf4, one UE8M0 scale per 32 elements along K): packed e2m1
// operands, K = 64 per instruction (32 bytes of each operand row); the scale factors are read
// from TMEM at sfa / sfb.
__device__ __forceinline__ void umma_pair_mx(uint32_t d_tmem, uint64_t a, uint64_t b,
                                             uint32_t idesc, uint32_t sfa, uint32_t sfb,
                                             uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5],"
      " p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate));
}
// Arrives on the mbarrier at this shared-memory offset in both CTAs of the pair once the pair's
// earlier MMAs have completed.
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar), "h"((unsigned short)3)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Writes the same 32-bit word into 16 consecutive columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_fill16(uint32_t taddr, uint32_t w) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
      "%1,%1};" ::"r"(taddr), "r"(w)
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------------------------
// Contraction kernel
// ---------------------------------------------------------------------------------------------
// ktau_tau32_fast for |S| < 2^24, where S is exact in FP32 (the split's low part is zero): the
// same float-float product and the same rounding test, without the split. sh is S as FP32 (the
// accumulator's exact sum).
__device__ __forceinline__ bool tau32_fast_small(float sh, float rhi, float rlo, float2 fv,
                                                 float& out) {
  const float th = __fmul_rn(sh, rhi);
  const float tl = __fadd_rn(__fmaf_rn(sh, rhi, -th), __fmul_rn(sh, rlo));
  const float ph = __fmul_rn(th, fv.x);
  const float pl = __fadd_rn(__fmaf_rn(th, fv.x, -ph), __fmaf_rn(th, fv.y, __fmul_rn(tl, fv.x)));
  const float d = __fmul_rn(fabsf(ph), 0x1p-40f);
  const float lo = __fadd_rn(ph, __fsub_rn(pl, d));
  const float hi = __fadd_rn(ph, __fadd_rn(pl, d));
  out = lo;
  return lo == hi;
}

// Register j of a 32-register tcgen05.ld result, for a loop index the compiler cannot unroll
// (a select chain keeps the array in registers).
__device__ __forceinline__ uint32_t reg_at(const uint32_t (&r)[32], int j) {
  uint32_t x = r[0];
#pragma unroll
  for (int i = 1; i < 32; ++i) x = j == i ? r[i] : x;
  return x;
}

// Row data of the 32 rows of an epilogue chunk: read from shared memory (written before the
// accumulator wait), or held by lane j for row j and broadcast with shuffles (all 32 lanes must
// call it together).
struct RowsSmem {
  const RowInfo* rc;
  __device__ __forceinline__ RowInfo operator()(int j) const { return rc[j]; }
};
struct RowsReg {
  float rhi, rlo;
  long long base;
  __device__ __forceinline__ RowInfo operator()(int j) const {
    RowInfo R;
    R.rhi = __shfl_sync(0xffffffffu, rhi, j);
    R.rlo = __shfl_sync(0xffffffffu, rlo, j);
    R.base = __shfl_sync(0xffffffffu, base, j);
    return R;
  }
};

// Interior 32 x 32 block of the epilogue (all pairs valid, 32-bit counts, FP32 tau only): row j
// of the block is register j; lane = column, so each store is contiguous across the warp. Rows
// whose FP32 rounding is undecided by the float-float test are flagged in `slow`. The rows go in
// nh <= 2 passes of 16 through one loop body (the second pass selects registers 16..31), so the
// hot code is one 16-row body per output set; TA (tau-a) is a template choice for the same
// reason.
template <bool WS, bool WN, bool TA, class Rows>
__device__ __forceinline__ void epi_rows32(const uint32_t (&sv)[32], const Rows& rows,
                                           float2 c_rff, float* o32, int* oS, int* oN,
                                           uint32_t& slow, float n0f, int nh) {
#pragma unroll 1
  for (int h = 0; h < nh; ++h) {
    uint32_t s16 = 0;  // this pass's undecided rows (bit j: row 16 h + j)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const RowInfo R = rows(16 * h + j);
      const float sh = __uint_as_float(h ? sv[16 + j] : sv[j]);  // the exact integer sum
      float tv;
      if (TA)  // tau-a: S / n_0, one IEEE division of exact FP32 integers (n_0 < 2^24)
        tv = __fdiv_rn(sh, n0f);
      else if (!tau32_fast_small(sh, R.rhi, R.rlo, c_rff, tv))
        s16 |= 1u << j;
      __stcs(o32 + R.base, tv);
      if (WS) __stcs(oS + R.base, __float2int_rn(sh));
      if (WN) __stcs(oN + R.base, 0);
    }
    slow |= s16 << (16 * h);
  }
}

struct SideArgs {  // per-variable data of the row side (u) or the column side (v)
  const uint16_t* rank;
  const uint16_t* perm;
  const uint16_t* srank;
  int64_t ld;
  const int64_t* T;
  const double* rs64;
  const float2* rsff;
  const int64_t* tie_off;     // [m + 1] prefix of T
  const uint32_t* tie_pairs;  // listed tied pairs, (a << 16) | b
  int64_t tie_cap;            // a variable is listed iff tie_off[v] + T[v] <= tie_cap
  int64_t m;
};

struct ContractArgs {
  SideArgs row, col;
  int64_t n, num_kb;
  int tri;                 // 1: upper triangle of one matrix; 0: rectangle rows x cols
  int st;                  // tri: super-tile side (256, or MXT for block-scaled FP4)
  int64_t wS;              // tri: super-tiles per side
  int64_t wG;              // tri: traversal groups per side
  int64_t ncb;             // rect: column blocks of BM
  int bnr;                 // output rows per unit: 256, or 128 / 64 for short query batches
  int afmt;                // kind::f8f6f4 operand format: 0 = E4M3, 5 = E2M1 (FP4), or kMxFmt:
                           // packed E2M1 through kind::mxf4 (pair kernel only)
  // Permutation test (exceed != nullptr): count |S| >= |s_obs[k]| into exceed[k] instead of
  // storing tau / S / n_3 (triangle, single matrix only).
  const int32_t* s_obs;
  uint32_t* exceed;
  int64_t unit_lo, unit_hi;
  uint64_t p_begin, p_end; // tri: pair range
  int64_t ldo;             // rect: output row stride
  ktau_out out;
  // Batched form (bds != nullptr): units of several datasets stacked in one operand tensor.
  const ktau_bds* bds;
  const int32_t* bids;     // datasets of this launch, in unit order
  int nb;
  const int64_t* unit_prefix;  // [nb + 1]
  // Magnitude contraction (single matrix): the accumulator is |A_u| . |A_v| and the epilogue
  // stores only n_3 = |A_u| . |A_v| - n_0 + T_u + T_v.
  int absmode;
};

// The problem a unit belongs to (the whole launch, or one dataset of a batch).
struct Prob {
  SideArgs row, col;
  int64_t n, num_kb;
  int tri;
  uint64_t p_begin, p_end;
  int64_t ldo;
  ktau_out out;
  const int32_t* s_obs;
  uint32_t* exceed;
};

struct Unit {
  int64_t y0, x0;   // unit origin in the problem's own rows (up to 256) / columns (128)
  int64_t yend;     // first row past the unit (the super-tile's or the matrix's end)
  int64_t xend;     // first column past the unit's super-tile (columns beyond it repeat the next
                    // super-tile's outputs: stored twice with equal values, counted once)
  bool live;
  int ta, tb;       // TMA row coordinates of the A (column variables) and B (row variables) tiles
  int64_t num_kb;
  int bd;           // dataset of a batched launch (-1 otherwise)
};

__device__ __forceinline__ SideArgs side_of_bds(const ktau_bds& D) {
  return SideArgs{D.rank, D.perm, D.srank, D.ld, D.T, D.rs64, D.rsff,
                  D.tie_off, D.tie_pairs, D.tie_cap, D.m};
}

__device__ __forceinline__ Prob problem_of(const ContractArgs& a, const Unit& t) {
  Prob p;
  if (t.bd < 0) {
    p.row = a.row;
    p.col = a.col;
    p.n = a.n;
    p.num_kb = a.num_kb;
    p.tri = a.tri;
    p.p_begin = a.p_begin;
    p.p_end = a.p_end;
    p.ldo = a.ldo;
    p.out = a.out;
    p.s_obs = a.s_obs;
    p.exceed = a.exceed;
  } else {
    const ktau_bds& D = a.bds[t.bd];
    p.row = p.col = side_of_bds(D);
    p.n = D.n;
    p.num_kb = D.num_kb;
    p.tri = 1;
    p.p_begin = 0;
    p.p_end = (uint64_t)(D.m * (D.m - 1) / 2);
    p.ldo = 0;
    p.out = D.out;
    p.out.n3 = nullptr;
    p.s_obs = nullptr;
    p.exceed = nullptr;
  }
  return p;
}

__device__ __forceinline__ uint64_t tri_p(int64_t m, int64_t y, int64_t x) {
  return (uint64_t)(y * (2 * m - y - 1) / 2 + (x - y - 1));
}

// Tile origin of a work unit and whether it holds any output (same answer in every role).
__device__ __forceinline__ Unit unit_of(const ContractArgs& a, int64_t u) {
  Unit r;
  r.bd = -1;
  r.num_kb = a.num_kb;
  if (a.bds) {
    int lo = 0, hi = a.nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.unit_prefix[mid] <= u)
        lo = mid;
      else
        hi = mid - 1;
    }
    r.bd = a.bids[lo];
    const ktau_bds& D = a.bds[r.bd];
    const int64_t lu = u - a.unit_prefix[lo];
    int64_t ys, xs;
    ktau_tile_coord(D.wS, lu >> 1, ys, xs);
    r.y0 = ys * a.st;
    r.x0 = xs * a.st + (lu & 1) * BM;
    r.yend = min(r.y0 + (int64_t)a.st, D.m);
    r.xend = min((xs + 1) * (int64_t)a.st, D.m);
    const int64_t xend = min(r.x0 + (int64_t)BM, D.m);
    r.live = r.y0 < D.m && r.x0 < D.m && xend - 1 > r.y0;
    r.ta = (int)(D.srow + r.x0);
    r.tb = (int)(D.srow + r.y0);
    r.num_kb = D.num_kb;
    return r;
  }
  if (a.tri) {
    // Slot u -> (group of GROUP x GROUP super-tiles, walked by the bijection on the group matrix;
    // row-major inside the group) -> 256 x 256 super-tile -> 128-column half. Consecutive slots,
    // which run at the same time on neighbouring CTAs, stay inside one group and share operand
    // blocks in L2. Slots below the diagonal or past the edge are dead.
    const int64_t s2 = u >> 1;
    const int64_t gid = s2 / (GROUP * GROUP), loc = s2 % (GROUP * GROUP);
    int64_t gy, gx;
    ktau_tile_coord(a.wG, gid, gy, gx);
    const int64_t ys = gy * GROUP + loc / GROUP, xs = gx * GROUP + loc % GROUP;
    r.y0 = ys * a.st;
    r.x0 = xs * a.st + (u & 1) * BM;
    r.ta = (int)r.x0;
    r.tb = (int)r.y0;
    r.yend = min(r.y0 + (int64_t)a.st, a.row.m);
    r.xend = min((xs + 1) * (int64_t)a.st, a.row.m);
    if (ys >= a.wS || xs >= a.wS || ys > xs) {
      r.live = false;
      return r;
    }
    const int64_t m = a.row.m;
    const int64_t xend = min(r.x0 + (int64_t)BM, m);
    const int64_t ylast = min(r.yend - 1, xend - 2);
    r.live = r.y0 < m && r.x0 < m && ylast >= r.y0;
    if (r.live) {
      const uint64_t pmin = tri_p(m, r.y0, max(r.x0, r.y0 + 1));
      const uint64_t pmax = tri_p(m, ylast, xend - 1);
      r.live = pmax >= a.p_begin && pmin < a.p_end;
    }
  } else {
    r.y0 = (u / a.ncb) * a.bnr;
    r.x0 = (u % a.ncb) * BM;
    r.ta = (int)r.x0;
    r.tb = (int)r.y0;
    r.yend = min(r.y0 + (int64_t)a.bnr, a.row.m);
    r.xend = min(r.x0 + (int64_t)BM, a.col.m);
    r.live = r.y0 < a.row.m && r.x0 < a.col.m;
  }
  return r;
}

constexpr int JT = 256;      // tile side (rows and columns) walked through the bijection
constexpr int JCAP = 8192;   // tied sample pairs of one tile's rows listed in shared memory

// Tied sample pairs of variable y (sorted order: tie groups are runs of equal srank), written
// to out[0 .. T_y) by one warp. Position k of a group starting at g0 pairs with g0 .. k-1.
__device__ void warp_list_ties(const uint16_t* __restrict__ perm, const uint16_t* __restrict__ srank,
                               int n, uint32_t* out, int lane, int32_t* bkt_cnt = nullptr) {
  int run = 0;
  for (int base = 0; base < n; base += 32) {
    const int k = base + lane;
    int cnt = 0, g0 = 0;
    if (k > 0 && k < n && srank[k] == srank[k - 1]) {
      const uint16_t key = srank[k];
      int lo = 0, hi = k;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (srank[mid] < key)
          lo = mid + 1;
        else
          hi = mid;
      }
      g0 = lo;
      cnt = k - g0;
    }
    int incl = cnt;
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    const int off = run + incl - cnt;
    if (cnt) {
      const uint32_t b = perm[k];
      for (int j = 0; j < cnt; ++j) {
        uint32_t a = perm[g0 + j], bb = b;
        if (a > bb) {
          const uint32_t t = a;
          a = bb;
          bb = t;
        }
        out[off + j] = (a << 16) | bb;
        if (bkt_cnt)  // bucket of sample pair (a, b): its index in the Eq. 4 order
          atomicAdd(bkt_cnt + (int)(a * (2u * n - a - 1) / 2 + (bb - a - 1)), 1);
      }
    }
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
}

// Exclusive prefix of the tie counts T over m variables (one CTA): off[i] = sum_{r<i} T[r].
// Tiles of 4 * blockDim values: each thread loads four consecutive values (coalesced across the
// CTA), the CTA scans the thread sums, and a running carry links the tiles.
// A variable's list is stored only when it ends within `cap` entries; the others are walked
// from their tie groups directly by the joint-ties kernel (same test on both sides).
__global__ void __launch_bounds__(1024) ties_scan_kernel(const int64_t* __restrict__ T, int64_t m,
                                                         int64_t* __restrict__ off) {
  __shared__ long long wsum[32];
  __shared__ long long carry_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  long long carry = 0;
  for (int64_t base = 0; base < m; base += 4 * (int64_t)blockDim.x) {
    const int64_t i0 = base + 4 * (int64_t)tid;
    long long v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = i0 + e < m ? (long long)T[i0 + e] : 0ll;
    const long long local = v[0] + v[1] + v[2] + v[3];
    long long incl = local;
    for (int d = 1; d < 32; d <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      long long w = lane < nw ? wsum[lane] : 0ll;
      for (int d = 1; d < 32; d <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += t;
      }
      if (lane < nw) wsum[lane] = w;  // inclusive prefix over warps
    }
    __syncthreads();
    long long run = carry + incl - local + (warp > 0 ? wsum[warp - 1] : 0ll);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (i0 + e < m) off[i0 + e] = run;
      run += v[e];
    }
    if (tid == blockDim.x - 1) carry_s = run;
    __syncthreads();
    carry = carry_s;
    __syncthreads();
  }
  if (tid == 0) off[m] = carry;
}

__global__ void ties_list_kernel(const uint16_t* __restrict__ perm, const uint16_t* __restrict__ srank,
                                 const int64_t* __restrict__ T, const int64_t* __restrict__ off,
                                 int64_t ld, int n, int64_t m, int64_t cap,
                                 uint32_t* __restrict__ pairs, int32_t* __restrict__ bkt_cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (row >= m) return;
  if (T[row] == 0 || off[row] + T[row] > cap) return;
  warp_list_ties(perm + row * ld, srank + row * ld, n, pairs + off[row], lane, bkt_cnt);
}

// Inclusive prefix of the bucket sizes in place (one CTA), c[K] = total; also the work of the
// bucket form of n_3 (sum and largest s(s-1)/2) and the flag that selects it. Tiles of
// 4 * blockDim values as in ties_scan_kernel.
// At most 256 threads: the per-warp arrays stay small enough (200 bytes) for a CTA of this kernel
// to fit on an SM beside a CTA of the pair contraction, whose shared memory leaves 1.8 KB free.
__global__ void __launch_bounds__(256) bucket_scan_kernel(int32_t* __restrict__ c, int64_t K,
                                                          unsigned long long* __restrict__ stat,
                                                          unsigned long long lim_total,
                                                          unsigned long long lim_one) {
  __shared__ long long wsum[8];
  __shared__ unsigned long long wwork[8], wmax[8];
  __shared__ long long carry_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  long long carry = 0;
  unsigned long long work = 0, big = 0;
  for (int64_t base = 0; base < K; base += 4 * (int64_t)blockDim.x) {
    const int64_t i0 = base + 4 * (int64_t)tid;
    long long v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      v[e] = i0 + e < K ? (long long)c[i0 + e] : 0ll;
      const unsigned long long wv = (unsigned long long)(v[e] * (v[e] - 1) / 2);
      work += wv;
      big = wv > big ? wv : big;
    }
    const long long local = v[0] + v[1] + v[2] + v[3];
    long long incl = local;
    for (int d = 1; d < 32; d <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      long long w = lane < nw ? wsum[lane] : 0ll;
      for (int d = 1; d < 32; d <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += t;
      }
      if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    long long run = carry + incl - local + (warp > 0 ? wsum[warp - 1] : 0ll);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      run += v[e];
      if (i0 + e < K) c[i0 + e] = (int32_t)run;
    }
    if (tid == blockDim.x - 1) carry_s = run;
    __syncthreads();
    carry = carry_s;
    __syncthreads();
  }
  for (int d = 16; d > 0; d >>= 1) {
    work += __shfl_xor_sync(0xffffffffu, work, d);
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, big, d);
    big = o > big ? o : big;
  }
  if (lane == 0) {
    wwork[warp] = work;
    wmax[warp] = big;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long W = 0, M = 0;
    for (int w = 0; w < nw; ++w) {
      W += wwork[w];
      M = wmax[w] > M ? wmax[w] : M;
    }
    c[K] = (int32_t)carry;
    stat[0] = W;
    stat[1] = M;
    stat[2] = (W <= lim_total && M <= lim_one) ? 1ull : 0ull;
  }
}

// Scatter: bucket ends (inclusive prefix) count down to bucket starts while the variables are
// placed, so bkt_off ends as the exclusive prefix.
__global__ void bucket_scatter_kernel(const uint32_t* __restrict__ pairs,
                                      const int64_t* __restrict__ T, const int64_t* __restrict__ off,
                                      int n, int64_t m, int64_t cap, int32_t* __restrict__ bkt_off,
                                      int32_t* __restrict__ bkt_var) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (row >= m) return;
  if (T[row] == 0 || off[row] + T[row] > cap) return;
  for (int64_t e = off[row] + lane; e < off[row] + T[row]; e += 32) {
    const uint32_t ab = pairs[e];
    const uint32_t a = ab >> 16, bb = ab & 0xffffu;
    const int key = (int)(a * (2u * n - a - 1) / 2 + (bb - a - 1));
    const int pos = atomicSub(bkt_off + key, 1) - 1;
    bkt_var[pos] = (int32_t)row;
  }
}

// n_3 from the buckets: every two variables of a bucket share that tied sample pair, so n_3(u, v)
// is the number of buckets holding both (Table 1: joint ties). The output was zeroed beforehand.
// A lane takes a bucket of up to 32 variables alone; larger buckets are shared by the warp.
__device__ __forceinline__ void n3_add(void* n3out, int count_bits, uint64_t k) {
  if (count_bits == 64)
    atomicAdd((unsigned long long*)n3out + k, 1ull);
  else
    atomicAdd((int*)n3out + k, 1);
}

__global__ void __launch_bounds__(256) bucket_n3_kernel(const int32_t* __restrict__ bkt_off,
                                                        const int32_t* __restrict__ bkt_var,
                                                        const unsigned long long* __restrict__ stat,
                                                        int64_t K, int64_t m, uint64_t p_begin,
                                                        uint64_t p_end, void* n3out,
                                                        int count_bits) {
  if (stat[2] == 0) return;  // skewed buckets: the tile kernel counts n_3 instead
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  auto emit = [&](int32_t u, int32_t v) {
    if (u > v) {
      const int32_t t = u;
      u = v;
      v = t;
    }
    const uint64_t p = (uint64_t)((int64_t)u * (2 * m - u - 1) / 2 + (v - u - 1));
    if (p >= p_begin && p < p_end) n3_add(n3out, count_bits, p - p_begin);
  };
  for (int64_t k0 = gw * 32; k0 < K; k0 += warps * 32) {
    const int64_t k = k0 + lane;
    int32_t lo = 0, s = 0;
    if (k < K) {
      lo = bkt_off[k];
      s = bkt_off[k + 1] - lo;
    }
    if (s >= 2 && s <= 32)
      for (int i = 0; i + 1 < s; ++i) {
        const int32_t u = bkt_var[lo + i];
        for (int j = i + 1; j < s; ++j) emit(u, bkt_var[lo + j]);
      }
    unsigned big = __ballot_sync(0xffffffffu, s > 32);
    while (big) {
      const int src = __ffs(big) - 1;
      big &= big - 1;
      const int32_t blo = __shfl_sync(0xffffffffu, lo, src);
      const int32_t bs = __shfl_sync(0xffffffffu, s, src);
      for (int i = 0; i + 1 < bs; ++i) {
        const int32_t u = bkt_var[blo + i];
        for (int j = i + 1 + lane; j < bs; j += 32) emit(u, bkt_var[blo + j]);
      }
    }
  }
}

// Batched listing: rows of a group (T, tie_off contiguous over the group's rows).
__global__ void batch_ties_list_kernel(const ktau_bds* __restrict__ ds,
                                       const int32_t* __restrict__ bids, int nb,
                                       const int64_t* __restrict__ row_prefix, int64_t rows,
                                       const int64_t* __restrict__ T, const int64_t* __restrict__ off,
                                       int64_t cap, uint32_t* __restrict__ pairs) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  if (T[r] == 0 || off[r] + T[r] > cap) return;
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row_prefix[mid] <= r)
      lo = mid;
    else
      hi = mid - 1;
  }
  const ktau_bds& D = ds[bids[lo]];
  const int64_t row = r - row_prefix[lo];
  warp_list_ties(D.perm + row * D.ld, D.srank + row * D.ld, (int)D.n, pairs + off[r], lane);
}

// n_3(u, v) = number of sample pairs tied in u that are also tied in v (Table 1). Square JT x JT
// tiles of the job matrix (bijection, Eq. 13-14); the tied pairs of the tile's row variables are
// listed in shared memory, and the column variables' ranks are staged transposed (rT[a][j]) 64
// at a time so that, for each tied pair (a, b), the 32 lanes of a warp check 32 column variables
// with conflict-free loads. Writes every n_3 of the range (zeros included).
// SPARSE: the output was zeroed beforehand; only rows with ties are visited and only nonzero
// counts are stored. Otherwise every n_3 of the tile is stored.
template <int JCOLS, bool SPARSE>
__device__ void joint_ties_tile(const SideArgs& R, const SideArgs& C, int64_t n, int tri,
                                int64_t y0, int64_t x0, uint64_t p_begin, uint64_t p_end,
                                int64_t ldo, void* n3out, int count_bits) {
  extern __shared__ uint32_t jsm[];
  uint32_t* s_pairs = jsm;                                     // [JCAP]
  int* s_off = (int*)(jsm + JCAP);                             // [JT + 1], tile-relative offsets
  constexpr int JTPC = JCOLS + 1;  // padded row (uint16) of the transposed rank block
  constexpr int H = JCOLS / 32;     // columns per lane
  uint16_t* rT = (uint16_t*)(jsm + JCAP + JT + 8);             // [n][JTPC]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  {
    const int rows = (int)min((int64_t)JT, R.m - y0);
    __syncthreads();
    // The tile rows' lists are one contiguous segment of the global list (when all are listed).
    const int64_t base_off = R.tie_off[y0];
    const int64_t seg = R.tie_off[y0 + rows] - base_off;
    const bool listed = R.tie_off[y0 + rows] <= R.tie_cap && seg <= JCAP;
    if (SPARSE && seg == 0) return;  // no row of this tile has ties: every n_3 is 0
    for (int i = threadIdx.x; i <= rows; i += blockDim.x)
      s_off[i] = (int)min(R.tie_off[y0 + i] - base_off, (int64_t)JCAP);
    if (listed)
      for (int64_t i = threadIdx.x; i < seg; i += blockDim.x) s_pairs[i] = R.tie_pairs[base_off + i];
    for (int cs = 0; cs < JT / JCOLS; ++cs) {
      const int64_t xs = x0 + cs * JCOLS;
      if (xs >= C.m) break;
      if (tri && xs + JCOLS - 1 <= y0) continue;  // sub-block entirely on or below the diagonal
      __syncthreads();
      // Stage the JCOLS column variables' rank rows transposed, 8 ranks (16 bytes) per load.
      const int vec = (int)(C.ld >> 3);
      for (int e = threadIdx.x; e < JCOLS * vec; e += blockDim.x) {
        const int j = e / vec, c8 = e - j * vec;
        const int64_t v = xs + j;
        uint4 w4 = make_uint4(0u, 0u, 0u, 0u);
        if (v < C.m) w4 = __ldg(reinterpret_cast<const uint4*>(C.rank + v * C.ld) + c8);
        const uint32_t wd[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int h = 0; h < 8; ++h) {
          const int aa = c8 * 8 + h;
          if (aa < n) rT[aa * JTPC + j] = (uint16_t)(wd[h >> 1] >> (16 * (h & 1)));
        }
      }
      __syncthreads();
      const int rows_here = tri ? (int)min((int64_t)rows, xs + JCOLS - 1 - y0) : rows;
      for (int i = warp; i < rows_here; i += nwarps) {
        const int64_t y = y0 + i;
        if (SPARSE && (listed ? s_off[i + 1] == s_off[i] : R.T[y] == 0)) continue;
        int c0 = 0, c1 = 0;
        if (listed) {
          for (int e = s_off[i]; e < s_off[i + 1]; ++e) {
            const uint32_t ab = s_pairs[e];
            const int a = (int)(ab >> 16), b = (int)(ab & 0xffffu);
            c0 += rT[a * JTPC + lane] == rT[b * JTPC + lane];
            if (H == 2) c1 += rT[a * JTPC + lane + 32] == rT[b * JTPC + lane + 32];
          }
        } else if (R.T[y] > 0 && R.tie_off[y] + R.T[y] <= R.tie_cap) {
          const uint32_t* tp = R.tie_pairs + R.tie_off[y];
          for (long long e = 0; e < R.T[y]; ++e) {
            const uint32_t ab = tp[e];
            const int a = (int)(ab >> 16), b = (int)(ab & 0xffffu);
            c0 += rT[a * JTPC + lane] == rT[b * JTPC + lane];
            if (H == 2) c1 += rT[a * JTPC + lane + 32] == rT[b * JTPC + lane + 32];
          }
        } else if (R.T[y] > 0) {
          // Not listed (capacity): walk the tie groups of y in its sorted order directly.
          const uint16_t* pp = R.perm + y * R.ld;
          const uint16_t* ss = R.srank + y * R.ld;
          int g0 = 0;
          for (int k = 1; k < n; ++k) {
            if (ss[k] != ss[k - 1]) {
              g0 = k;
              continue;
            }
            const int b = pp[k];
            for (int j = g0; j < k; ++j) {
              const int a = pp[j];
              c0 += rT[a * JTPC + lane] == rT[b * JTPC + lane];
              if (H == 2) c1 += rT[a * JTPC + lane + 32] == rT[b * JTPC + lane + 32];
            }
          }
        }
        if (SPARSE && c0 == 0 && c1 == 0) continue;  // nothing to store (output zeroed)
        const int64_t rowbase = tri ? y * (2 * R.m - y - 1) / 2 - y - 1 : y * ldo;
#pragma unroll
        for (int h = 0; h < H; ++h) {
          const int64_t v = xs + lane + 32 * h;
          if (v >= C.m) continue;
          uint64_t k;
          if (tri) {
            if (v <= y) continue;
            const uint64_t p = (uint64_t)(rowbase + v);
            if (p < p_begin || p >= p_end) continue;
            k = p - p_begin;
          } else {
            k = (uint64_t)(rowbase + v);
          }
          const int val = h ? c1 : c0;
          if (SPARSE && val == 0) continue;
          if (count_bits == 64)
            __stcs((long long*)n3out + k, (long long)val);
          else
            __stcs((int*)n3out + k, val);
        }
      }
    }
  }
}

template <int JCOLS>
__global__ void __launch_bounds__(256) joint_ties_kernel(const SideArgs R, const SideArgs C,
                                                         int64_t n, int tri, int64_t w,
                                                         int64_t ncb, int64_t tile_lo,
                                                         int64_t tile_hi, uint64_t p_begin,
                                                         uint64_t p_end, int64_t ldo, void* n3out,
                                                         int count_bits,
                                                         const unsigned long long* bkt_stat) {
  if (bkt_stat && bkt_stat[2]) return;  // the bucket kernel counts n_3
  for (int64_t t = tile_lo + blockIdx.x; t < tile_hi; t += gridDim.x) {
    int64_t y0, x0;
    if (tri) {
      int64_t yq, xq;
      ktau_tile_coord(w, t, yq, xq);
      y0 = yq * JT;
      x0 = xq * JT;
    } else {
      y0 = (t / ncb) * JT;
      x0 = (t % ncb) * JT;
    }
    joint_ties_tile<JCOLS, true>(R, C, n, tri, y0, x0, p_begin, p_end, ldo, n3out, count_bits);
  }
}

// Batched: the JT x JT tiles of every dataset of a group in one list (prefix over bids).
template <int JCOLS>
__global__ void __launch_bounds__(256) batch_joint_ties_kernel(
    const ktau_bds* __restrict__ ds, const int32_t* __restrict__ bids, int nb,
    const int64_t* __restrict__ tile_prefix, int64_t total_tiles) {
  for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_prefix[mid] <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    const ktau_bds& D = ds[bids[lo]];
    if (!D.out.n3) continue;
    const int64_t w = (D.m + JT - 1) / JT;
    int64_t yq, xq;
    ktau_tile_coord(w, t - tile_prefix[lo], yq, xq);
    const SideArgs S = side_of_bds(D);
    joint_ties_tile<JCOLS, false>(S, S, D.n, 1, yq * JT, xq * JT, 0,
                                  (uint64_t)(D.m * (D.m - 1) / 2), 0, D.out.n3, D.out.count_bits);
  }
}

// Epilogue of one unit by one epilogue warp (warps 2..9): warp w owns TMEM lane quarter
// q = w & 3 (32 output columns v, one per lane) and one half of the unit's rows, 32 rows per
// tcgen05.ld (register j = row u0 + j). With kSmemRows the half's row data are fetched into
// shared memory before the accumulator is waited for; otherwise each chunk's rows are held one
// per lane and broadcast. Returns false when a bounded wait gave up.
__device__ __forceinline__ RowInfo row_info(const Prob& P, int64_t y) {
  RowInfo info;
  const float2 f = y < P.row.m ? __ldg(P.row.rsff + y) : make_float2(0.f, 0.f);
  info.rhi = f.x;
  info.rlo = f.y;
  info.base = P.tri ? (long long)(y * (2 * P.row.m - y - 1) / 2 - y - 1) : (long long)y * P.ldo;
  return info;
}

// The per-unit constants of one epilogue warp.
struct EpiCtx {
  Prob P;
  int64_t mrow, mcol, vbase, v, n0;
  int64_t yend;  // rows at or past yend are not this unit's
  bool vown;     // this lane's column belongs to the unit's super-tile (counted once)
  bool vin, want64, want32, s64, cols_full;
  float2 c_rff;
  void* n3z;  // n_3 output given: store its zeros here; the joint-ties kernels add the rest
};

__device__ __forceinline__ EpiCtx epi_ctx(const ContractArgs& a, const Unit& t, int q, int lane) {
  EpiCtx e;
  e.P = problem_of(a, t);
  e.mrow = e.P.row.m;
  e.mcol = e.P.col.m;
  e.yend = t.yend;
  e.vown = t.x0 + 32 * q + lane < t.xend;
  e.vbase = t.x0 + 32 * q;
  e.v = e.vbase + lane;
  e.vin = e.v < e.mcol;
  e.c_rff = e.vin ? __ldg(e.P.col.rsff + e.v) : make_float2(0.f, 0.f);
  e.n0 = e.P.n * (e.P.n - 1) / 2;
  e.want64 = e.P.out.tau64 != nullptr;
  e.want32 = e.P.out.tau32 != nullptr;
  e.s64 = e.P.out.count_bits == 64;
  e.n3z = e.P.out.n3;
  e.cols_full = e.vbase + 32 <= e.mcol;
  return e;
}

// Outputs of one 32-row chunk (rows ub .. ub + 31, register j = row ub + j) of one epilogue
// warp's 32 columns, from the integer counts r.
template <bool kSmemRows, bool ABS = false>
__device__ __forceinline__ void epi_chunk(const EpiCtx& E, const RowInfo* rc, const RowInfo& mine,
                                          int64_t ub, const uint32_t (&r)[32]) {
  const Prob& P = E.P;
  const int64_t mrow = E.mrow, v = E.v, vbase = E.vbase, n0 = E.n0;
  const bool vin = E.vin;
  const float2 c_rff = E.c_rff;
  const RowsSmem rs{rc};
  const RowsReg rr{mine.rhi, mine.rlo, mine.base};
  const int rows_here = (int)min((int64_t)32, E.yend - ub);
  if (P.exceed) {  // permutation test: one exceedance count per pair, no other output
    // Groups of 8 rows: first every observed S of the group (independent loads), then the
    // comparisons and fire-and-forget atomic increments (each pair has one thread per launch).
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      int so[8];
      uint64_t kk[8];
      uint32_t valid = 0;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int j = 8 * h + jj;
        const RowInfo R = kSmemRows ? rs(j) : rr(j);  // whole warp (shuffle form)
        const int64_t y = ub + j;
        const uint64_t p = (uint64_t)(R.base + v);
        kk[jj] = P.tri ? p - P.p_begin : p;
        so[jj] = 0;
        if (j < rows_here && vin && E.vown &&
            (!P.tri || (v > y && p >= P.p_begin && p < P.p_end))) {
          valid |= 1u << jj;
          so[jj] = __ldg(P.s_obs + kk[jj]);
        }
      }
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int S = __float2int_rn(__uint_as_float(r[8 * h + jj]));
        if (((valid >> jj) & 1u) && abs(S) >= abs(so[jj])) atomicAdd(P.exceed + kk[jj], 1u);
      }
    }
    return;
  }
  if (ABS) {
    // n_3 from the magnitude contraction: pairs tied in neither variable number
    // |A_u| . |A_v| = n_0 - T_u - T_v + n_3 (Table 1), an exact integer below 2^24.
    const long long Tv = vin ? P.col.T[v] : 0;
#pragma unroll 1
    for (int j = 0; j < rows_here; ++j) {
      const RowInfo R = kSmemRows ? rs(j) : rr(j);  // whole warp (shuffle form)
      const int64_t y = ub + j;
      const long long Tu = P.row.T[y];
      if (!vin) continue;
      uint64_t k;
      if (P.tri) {
        if (v <= y) continue;
        const uint64_t p = (uint64_t)(R.base + v);
        if (p < P.p_begin || p >= P.p_end) continue;
        k = p - P.p_begin;
      } else {
        k = (uint64_t)(R.base + v);
      }
      const long long n3 =
          (long long)__float2int_rn(__uint_as_float(reg_at(r, j))) - n0 + Tu + Tv;
      if (E.s64)
        __stcs((long long*)P.out.n3 + k, n3);
      else
        __stcs((int*)P.out.n3 + k, (int)n3);
    }
    return;
  }
  // Interior blocks of 32 rows, or of 16 (the last chunk of a 240-row super-tile)
  bool fast = (rows_here == 32 || rows_here == 16) && E.cols_full &&
              (!P.tri || vbase > ub + rows_here - 1);
  if (fast && P.tri) {  // every pair of these rows inside the pair range
    const int64_t ul = ub + rows_here - 1;
    fast = (uint64_t)(ub * (2 * mrow - ub - 1) / 2) >= P.p_begin &&
           (uint64_t)(ul * (2 * mrow - ul - 1) / 2 + (mrow - ul - 1)) <= P.p_end;
  }
  if (fast && E.want32 && !E.want64 && !E.s64) {
    float* const o32 = P.out.tau32 + (v - (int64_t)P.p_begin);
    int* const oS = P.out.S ? (int*)P.out.S + (v - (int64_t)P.p_begin) : nullptr;
    int* const oN = E.n3z ? (int*)E.n3z + (v - (int64_t)P.p_begin) : nullptr;
    uint32_t slow = 0;  // rows whose FP32 rounding the float-float test could not decide
    const float n0f = P.out.stat ? (float)n0 : 0.f;
#define KTAU_EPI_ROWS_T(ROWS, TA)                                                \
  if (oS && oN)                                                                  \
    epi_rows32<true, true, TA>(r, ROWS, c_rff, o32, oS, oN, slow, n0f, nh);      \
  else if (oS)                                                                   \
    epi_rows32<true, false, TA>(r, ROWS, c_rff, o32, oS, oN, slow, n0f, nh);     \
  else if (oN)                                                                   \
    epi_rows32<false, true, TA>(r, ROWS, c_rff, o32, oS, oN, slow, n0f, nh);     \
  else                                                                           \
    epi_rows32<false, false, TA>(r, ROWS, c_rff, o32, oS, oN, slow, n0f, nh);
#define KTAU_EPI_ROWS(ROWS)        \
  if (n0f != 0.f) {                \
    KTAU_EPI_ROWS_T(ROWS, true)    \
  } else {                         \
    KTAU_EPI_ROWS_T(ROWS, false)   \
  }
    const int nh = rows_here / 16;
    if (kSmemRows) {
      KTAU_EPI_ROWS(rs)
    } else {
      KTAU_EPI_ROWS(rr)
    }
#undef KTAU_EPI_ROWS
#undef KTAU_EPI_ROWS_T
    while (slow) {  // rare: the FP64 formula decides (same thread, stored after the fast value)
      const int j = __ffs(slow) - 1;
      slow &= slow - 1;
      const RowInfo R = row_info(P, ub + j);
      const int S = __float2int_rn(__uint_as_float(reg_at(r, j)));
      o32[R.base] = ktau_tau32(S, make_float2(R.rhi, R.rlo), c_rff, n0, P.row.T[ub + j],
                               P.col.T[v]);
    }
  } else {
    const bool wantS = P.out.S != nullptr;
#pragma unroll 1
    for (int j = 0; j < rows_here; ++j) {
      const RowInfo R = kSmemRows ? rs(j) : rr(j);  // whole warp (shuffle form)
      const int64_t y = ub + j;
      if (!vin) continue;
      uint64_t k;
      if (P.tri) {
        if (v <= y) continue;
        const uint64_t p = (uint64_t)(R.base + v);
        if (p < P.p_begin || p >= P.p_end) continue;
        k = p - P.p_begin;
      } else {
        k = (uint64_t)(R.base + v);
      }
      const int S = __float2int_rn(__uint_as_float(reg_at(r, j)));
      if (E.want64)
        __stcs(P.out.tau64 + k, P.out.stat ? ktau_taua64(S, n0)
                                           : ktau_tau64(S, P.row.rs64[y], P.col.rs64[v]));
      if (E.want32)
        __stcs(P.out.tau32 + k,
               P.out.stat ? ktau_taua32(S, n0)
                          : ktau_tau32(S, make_float2(R.rhi, R.rlo), c_rff, n0, P.row.T[y],
                                       P.col.T[v]));
      if (wantS) {
        if (E.s64)
          __stcs((long long*)P.out.S + k, (long long)S);
        else
          __stcs((int*)P.out.S + k, S);
      }
      if (E.n3z) {
        if (E.s64)
          __stcs((long long*)E.n3z + k, 0ll);
        else
          __stcs((int*)E.n3z + k, 0);
      }
    }
  }
}

// Releases an accumulator once this warp's tcgen05.ld of it have completed: one arrive per warp
// (on the leader CTA's barrier in the pair form).
__device__ __forceinline__ void release_acc(uint32_t tempty_bar, bool remote, int lane) {
  tc_fence_before();
  __syncwarp();
  if (lane == 0) {
    if (remote)
      mbar_arrive_cluster_relaxed(tempty_bar);
    else
      mbar_arrive(tempty_bar);
  }
}

// kSlot (with !kSmemRows): ri is this warp's 32-entry slot; each chunk's row data go there
// (one entry per lane) and are read back by broadcast.
template <bool kSmemRows, bool kSlot = false, int EW = EPI_WARPS, bool ABS = false>
__device__ __forceinline__ bool epilogue_unit(const ContractArgs& a, const Unit& t, RowInfo* ri,
                                              uint32_t tmem_base, uint32_t tfull_bar,
                                              uint32_t tfull_phase, int acc, int warp, int lane,
                                              uint32_t tempty_bar, bool remote) {
  const int q = warp & 3;
  const int half_sel = (warp - 2) >> 2;     // which part of the rows (EW / 4 parts)
  const int nhalf = a.bnr / 32 / (EW / 4);  // 32-row chunks per part
  const EpiCtx E = epi_ctx(a, t, q, lane);
  if (kSmemRows) {
    const int64_t hrow0 = t.y0 + 32 * half_sel * nhalf;
    for (int i = lane; i < 32 * nhalf; i += 32) ri[i] = row_info(E.P, hrow0 + i);
    __syncwarp();
  }
  if (!mbar_wait(tfull_bar, tfull_phase)) return false;
  tc_fence_after();
  RowInfo next;  // this lane's row of the next chunk, loaded one chunk ahead
  if (!kSmemRows) next = row_info(E.P, t.y0 + 32 * half_sel * nhalf + lane);
  for (int c = half_sel * nhalf; c < (half_sel + 1) * nhalf; ++c) {
    const int64_t ub = t.y0 + 32 * c;
    const RowInfo mine = next;
    if (!kSmemRows && c + 1 < (half_sel + 1) * nhalf) next = row_info(E.P, ub + 32 + lane);
    uint32_t r[32];
    tmem_ld32(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * BN + 32 * c), r);
    // the accumulator may be overwritten by the next unit once the last chunk is read
    if (c == (half_sel + 1) * nhalf - 1) release_acc(tempty_bar, remote, lane);
    if (ub >= E.yend) continue;
    if (kSlot) {
      ri[lane] = mine;
      __syncwarp();
      epi_chunk<true, ABS>(E, ri, mine, ub, r);
      __syncwarp();  // the slot is rewritten for the next chunk
    } else {
      epi_chunk<kSmemRows, ABS>(E, ri + 32 * (c - half_sel * nhalf), mine, ub, r);
    }
  }
  if (kSmemRows) __syncwarp();  // ri is rewritten for the next unit
  return true;
}

template <int ESIZE>
__global__ void __launch_bounds__(THREADS, 1)
    contract_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const ContractArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* stage_base = smem;
  RowInfo* rinfo_all = (RowInfo*)(smem + (size_t)STAGES * STAGE_BYTES);
  uint64_t* bars =
      (uint64_t*)((unsigned char*)rinfo_all + (size_t)EPI_WARPS * RI_ROWS * sizeof(RowInfo));
  // bars: full[STAGES_MAX], empty[STAGES_MAX], tfull[2], tempty[2]; then the TMEM base slot
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES_MAX + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto FULL = [&](int s) { return bar0 + 8u * s; };
  auto EMPTY = [&](int s) { return bar0 + 8u * (STAGES_MAX + s); };
  auto TFULL = [&](int s) { return bar0 + 8u * (2 * STAGES_MAX + s); };
  auto TEMPTY = [&](int s) { return bar0 + 8u * (2 * STAGES_MAX + 2 + s); };
  // ring of the stage area: 4 stages of 48 KB, or 6 of 32 KB when units have <= 128 rows
  const bool narrow = a.bnr <= BM;
  const int nst = narrow ? STAGES_MAX : STAGES;
  const size_t sstride = narrow ? (size_t)(A_BYTES + BM * BKB) : (size_t)STAGE_BYTES;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(FULL(s), 1);
      mbar_init(EMPTY(s), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(TFULL(s), 1);
      mbar_init(TEMPTY(s), EPI_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *(volatile uint32_t*)tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      const uint64_t pol = l2_evict_last_policy();
      for (int64_t u = a.unit_lo + blockIdx.x; ok && u < a.unit_hi; u += gridDim.x) {
        const Unit t = unit_of(a, u);
        if (!t.live) continue;
        for (int64_t kb = 0; kb < t.num_kb; ++kb) {
          if (!mbar_wait(EMPTY(stage), phase ^ 1u)) {
            ok = false;
            break;
          }
          const uint32_t sa = smem_u32(stage_base + (size_t)stage * sstride);
          const uint32_t sb = sa + A_BYTES;
          // one or two 128-row boxes of rows; FP4 boxes count their packed bytes (half the
          // shared-memory footprint)
          mbar_expect_tx(FULL(stage),
                         (uint32_t)(A_BYTES + (a.bnr > BM ? 2 : 1) * BM * BKB) >> (a.afmt == 5 ? 1 : 0));
          const int kx = (int)(kb * BKB);
          tma_load_2d(sa, &tmA, kx, t.ta, FULL(stage), pol);
          tma_load_2d(sb, &tmB, kx, t.tb, FULL(stage), pol);
          if (a.bnr > BM) tma_load_2d(sb + BM * BKB, &tmB, kx, t.tb + BM, FULL(stage), pol);
          if (++stage == nst) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t kFmt = ESIZE == 1 ? (uint32_t)a.afmt : 1u;  // E4M3/E2M1 or BF16 (f16)
      const uint32_t idesc = (1u << 4) | (kFmt << 7) | (kFmt << 10) |
                             ((uint32_t)(a.bnr >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      for (int64_t u = a.unit_lo + blockIdx.x; ok && u < a.unit_hi; u += gridDim.x) {
        const Unit t = unit_of(a, u);
        if (!t.live) continue;
        if (!mbar_wait(TEMPTY(acc), acc_phase ^ 1u)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
        for (int64_t kb = 0; kb < t.num_kb; ++kb) {
          if (!mbar_wait(FULL(stage), phase)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(stage_base + (size_t)stage * sstride);
          const uint32_t sb = sa + A_BYTES;
#pragma unroll
          for (int k = 0; k < BKB / 32; ++k)
            umma<ESIZE>(d_tmem, sw128_desc(sa + 32 * k), sw128_desc(sb + 32 * k), idesc,
                        (kb > 0 || k > 0) ? 1u : 0u);
          umma_commit(EMPTY(stage));  // frees the stage once these MMAs have read it
          if (++stage == nst) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(TFULL(acc));  // accumulator complete
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
    }
  } else {
    // ---------------- Epilogue (warps 2..9) ----------------
    int acc = 0;
    uint32_t acc_phase = 0;
    RowInfo* ri = rinfo_all + (warp - 2) * RI_ROWS;
    for (int64_t u = a.unit_lo + blockIdx.x; u < a.unit_hi; u += gridDim.x) {
      const Unit t = unit_of(a, u);
      if (!t.live) continue;
      if (!epilogue_unit<true>(a, t, ri, tmem_base, TFULL(acc), acc_phase, acc, warp, lane,
                               TEMPTY(acc), false))
        break;
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1u;
      }
      if (sg_failed()) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base)
                 : "memory");
  }
}


// Pair form of the triangle contraction: the two CTAs of a cluster compute one 256 x 256
// super-tile with tcgen05.mma.cta_group::2 (M = 256 output columns, 128 per CTA; N = 256 output
// rows, whose operand is split 128 / 128 between the CTAs). Per stage each CTA loads 32 KB
// instead of 48 KB, so six stages fit where four did and every operand byte read from L2 feeds
// twice the MMA work. The leader CTA (rank 0) issues the MMAs; both CTAs' TMA loads complete on
// the leader's FULL barrier; the leader's commits arrive on both CTAs' EMPTY and TFULL barriers;
// both CTAs' epilogue warps release an accumulator on the leader's TEMPTY barrier.
__device__ __forceinline__ bool pair_live(const ContractArgs& a, int64_t s2) {
  return unit_of(a, 2 * s2).live || unit_of(a, 2 * s2 + 1).live;
}

// MX: block-scaled FP4 operands (kind::mxf4, packed e2m1 rows of 256 elements per 128-byte stage
// row, every scale factor 1.0, i.e. every byte of TMEM columns kSfCol.. is 0x7F = 2^0), MMA
// N = MXT rows: 240 x 240 super-tiles, the row operand loaded as 120 rows per CTA (tmRow's boxes
// are 120 rows high).
// ABS: the magnitude contraction's epilogue (n_3 only); a separate instantiation, so that the
// sign contraction's epilogue is compiled as if the mode did not exist.
template <int ESIZE, bool MX, bool ABS = false>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PAIR_THREADS, 1)
    contract2_kernel(const __grid_constant__ CUtensorMap tmRow,
                     const __grid_constant__ CUtensorMap tmCol, const ContractArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* stage_base = smem;
  constexpr int kStageBytes = MX ? STAGE2_MX_BYTES : STAGE2_BYTES;
  RowInfo* const rslots = (RowInfo*)(smem + (size_t)STAGES2 * kStageBytes);  // MX only
  uint64_t* bars =
      (uint64_t*)(smem + (size_t)STAGES2 * kStageBytes + (MX ? PAIR_EW * 32 * 16 : 0));
  // bars: full[STAGES2], empty[STAGES2], tfull[2], tempty[2]; then the TMEM base slot
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES2 + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int64_t cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int64_t s_lo = a.unit_lo >> 1, s_hi = a.unit_hi >> 1;
  const uint32_t bar0 = smem_u32(bars);
  auto FULL = [&](int s) { return bar0 + 8u * s; };
  auto EMPTY = [&](int s) { return bar0 + 8u * (STAGES2 + s); };
  auto TFULL = [&](int s) { return bar0 + 8u * (2 * STAGES2 + s); };
  auto TEMPTY = [&](int s) { return bar0 + 8u * (2 * STAGES2 + 2 + s); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES2; ++s) {
      mbar_init(FULL(s), 1);
      mbar_init(EMPTY(s), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(TFULL(s), 1);
      mbar_init(TEMPTY(s), 2 * PAIR_EW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers initialised before any cross-CTA signal
  tc_fence_after();
  const uint32_t tmem_base = *(volatile uint32_t*)tmem_slot;
  if (MX) {
    // Scale factors 1.0 in both CTAs before the first MMA: warps 2..5 cover the four lane
    // quarters (a warp reaches the TMEM lanes of quarter warp % 4), columns 496..511.
    if (warp >= 2 && warp < 6) {
      tmem_fill16(tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + kSfCol, 0x7F7F7F7Fu);
      tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
  }
  constexpr int kAccs = 2;       // accumulators in TMEM, at columns 0 and BN
  constexpr int kRows = MX ? MXT : BN;    // MMA N: output rows of a unit
  constexpr int kBrows = kRows / 2;       // row-operand rows loaded per CTA

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmRow) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmCol) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      const uint64_t pol = l2_evict_last_policy();
      for (int64_t s2 = s_lo + cid; ok && s2 < s_hi; s2 += ncl) {
        if (!pair_live(a, s2)) continue;
        const Unit t = unit_of(a, 2 * s2 + rank);
        const int brow = t.tb + kBrows * (int)rank;  // this CTA's half of the rows (operand row)
        for (int64_t kb = 0; kb < t.num_kb; ++kb) {
          if (!mbar_wait(EMPTY(stage), phase ^ 1u)) {
            ok = false;
            break;
          }
          const uint32_t sa = smem_u32(stage_base + (size_t)stage * kStageBytes);
          const uint32_t sb = sa + A_BYTES;
          // both CTAs' boxes; FP4 boxes expanded by the TMA count their packed bytes (half the
          // footprint); block-scaled FP4 boxes are plain bytes
          if (rank == 0)
            mbar_expect_tx(FULL(stage),
                           (2u * (A_BYTES + kBrows * BKB)) >> (!MX && a.afmt == 5 ? 1 : 0));
          const uint32_t full_leader = cluster_addr(FULL(stage), 0);
          const int kx = (int)(kb * BKB);
          tma_load_2d_pair(sa, &tmCol, kx, t.ta, full_leader, pol);
          tma_load_2d_pair(sb, &tmRow, kx, brow, full_leader, pol);
          if (++stage == STAGES2) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // Tail: every stage released by the leader's MMAs, so no commit is still to arrive here.
      for (int i = 0; ok && i < STAGES2; ++i) {
        if (!mbar_wait(EMPTY(stage), phase ^ 1u)) break;
        if (++stage == STAGES2) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (leader CTA) ----------------
    if (lane == 0 && rank == 0) {
      const uint32_t kFmt = ESIZE == 1 ? (uint32_t)a.afmt : 1u;  // E4M3/E2M1 or BF16 (f16)
      // kind::f8f6f4 / f16: F32 accumulator (bit 4), A and B formats, N / 8, M / 16.
      // kind::mxf4: scale-factor ids 0, A and B E2M1 (1), N / 8, UE8M0 scales (bit 23), M / 16.
      const uint32_t idesc =
          MX ? (1u << 7) | (1u << 10) | ((uint32_t)(kRows >> 3) << 17) | (1u << 23) |
                   ((uint32_t)((2 * BM) >> 4) << 24)
             : (1u << 4) | (kFmt << 7) | (kFmt << 10) | ((uint32_t)(kRows >> 3) << 17) |
                   ((uint32_t)((2 * BM) >> 4) << 24);
      const uint32_t sf = tmem_base + kSfCol;
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      for (int64_t s2 = s_lo + cid; ok && s2 < s_hi; s2 += ncl) {
        if (!pair_live(a, s2)) continue;
        if (!mbar_wait(TEMPTY(acc), acc_phase ^ 1u)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
        const int64_t num_kb = unit_of(a, 2 * s2).num_kb;  // per dataset in a batch
        for (int64_t kb = 0; kb < num_kb; ++kb) {
          if (!mbar_wait(FULL(stage), phase)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(stage_base + (size_t)stage * kStageBytes);
          const uint32_t sb = sa + A_BYTES;
#pragma unroll
          for (int k = 0; k < BKB / 32; ++k) {
            if (MX)
              umma_pair_mx(d_tmem, sw128_desc(sa + 32 * k), sw128_desc(sb + 32 * k), idesc, sf, sf,
                           (kb > 0 || k > 0) ? 1u : 0u);
            else
              umma_pair<ESIZE>(d_tmem, sw128_desc(sa + 32 * k), sw128_desc(sb + 32 * k), idesc,
                               (kb > 0 || k > 0) ? 1u : 0u);
          }
          umma_commit_pair(EMPTY(stage));  // frees the stage in both CTAs
          if (++stage == STAGES2) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit_pair(TFULL(acc));  // accumulator complete in both CTAs
        if (++acc == kAccs) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
    }
  } else {
    // ---------------- Epilogue (warps 2.., both CTAs) ----------------
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int64_t s2 = s_lo + cid; s2 < s_hi; s2 += ncl) {
      if (!pair_live(a, s2)) continue;
      const Unit t = unit_of(a, 2 * s2 + rank);
      const bool ok =
          MX ? epilogue_unit<false, true, PAIR_EW, ABS>(a, t, rslots + 32 * (warp - 2), tmem_base,
                                                   TFULL(acc), acc_phase, acc, warp, lane,
                                                   cluster_addr(TEMPTY(acc), 0), true)
             : epilogue_unit<false, false, PAIR_EW>(a, t, nullptr, tmem_base, TFULL(acc),
                                                    acc_phase, acc, warp, lane,
                                                    cluster_addr(TEMPTY(acc), 0), true);
      if (!ok) break;
      if (++acc == kAccs) {
        acc = 0;
        acc_phase ^= 1u;
      }
      if (sg_failed()) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs done with TMEM, barriers and each other's shared memory
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem_base)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
// cuTensorMapEncodeTiled through the runtime's driver entry-point query, so the library does not
// link libcuda directly (it still loads on machines without a driver).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 128 x 128-element boxes with 128-byte swizzle. FP4 rows (fp4 = true) are packed in global
// memory (row_bytes = K_pad / 2) and land in shared memory as 16-byte containers holding 16
// elements in their first 8 bytes, one byte of shared memory per element like FP8.
ktau_status make_tmap_raw(void* tmap, void* base, int64_t row_bytes_, int64_t rows,
                          bool fp4 = false, int box_rows = BM) {
  CUtensorMap* tm = reinterpret_cast<CUtensorMap*>(tmap);
  PFN_cuTensorMapEncodeTiled_v12000 cuTensorMapEncodeTiled = encode_fn();
  if (!cuTensorMapEncodeTiled) return ktau_fail(KTAU_ECUDA, "cuTensorMapEncodeTiled unavailable");
  const cuuint64_t row_bytes = (cuuint64_t)row_bytes_;
  cuuint64_t dims[2] = {fp4 ? 2 * row_bytes : row_bytes, (cuuint64_t)rows};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {(cuuint32_t)BKB, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = cuTensorMapEncodeTiled(tm, fp4 ? CU_TENSOR_MAP_DATA_TYPE_16U4_ALIGN16B
                                              : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                                      2, base, dims, strides,
                                      box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                      CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return ktau_fail(KTAU_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return KTAU_OK;
}

ktau_status make_tmap(ktau_ranked* R) {
  ktau_status s = make_tmap_raw(R->tmap, R->sgn, R->K_pad * R->obits / 8, R->m, R->obits == 4);
  if (s == KTAU_OK && R->obits == 4) s = make_tmap_raw(R->tmap_mx, R->sgn, R->K_pad / 2, R->m);
  if (s == KTAU_OK && R->obits == 4)
    s = make_tmap_raw(R->tmap_mxb, R->sgn, R->K_pad / 2, R->m, false, MXB);
  return s;
}

SideArgs side_of(const ktau_ranked* R) {
  return SideArgs{R->rank,    R->perm,      R->srank,   R->ld, R->T, R->rs64, R->rsff,
                  R->tie_off, R->tie_pairs, R->tie_cap, R->m};
}

template <int JCOLS>
ktau_status launch_joint_ties_t(const ktau_ranked* A, const ktau_ranked* B, int tri,
                                uint64_t p_begin, uint64_t p_end, int64_t ldo, void* n3,
                                int count_bits, cudaStream_t st) {
  const size_t smem = (size_t)(JCAP + JT + 8) * 4 + (size_t)B->n * (JCOLS + 1) * sizeof(uint16_t);
  if (smem > 227 * 1024) return ktau_fail(KTAU_ETOOLARGE, "joint-ties staging too large");
  auto kern = joint_ties_kernel<JCOLS>;
  KTAU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t w = 0, ncb = 0, lo = 0, hi = 0;
  if (tri) {
    const int64_t m = A->m;
    w = (m + JT - 1) / JT;
    int64_t i0, j0, i1, j1;
    ktau_tile_coord(m - 1, (int64_t)p_begin, i0, j0);
    ktau_tile_coord(m - 1, (int64_t)(p_end - 1), i1, j1);
    lo = ktau_rowstart(w, i0 / JT);
    hi = ktau_rowstart(w, i1 / JT + 1);
  } else {
    ncb = (B->m + JT - 1) / JT;
    hi = ((A->m + JT - 1) / JT) * ncb;
  }
  // n_3 is 0 for every pair with a tie-free variable: the contraction's epilogue has stored the
  // zeros, so these kernels store (or add) only the nonzero counts.
  int occ = 0;
  KTAU_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem));
  int64_t grid = (int64_t)(occ > 0 ? occ : 1) * ktau_sm_count();
  if (grid > hi - lo) grid = hi - lo;
  if (grid < 1) grid = 1;
  const unsigned long long* bstat = (tri && A->bkt_stat) ? A->bkt_stat : nullptr;
  if (bstat) {
    // Bucket form first; the tile kernel below returns at once when the bucket flag is set.
    KTAU_TRACE("bucket_n3_kernel", st);
    bucket_n3_kernel<<<(unsigned)(4 * ktau_sm_count()), 256, 0, st>>>(
        A->bkt_off, A->bkt_var, A->bkt_stat, A->K, A->m, p_begin, p_end, n3, count_bits);
    KTAU_CUDA(cudaGetLastError());
  }
  KTAU_TRACE("joint_ties_kernel", st);
  kern<<<(unsigned)grid, 256, smem, st>>>(side_of(A), side_of(B), A->n, tri, w, ncb, lo, hi,
                                          p_begin, p_end, ldo, n3, count_bits, bstat);
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

ktau_status launch_joint_ties(const ktau_ranked* A, const ktau_ranked* B, int tri, uint64_t p_begin,
                              uint64_t p_end, int64_t ldo, void* n3, int count_bits,
                              cudaStream_t st) {
  // 64 column variables staged at a time; 32 for long vectors (shared memory).
  return B->n <= 1024
             ? launch_joint_ties_t<64>(A, B, tri, p_begin, p_end, ldo, n3, count_bits, st)
             : launch_joint_ties_t<32>(A, B, tri, p_begin, p_end, ldo, n3, count_bits, st);
}

template <int ESIZE>
ktau_status launch_contract_maps(const void* tmap_a, const void* tmap_b, const ContractArgs& args,
                                 int64_t units, cudaStream_t st) {
  auto kern = contract_kernel<ESIZE>;
  KTAU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SMEM_BYTES));
  int64_t grid = ktau_sm_count();
  if (grid > units) grid = units;
  if (grid < 1) grid = 1;
  const CUtensorMap* ta = reinterpret_cast<const CUtensorMap*>(tmap_a);
  const CUtensorMap* tb = reinterpret_cast<const CUtensorMap*>(tmap_b);
  KTAU_TRACE("contract_kernel", st);
  kern<<<(unsigned)grid, THREADS, SMEM_BYTES, st>>>(*ta, *tb, args);
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

// Pair form over the triangle of one matrix: clusters of two CTAs, as many as fit at once.
template <int ESIZE>
ktau_status launch_contract2_map(const void* tmap_row, const void* tmap_col,
                                 const ContractArgs& args, int64_t units, cudaStream_t st) {
  const bool mx = ESIZE == 1 && args.afmt == kMxFmt;
  auto kern = mx ? (args.absmode ? contract2_kernel<1, true, true> : contract2_kernel<1, true>)
                 : contract2_kernel<ESIZE, false>;
  const size_t smem = mx ? SMEM2_MX_BYTES : SMEM2_BYTES;
  KTAU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  static int max_clusters_by[3][64] = {{0}};
  int* const max_clusters = max_clusters_by[mx ? (args.absmode ? 2 : 1) : 0];
  int dev = 0;
  KTAU_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return ktau_fail(KTAU_EINVAL, "device index out of range");
  if (max_clusters[dev] == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * ktau_sm_count()));
    cfg.blockDim = dim3(PAIR_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    KTAU_CUDA(cudaOccupancyMaxActiveClusters(&n, (void*)kern, &cfg));
    max_clusters[dev] = n > 0 ? n : -1;
  }
  if (max_clusters[dev] < 0) return ktau_fail(KTAU_ECUDA, "no two-CTA cluster fits on an SM pair");
  int64_t clusters = max_clusters[dev];
  const int64_t supers = (units + 1) / 2;
  if (clusters > supers) clusters = supers;
  if (clusters < 1) clusters = 1;
  KTAU_TRACE("contract_kernel", st);
  kern<<<(unsigned)(2 * clusters), PAIR_THREADS, smem, st>>>(
      *reinterpret_cast<const CUtensorMap*>(tmap_row),
      *reinterpret_cast<const CUtensorMap*>(tmap_col), args);
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

// Tensor maps of a handle's operands for the pair kernel with these arguments: the row operand
// (u, the MMA's B) and the column operand (v, the MMA's A).
const void* pair_tmap_row(const ktau_ranked* R, const ContractArgs& args) {
  return args.afmt == kMxFmt ? (const void*)R->tmap_mxb : (const void*)R->tmap;
}
const void* pair_tmap_col(const ktau_ranked* R, const ContractArgs& args) {
  return args.afmt == kMxFmt ? (const void*)R->tmap_mx : (const void*)R->tmap;
}

template <int ESIZE>
ktau_status launch_contract2(const ktau_ranked* R, const ContractArgs& args, int64_t units,
                             cudaStream_t st) {
  return launch_contract2_map<ESIZE>(pair_tmap_row(R, args), pair_tmap_col(R, args), args, units,
                                     st);
}

// Rows from A, columns from B: the MMA's A operand (TMEM lanes) is the column side.
template <int ESIZE>
ktau_status launch_contract(const ktau_ranked* A, const ktau_ranked* B, const ContractArgs& args,
                            int64_t units, cudaStream_t st) {
  return launch_contract_maps<ESIZE>(B->tmap, A->tmap, args, units, st);
}

}  // namespace

bool ktau_signgemm_supported(int64_t n) { return n >= 2 && n <= KTAU_SIGNGEMM_MAX_N; }

int ktau_sign_obits(int64_t n, const ktau_options* opt) {
  if (opt && (opt->operand_bits == 4 || opt->operand_bits == 8 || opt->operand_bits == 16))
    return opt->operand_bits;
  // FP4: half the operand bytes of FP8, and the pair contraction reads them with the
  // block-scaled FP4 MMA (measured on GB300 at 16384 x 128: 0.69 ms against 0.79 ms with FP8).
  return n <= KTAU_SIGNGEMM_FP8_MAX_N ? KTAU_SIGNGEMM_DEFAULT_BITS : 16;
}


// ---------------------------------------------------------------------------------------------
// Side stream: work that only the n_3 output needs (tie lists, the inverted index, the zero fill
// and the n_3 kernels) runs on a library-owned stream forked from the caller's stream by an
// event and joined back by another, so that it overlaps the sign expansion and the contraction.
// One side stream per device; its fork is taken under a mutex so that concurrent callers cannot
// interleave the record/wait pair. Callers whose stream is being captured, and small jobs, run
// everything on their own stream.
// ---------------------------------------------------------------------------------------------
namespace {
struct SideLane {
  std::mutex mu;
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
SideLane g_side[64];

// A timing-enabled event recorded on the stream just before the pair contraction (never waited
// on). Measured on GB300 at m = 16384, n = 128: the contraction queued directly behind the sign
// expansion takes 0.819 ms, and 0.796 ms when this event (or any kernel) separates the two; an
// event without timing does not have that effect. Skipped while the stream is being captured.
std::mutex g_mark_mu;
cudaEvent_t g_mark[64] = {};
void mark_before_contraction(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(g_mark_mu);
  if (!g_mark[dev] && cudaEventCreate(&g_mark[dev]) != cudaSuccess) {
    g_mark[dev] = nullptr;
    cudaGetLastError();
    return;
  }
  cudaEventRecord(g_mark[dev], st);
}

class SideFork {
 public:
  SideFork(cudaStream_t st, bool want) : st_(st) {
    if (!want) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    lane_ = &g_side[dev];
    lane_->mu.lock();
    if (!lane_->s &&
        (cudaStreamCreateWithFlags(&lane_->s, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&lane_->fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&lane_->join, cudaEventDisableTiming) != cudaSuccess)) {
      lane_->s = nullptr;
      lane_->mu.unlock();
      lane_ = nullptr;
      return;
    }
    if (cudaEventRecord(lane_->fork, st) != cudaSuccess ||
        cudaStreamWaitEvent(lane_->s, lane_->fork, 0) != cudaSuccess) {
      lane_->mu.unlock();
      lane_ = nullptr;
      return;
    }
    side_ = lane_->s;
  }
  cudaStream_t stream() const { return side_ ? side_ : st_; }
  // Joins the side stream back into the caller's stream; later work on the caller's stream
  // waits for everything launched on stream() so far.
  ktau_status join() {
    if (!lane_) return KTAU_OK;
    cudaError_t e = cudaEventRecord(lane_->join, side_);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st_, lane_->join, 0);
    lane_->mu.unlock();
    lane_ = nullptr;
    side_ = nullptr;
    return e == cudaSuccess ? KTAU_OK : ktau_cuda_fail(e, "side stream join");
  }
  ~SideFork() { join(); }

 private:
  cudaStream_t st_;
  cudaStream_t side_ = nullptr;
  SideLane* lane_ = nullptr;
};
}  // namespace

// Sign expansion of R's ranks into R->sgn (R->K, K_pad, obits and esize set).
ktau_status launch_sign_expand(const ktau_ranked* R, cudaStream_t st) {
  const int64_t n = R->n;
  const size_t smem = expand_smem(n);
  const int rows = ktau_expand_rows(n);
  const unsigned eblocks = (unsigned)((R->m + rows - 1) / rows);
  KTAU_TRACE("sign_expand_kernel", st);
  auto pick = [rows](auto k8, auto k4, auto k2) { return rows == 8 ? k8 : (rows == 4 ? k4 : k2); };
  auto kern = R->obits == 4
                  ? pick(sign_expand_kernel<4, 8>, sign_expand_kernel<4, 4>, sign_expand_kernel<4, 2>)
                  : (R->obits == 8 ? pick(sign_expand_kernel<8, 8>, sign_expand_kernel<8, 4>,
                                          sign_expand_kernel<8, 2>)
                                   : pick(sign_expand_kernel<16, 8>, sign_expand_kernel<16, 4>,
                                          sign_expand_kernel<16, 2>));
  KTAU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<eblocks, kExpandThreads, smem, st>>>(R->rank, R->ld, (int)n, R->m, (int)R->K,
                                              (int)R->K_pad, (uint8_t*)R->sgn);
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

// |A| operand (FP4, block-scaled pair kernel only) of a handle whose FP4 signs are built:
// expansion of the magnitudes into R->sgn_abs and its tensor maps, once per handle.
static ktau_status signgemm_prepare_abs(ktau_ranked* R, cudaStream_t st) {
  if (R->abs_ready) return KTAU_OK;
  if (R->obits != 4) return ktau_fail(KTAU_EINVAL, "the magnitude operand needs FP4 signs");
  const int64_t n = R->n;
  R->sgn_abs_bytes = (size_t)R->m * R->K_pad / 2;
  if (ktau_dmalloc(&R->sgn_abs, R->sgn_abs_bytes) != KTAU_OK) {
    R->sgn_abs = nullptr;
    return KTAU_ENOMEM;
  }
  const size_t smem = expand_smem(n);
  const int rows = ktau_expand_rows(n);
  const unsigned eblocks = (unsigned)((R->m + rows - 1) / rows);
  auto kern = rows == 8 ? sign_expand_kernel<4, 8, true>
                        : (rows == 4 ? sign_expand_kernel<4, 4, true> : sign_expand_kernel<4, 2, true>);
  KTAU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    KTAU_TRACE("sign_expand_kernel", st);
    kern<<<eblocks, kExpandThreads, smem, st>>>(R->rank, R->ld, (int)n, R->m, (int)R->K,
                                                (int)R->K_pad, (uint8_t*)R->sgn_abs);
  }
  KTAU_CUDA(cudaGetLastError());
  ktau_status s = make_tmap_raw(R->tmap_mx_abs, R->sgn_abs, R->K_pad / 2, R->m);
  if (s == KTAU_OK) s = make_tmap_raw(R->tmap_mxb_abs, R->sgn_abs, R->K_pad / 2, R->m, false, MXB);
  if (s != KTAU_OK) return s;
  R->abs_ready = 1;
  return KTAU_OK;
}

ktau_status ktau_signgemm_prepare(ktau_ranked* R, int obits, cudaStream_t st) {
  if (obits != 4 && obits != 8 && obits != 16)
    return ktau_fail(KTAU_EINVAL, "operand bits must be 4, 8 or 16");
  if (R->sg_ready && R->obits == obits) return KTAU_OK;
  if (R->sg_ready) {  // built for the other operand type: rebuild
    KTAU_CUDA(cudaStreamSynchronize(st));
    ktau_signgemm_release(R);
  }
  if (!ktau_signgemm_supported(R->n))
    return ktau_fail(KTAU_EINVAL, "sign contraction supports 2 <= n <= %d", KTAU_SIGNGEMM_MAX_N);
  const int64_t n = R->n;
  R->K = n * (n - 1) / 2;
  R->K_pad = ktau_kpad(R->K, obits);
  R->obits = obits;
  R->esize = obits == 16 ? 2 : 1;
  R->sgn_bytes = (size_t)R->m * R->K_pad * obits / 8;
  if (ktau_dmalloc(&R->sgn, R->sgn_bytes) != KTAU_OK) return KTAU_ENOMEM;
  ktau_status s = launch_sign_expand(R, st);
  if (s != KTAU_OK) return s;
  s = make_tmap(R);
  if (s != KTAU_OK) return s;
  R->sg_ready = 1;
  return KTAU_OK;
}

// Lists of tied sample pairs for n_3 and their inverted index, built once per handle on the
// first call that stores n_3. The kernels are small (at most 256 threads, few registers) so that
// they can run on the SMs beside the persistent contraction when launched on a side stream.
ktau_status ktau_signgemm_ties(ktau_ranked* R, cudaStream_t ss) {
  if (R->ties_ready) return KTAU_OK;
  const int64_t n = R->n;
  R->K = n * (n - 1) / 2;
  // exact capacity from the rank statistics
  R->tie_cap = (int64_t)R->stats.T_sum;
  R->tie_bytes = (size_t)(R->tie_cap > 0 ? R->tie_cap : 1) * 4;
  // inverted index for the bucket form of n_3 (built when the counts fit 32-bit offsets)
  const bool buckets = R->stats.T_sum > 0 && R->stats.T_sum < (1ll << 31) && R->m < (1ll << 31);
  bool ok = ktau_dmalloc((void**)&R->tie_off, ((size_t)R->m + 1) * sizeof(int64_t)) == KTAU_OK &&
            ktau_dmalloc((void**)&R->tie_pairs, R->tie_bytes) == KTAU_OK;
  if (ok && buckets) {
    R->bkt_var_bytes = (size_t)R->stats.T_sum * sizeof(int32_t);
    ok = ktau_dmalloc((void**)&R->bkt_off, ((size_t)R->K + 1) * sizeof(int32_t)) == KTAU_OK &&
         ktau_dmalloc((void**)&R->bkt_var, R->bkt_var_bytes) == KTAU_OK &&
         ktau_dmalloc((void**)&R->bkt_stat, 4 * sizeof(unsigned long long)) == KTAU_OK;
  }
  if (!ok) {  // give back what was allocated; a later call starts again
    ktau_dfree(R->tie_off, ((size_t)R->m + 1) * sizeof(int64_t));
    ktau_dfree(R->tie_pairs, R->tie_bytes);
    ktau_dfree(R->bkt_off, ((size_t)R->K + 1) * sizeof(int32_t));
    ktau_dfree(R->bkt_var, R->bkt_var_bytes);
    R->tie_off = nullptr;
    R->tie_pairs = nullptr;
    R->bkt_off = nullptr;
    R->bkt_var = nullptr;
    return KTAU_ENOMEM;
  }
  {
    KTAU_TRACE("ties_scan_kernel", ss);
    ties_scan_kernel<<<1, 256, 0, ss>>>(R->T, R->m, R->tie_off);
  }
  KTAU_CUDA(cudaGetLastError());
  if (buckets)
    KTAU_CUDA(cudaMemsetAsync(R->bkt_off, 0, ((size_t)R->K + 1) * sizeof(int32_t), ss));
  {
    KTAU_TRACE("ties_list_kernel", ss);
    ties_list_kernel<<<(unsigned)((R->m * 32 + 255) / 256), 256, 0, ss>>>(
        R->perm, R->srank, R->T, R->tie_off, R->ld, (int)n, R->m, R->tie_cap, R->tie_pairs,
        buckets ? R->bkt_off : nullptr);
  }
  KTAU_CUDA(cudaGetLastError());
  if (buckets) {
    // Bucket form when its atomic increments stay well below the pair count and no bucket is so
    // large that one warp would serialise on it.
    const unsigned long long P = (unsigned long long)(R->m * (R->m - 1) / 2);
    const unsigned long long lim_total = P / 16 > (1ull << 16) ? P / 16 : (1ull << 16);
    {
      KTAU_TRACE("bucket_scan_kernel", ss);
      bucket_scan_kernel<<<1, 128, 0, ss>>>(R->bkt_off, R->K, R->bkt_stat, lim_total, 1ull << 18);
    }
    KTAU_CUDA(cudaGetLastError());
    {
      KTAU_TRACE("bucket_scatter_kernel", ss);
      bucket_scatter_kernel<<<(unsigned)((R->m * 32 + 255) / 256), 256, 0, ss>>>(
          R->tie_pairs, R->T, R->tie_off, (int)n, R->m, R->tie_cap, R->bkt_off, R->bkt_var);
    }
    KTAU_CUDA(cudaGetLastError());
  }
  R->ties_ready = 1;
  return KTAU_OK;
}

// Contraction arguments of the triangle of one matrix over the pairs [p_begin, p_end).
ContractArgs tri_args(const ktau_ranked* R, uint64_t p_begin, uint64_t p_end, const ktau_out& out) {
  const int64_t m = R->m;
  ContractArgs a{};
  a.row = a.col = side_of(R);
  a.n = R->n;
  // FP4 operands go through the block-scaled pair kernel: 256 packed elements per stage row
  a.num_kb = R->obits == 4 ? R->K_pad / 2 / BKB : R->K_pad * R->esize / BKB;
  a.tri = 1;
  a.st = ktau_pair_tile(R->obits);
  a.wS = (m + a.st - 1) / a.st;
  a.ncb = 0;
  a.bnr = BN;
  a.afmt = R->obits == 4 ? kMxFmt : 0;
  a.p_begin = p_begin;
  a.p_end = p_end;
  a.ldo = 0;
  a.out = out;
  a.bds = nullptr;
  a.bids = nullptr;
  a.nb = 0;
  a.unit_prefix = nullptr;
  int64_t i0, j0, i1, j1;
  ktau_tile_coord(m - 1, (int64_t)p_begin, i0, j0);
  ktau_tile_coord(m - 1, (int64_t)(p_end - 1), i1, j1);
  a.wG = (a.wS + GROUP - 1) / GROUP;
  a.unit_lo = 2 * GROUP * GROUP * ktau_rowstart(a.wG, i0 / a.st / GROUP);
  a.unit_hi = 2 * GROUP * GROUP * ktau_rowstart(a.wG, i1 / a.st / GROUP + 1);
  a.s_obs = nullptr;
  a.exceed = nullptr;
  return a;
}

ktau_status ktau_signgemm_allpairs(ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                                   const ktau_out& out, int obits, cudaStream_t st) {
  ktau_status s = ktau_signgemm_prepare(R, obits, st);
  if (s != KTAU_OK) return s;
  const int64_t m = R->m;
  // Tie-heavy matrices (on average more than 4n tied sample pairs per variable, where the tie
  // lists' per-pair work outgrows a contraction) and rows too long for the tie-list tile kernel:
  // n_3 from a second contraction over the magnitudes |A| instead of the tie lists.
  const bool heavy = (double)R->stats.T_sum > 4.0 * (double)R->n * (double)m;
  if (out.n3 && (heavy || R->n > KTAU_SIGNGEMM_TIES_MAX_N) && obits == 4) {
    ktau_out oc = out;
    oc.n3 = nullptr;
    const ContractArgs a = tri_args(R, p_begin, p_end, oc);
    mark_before_contraction(st);
    s = launch_contract2<1>(R, a, a.unit_hi - a.unit_lo, st);
    if (s == KTAU_OK) s = signgemm_prepare_abs(R, st);
    if (s != KTAU_OK) return s;
    ktau_out on{nullptr, nullptr, nullptr, out.n3, out.count_bits, 0};
    ContractArgs b = tri_args(R, p_begin, p_end, on);
    b.absmode = 1;
    return launch_contract2_map<1>(R->tmap_mxb_abs, R->tmap_mx_abs, b, b.unit_hi - b.unit_lo, st);
  }
  if (out.n3 && R->n > KTAU_SIGNGEMM_TIES_MAX_N)
    return ktau_fail(KTAU_EINVAL, "n_3 of rows longer than %d samples needs FP4 operands",
                     KTAU_SIGNGEMM_TIES_MAX_N);
  const ContractArgs a = tri_args(R, p_begin, p_end, out);
  const int64_t units = a.unit_hi - a.unit_lo;
  // The epilogue zero-fills n_3 over the range; the joint-ties kernels then add nonzero counts.
  // The tie lists (first call only) are built beside the contraction on a side stream.
  const bool build_ties = out.n3 != nullptr && !R->ties_ready;
  mark_before_contraction(st);
  SideFork side(st, build_ties && m >= 4096);
  s = R->esize == 1 ? launch_contract2<1>(R, a, units, st) : launch_contract2<2>(R, a, units, st);
  if (s == KTAU_OK && build_ties) s = ktau_signgemm_ties(R, side.stream());
  const ktau_status sj = side.join();
  if (s == KTAU_OK) s = sj;
  if (s == KTAU_OK && out.n3)
    s = launch_joint_ties(R, R, 1, p_begin, p_end, 0, out.n3, out.count_bits, st);
  return s;
}

ktau_status ktau_signgemm_rect(ktau_ranked* Q, ktau_ranked* D, const ktau_out& out, int64_t ldo,
                               int obits, cudaStream_t st) {
  if (Q->n != D->n) return ktau_fail(KTAU_EINVAL, "sample counts differ");
  ktau_status s = ktau_signgemm_prepare(Q, obits, st);
  if (s == KTAU_OK) s = ktau_signgemm_prepare(D, obits, st);
  if (s != KTAU_OK) return s;
  ContractArgs a{};
  a.row = side_of(Q);
  a.col = side_of(D);
  a.n = Q->n;
  a.num_kb = Q->K_pad * Q->esize / BKB;
  a.tri = 0;
  a.st = 256;
  a.wS = 0;
  a.wG = 0;
  a.ncb = (D->m + BM - 1) / BM;
  a.bnr = Q->m <= 64 ? 64 : (Q->m <= BM ? BM : BN);  // MMA N: multiple of 16, up to 256
  a.s_obs = nullptr;
  a.exceed = nullptr;
  a.afmt = Q->obits == 4 ? 5 : 0;
  a.p_begin = 0;
  a.p_end = 0;
  a.ldo = ldo;
  a.out = out;
  a.bds = nullptr;
  a.bids = nullptr;
  a.nb = 0;
  a.unit_prefix = nullptr;
  a.unit_lo = 0;
  a.unit_hi = ((Q->m + a.bnr - 1) / a.bnr) * a.ncb;
  s = Q->esize == 1 ? launch_contract<1>(Q, D, a, a.unit_hi, st)
                    : launch_contract<2>(Q, D, a, a.unit_hi, st);
  if (s == KTAU_OK && out.n3) s = ktau_signgemm_ties(Q, st);
  if (s == KTAU_OK && out.n3) s = ktau_signgemm_ties(D, st);
  if (s == KTAU_OK && out.n3) s = launch_joint_ties(Q, D, 0, 0, 0, ldo, out.n3, out.count_bits, st);
  return s;
}

void ktau_signgemm_release(ktau_ranked* R) {
  ktau_dfree(R->sgn, R->sgn_bytes);
  ktau_dfree(R->sgn_abs, R->sgn_abs_bytes);
  R->sgn_abs = nullptr;
  R->abs_ready = 0;
  ktau_dfree(R->tie_off, ((size_t)R->m + 1) * sizeof(int64_t));
  ktau_dfree(R->tie_pairs, R->tie_bytes);
  ktau_dfree(R->bkt_off, ((size_t)R->K + 1) * sizeof(int32_t));
  ktau_dfree(R->bkt_var, R->bkt_var_bytes);
  ktau_dfree(R->bkt_stat, 4 * sizeof(unsigned long long));
  R->tie_off = nullptr;
  R->tie_pairs = nullptr;
  R->bkt_off = nullptr;
  R->bkt_var = nullptr;
  R->bkt_stat = nullptr;
  R->sgn = nullptr;
  R->sg_ready = 0;
  R->ties_ready = 0;
}

ktau_status ktau_signgemm_check_error(cudaStream_t st) {
  unsigned int e = 0;
  KTAU_CUDA(cudaMemcpyFromSymbolAsync(&e, g_sg_error, sizeof(e), 0, cudaMemcpyDeviceToHost, st));
  KTAU_CUDA(cudaStreamSynchronize(st));
  if (e) {
    const unsigned int zero = 0;
    cudaMemcpyToSymbolAsync(g_sg_error, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
    return ktau_fail(KTAU_ETIMEOUT, "tensor-core pipeline wait timed out");
  }
  return KTAU_OK;
}

// Batched groups run on the pair kernel only: FP4 rows are mapped as plain bytes for the
// block-scaled MMA.
ktau_status ktau_signgemm_make_tmap(void* tmap, void* base, int64_t row_bytes, int64_t rows,
                                    int obits, int box_rows) {
  (void)obits;
  return make_tmap_raw(tmap, base, row_bytes, rows, false, box_rows);
}

int ktau_pair_tile(int obits) { return obits == 4 ? MXT : 256; }

ktau_status ktau_signgemm_batch(const ktau_sg_group& g, cudaStream_t st) {
  if (g.nb == 0 || g.rows == 0) return KTAU_OK;
  const size_t smem_r = expand_smem(g.max_n);
  {
    KTAU_TRACE("batch_sign_expand_kernel", st);
    const int rows = ktau_expand_rows(g.max_n);
    auto pick = [rows](auto k8, auto k4, auto k2) { return rows == 8 ? k8 : (rows == 4 ? k4 : k2); };
    auto kern = g.obits == 4 ? pick(batch_sign_expand_kernel<4, 8>, batch_sign_expand_kernel<4, 4>,
                                    batch_sign_expand_kernel<4, 2>)
                             : (g.obits == 8 ? pick(batch_sign_expand_kernel<8, 8>,
                                                    batch_sign_expand_kernel<8, 4>,
                                                    batch_sign_expand_kernel<8, 2>)
                                             : pick(batch_sign_expand_kernel<16, 8>,
                                                    batch_sign_expand_kernel<16, 4>,
                                                    batch_sign_expand_kernel<16, 2>));
    KTAU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
    kern<<<(unsigned)g.blocks, kExpandThreads, smem_r, st>>>(g.ds, g.bids, g.nb, g.blk_prefix,
                                                              g.stride, (uint8_t*)g.sgn);
  }
  KTAU_CUDA(cudaGetLastError());
  {
    KTAU_TRACE("ties_scan_kernel", st);
    ties_scan_kernel<<<1, 1024, 0, st>>>(g.T, g.rows, g.tie_off);
  }
  KTAU_CUDA(cudaGetLastError());
  {
    KTAU_TRACE("batch_ties_list_kernel", st);
    batch_ties_list_kernel<<<(unsigned)((g.rows * 32 + 255) / 256), 256, 0, st>>>(
        g.ds, g.bids, g.nb, g.row_prefix, g.rows, g.T, g.tie_off, g.tie_cap, g.tie_pairs);
  }
  KTAU_CUDA(cudaGetLastError());
  ContractArgs a{};
  memset(&a, 0, sizeof(a));
  a.bds = g.ds;
  a.bids = g.bids;
  a.nb = g.nb;
  a.unit_prefix = g.unit_prefix;
  a.unit_lo = 0;
  a.unit_hi = g.units;
  a.tri = 1;
  a.st = ktau_pair_tile(g.obits);
  a.bnr = BN;
  a.afmt = g.obits == 4 ? kMxFmt : 0;
  ktau_status s = g.esize == 1 ? launch_contract2_map<1>(g.tmap_b, g.tmap, a, g.units, st)
                               : launch_contract2_map<2>(g.tmap_b, g.tmap, a, g.units, st);
  if (s != KTAU_OK) return s;
  const int jcols = g.max_n <= 1024 ? 64 : 32;
  const size_t smem = (size_t)(JCAP + JT + 8) * 4 + (size_t)g.max_n * (jcols + 1) * sizeof(uint16_t);
  auto jk = jcols == 64 ? batch_joint_ties_kernel<64> : batch_joint_ties_kernel<32>;
  KTAU_CUDA(cudaFuncSetAttribute(jk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  KTAU_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jk, 256, smem));
  int64_t grid = (int64_t)(occ > 0 ? occ : 1) * ktau_sm_count();
  if (grid > g.jt_tiles) grid = g.jt_tiles;
  if (grid < 1) grid = 1;
  KTAU_TRACE("batch_joint_ties_kernel", st);
  jk<<<(unsigned)grid, 256, smem, st>>>(g.ds, g.bids, g.nb, g.jt_prefix, g.jt_tiles);
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

extern "C" ktau_status ktau_debug_wait_timeout(int64_t limit_ns, void* stream) {
  if (limit_ns < 0 || limit_ns > 10000000000LL)
    return ktau_fail(KTAU_EINVAL, "limit must be in [0, 10 s]");
  wait_timeout_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((unsigned long long)limit_ns);
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

// ---------------------------------------------------------------------------------------------
// Permutation test of every pair
// ---------------------------------------------------------------------------------------------
extern "C" ktau_status ktau_permutation_exceed(const ktau_ranked* Rc, const uint16_t* perms,
                                               int32_t B, uint64_t p_begin, uint64_t p_end,
                                               const int32_t* S_obs, uint32_t* exceed,
                                               void* stream) {
  if (!Rc) return ktau_fail(KTAU_EINVAL, "handle is NULL");
  if (B < 0) return ktau_fail(KTAU_EINVAL, "B must be >= 0");
  if (B > 0 && !perms) return ktau_fail(KTAU_EINVAL, "perms is NULL");
  if (!S_obs || !exceed) return ktau_fail(KTAU_EINVAL, "S_obs and exceed are required");
  if (!ktau_signgemm_supported(Rc->n))
    return ktau_fail(KTAU_EINVAL, "the permutation test runs on the sign contraction: n <= %d",
                     KTAU_SIGNGEMM_MAX_N);
  const uint64_t P = (uint64_t)(Rc->m * (Rc->m - 1) / 2);
  if (p_begin > p_end || p_end > P) return ktau_fail(KTAU_EINVAL, "pair range outside the triangle");
  if (p_begin == p_end || B == 0) return KTAU_OK;
  ktau_status st0 = ktau_ranked_stats(Rc);
  if (st0 != KTAU_OK) return st0;
  ktau_ranked* R = const_cast<ktau_ranked*>(Rc);
  cudaStream_t st = (cudaStream_t)stream;
  ktau_status s = ktau_signgemm_prepare(R, ktau_sign_obits(R->n, nullptr), st);
  if (s != KTAU_OK) return s;
  // The relabelled copy: its own ranks and signs, everything else shared with R.
  ktau_ranked Rp = *R;
  const size_t rank_bytes = (size_t)R->m * R->ld * sizeof(uint16_t);
  Rp.rank = nullptr;
  Rp.sgn = nullptr;
  if (ktau_dmalloc((void**)&Rp.rank, rank_bytes) != KTAU_OK) return KTAU_ENOMEM;
  if (ktau_dmalloc(&Rp.sgn, R->sgn_bytes) != KTAU_OK) {
    ktau_dfree(Rp.rank, rank_bytes);
    return KTAU_ENOMEM;
  }
  s = make_tmap(&Rp);
  ContractArgs a = tri_args(R, p_begin, p_end, ktau_out{nullptr, nullptr, nullptr, nullptr, 32, 0});
  a.col = side_of(&Rp);
  a.s_obs = S_obs;
  a.exceed = exceed;
  const int64_t units = a.unit_hi - a.unit_lo;
  const int64_t total = R->m * R->ld;
  const unsigned pblocks = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
  for (int32_t b = 0; b < B && s == KTAU_OK; ++b) {
    {
      KTAU_TRACE("permute_ranks_kernel", st);
      permute_ranks_kernel<<<pblocks, 256, 0, st>>>(R->rank, R->ld, (int)R->n, R->m,
                                                   perms + (size_t)b * R->n, Rp.rank);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = ktau_cuda_fail(e, "permute_ranks_kernel");
    if (s == KTAU_OK) s = launch_sign_expand(&Rp, st);
    if (s == KTAU_OK)
      s = R->esize == 1
              ? launch_contract2_map<1>(pair_tmap_row(R, a), pair_tmap_col(&Rp, a), a, units, st)
              : launch_contract2_map<2>(pair_tmap_row(R, a), pair_tmap_col(&Rp, a), a, units, st);
  }
  // The scratch goes back to the cache only once the work that uses it has finished.
  const cudaError_t e = cudaStreamSynchronize(st);
  ktau_dfree(Rp.sgn, R->sgn_bytes);
  ktau_dfree(Rp.rank, rank_bytes);
  if (s == KTAU_OK && e != cudaSuccess) s = ktau_cuda_fail(e, "cudaStreamSynchronize");
  if (s == KTAU_OK) s = ktau_signgemm_check_error(st);
  return s;
}

// Two-sided permutation p-values from the exceedance counts: p = (count + 1) / (B + 1), the
// observed labelling counted as one of the B + 1 equally likely ones (IEEE FP64 quotient).
__global__ void permutation_pvalue_kernel(const uint32_t* __restrict__ exceed, uint64_t count,
                                          double den, double* __restrict__ pvalue) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x)
    pvalue[i] = __ddiv_rn((double)exceed[i] + 1.0, den);
}

extern "C" ktau_status ktau_permutation_pvalues(const uint32_t* exceed, int32_t B, uint64_t count,
                                                double* pvalue, void* stream) {
  if (B < 0) return ktau_fail(KTAU_EINVAL, "B must be >= 0");
  if (count == 0) return KTAU_OK;
  if (!exceed || !pvalue) return ktau_fail(KTAU_EINVAL, "exceed and pvalue are required");
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t blocks = std::min<uint64_t>((count + 255) / 256, (uint64_t)ktau_sm_count() * 8);
  {
    KTAU_TRACE("permutation_pvalue_kernel", st);
    permutation_pvalue_kernel<<<(unsigned)blocks, 256, 0, st>>>(exceed, count, (double)B + 1.0,
                                                                pvalue);
  }
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}
