// K-b: pairwise Knight counting (Sec. 3.2, Steps 1-5 with the merge-and-count of Algorithm 2)
// over the upper triangle of the job matrix, walked tile by tile through the job-id bijection
// (Sec. 4.1-4.2, Eq. 11-14) by persistent CTAs.
//
// Per pair (u, v) a "team" (one warp, or the whole CTA for long vectors) runs:
//   gather   : w_k = r_v[pi_u[k]] -- v's ranks listed in u's sorted order. This is the joint
//              list of Step 1 already ordered by u; only samples tied in u remain unordered.
//   Step 1   : if u has ties, sort the packed keys (group(u) << 16 | w) so that each tie group
//              of u is ordered by v (the 15/16-bit packing of the paper's vectorised kernel).
//              The keys arrive ordered by group, so when the largest u-tie group is short next
//              to n the merge levels stop at runs of that length and one fix-up pass places the
//              groups that straddle a run boundary.
//   Step 2   : n_3 = joint ties = sum over runs of equal keys of t(t-1)/2 (n_1 comes from K-a).
//   Step 3   : bottom-up merge sort of w; when an element of a right run is emitted while left
//              elements remain, all of those are larger (ties go left): add their number to n_d.
//   At every level of both sorts, a pair of runs already in order (last of the left run <= first
//   of the right run) is copied without merging (predict and skip: no inversion between them).
//   Step 4/5 : n_2 from K-a; S = n_0 - n_1 - n_2 + n_3 - 2 n_d; tau-b in FP64 (Eq. 3).
// The merge of two sorted runs is split among the team by merge-path co-ranks (a binary search
// along each thread's output diagonal); each thread then merges ITEMS outputs serially and counts
// exactly as Algorithm 2 does.
#include <algorithm>
#include <type_traits>

#include "ktau_impl.cuh"

namespace {

// Keys of the team buffers. 16-bit ranks (n <= 65535): 32-bit keys, (group << 16 | w) in Step 1.
// 32-bit ranks (longer rows): 64-bit keys, (group << 32 | w) -- the 64-bit packing of the paper's
// Sec. 6. The sentinel (all ones) sorts above every key.
template <typename RT>
using KeyOf = typename std::conditional<sizeof(RT) == 2, uint32_t, unsigned long long>::type;
template <typename K>
__device__ __forceinline__ constexpr K sentinel() { return (K)~(K)0; }
template <typename K>
constexpr int kGroupShift = (int)sizeof(K) * 4;

template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if (TEAM == 32)
    __syncwarp();
  else
    __syncthreads();
}

// Team-wide sum of a per-thread value (TEAM == 32: warp reduce; else CTA reduce via red[]).
template <int TEAM>
__device__ __forceinline__ unsigned long long team_sum(unsigned long long v,
                                                       unsigned long long* red) {
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  if (TEAM == 32) return v;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  unsigned long long t = 0;
  for (int w = 0; w < TEAM / 32; ++w) t += red[w];
  return t;
}

// Team buffers hold element i at word pd(i) = i + i / 32 when lanes own runs of 8 or more
// (lane l at l * ITEMS): unpadded, the accesses of one instruction would hit every
// (32 / ITEMS)-th bank; one pad word per 32 spreads them over all banks. Shorter runs are left
// unpadded: there the index arithmetic costs more than the conflicts (measured on 16384 x 128,
// four keys per lane: 1.75 ns per pair unpadded, 1.89 padded). Buffers are sized for the padded
// form: i + i / 32 + 1 words for n elements.
template <int ITEMS>
__device__ __forceinline__ int pd(int i) { return ITEMS >= 8 ? i + (i >> 5) : i; }

// Team-wide exclusive max-scan of one int per thread (lane order); -1 for the first lane.
template <int TEAM>
__device__ __forceinline__ int team_excl_max(int v, unsigned long long* red) {
  const int lane = threadIdx.x & 31, wid = (threadIdx.x % TEAM) >> 5;
  int incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl = max(incl, t);
  }
  int excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = -1;
  if (TEAM == 32) return excl;
  int* w = reinterpret_cast<int*>(red);  // TEAM / 32 warp maxima
  __syncthreads();
  if (lane == 31) w[wid] = incl;
  __syncthreads();
  for (int i = 0; i < wid; ++i) excl = max(excl, w[i]);
  __syncthreads();
  return excl;
}

// Step 1 with the merge levels stopped at runs of L >= the largest u-tie group (Sec. 3.2 Step 1
// sorts inside u-tie groups only). The keys (group << shift | w) are ordered by group on entry and
// every L-aligned run of `in` is sorted, so a tie group, at most L long, lies inside one run or
// straddles one run boundary; in the second case its part left of the boundary and its part right
// of it are each sorted. Each key of a straddling group moves to its final place: a left-part key
// past the right-part keys below it (found by binary search in the next run: keys of later groups
// are larger), a right-part key before the left-part keys above it (binary search in the previous
// run: keys of earlier groups are smaller). Equal keys keep left before right. Writes `out`.
template <int TEAM, int ITEMS, typename K>
__device__ __forceinline__ void team_group_fixup(const K* in, K* out, int n, int L, int lane) {
  constexpr int sh = kGroupShift<K>;
  for (int k = lane; k < n; k += TEAM) {
    const K key = in[pd<ITEMS>(k)];
    const int lo_b = k - k % L, hi_b = min(n, lo_b + L);
    int dst = k;
    if (hi_b < n && (in[pd<ITEMS>(hi_b)] >> sh) == (key >> sh)) {
      int lo = hi_b, hi = min(n, hi_b + L);  // first key of the next run that is >= key
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (in[pd<ITEMS>(mid)] < key)
          lo = mid + 1;
        else
          hi = mid;
      }
      dst = k + (lo - hi_b);
    } else if (lo_b > 0 && (in[pd<ITEMS>(lo_b - 1)] >> sh) == (key >> sh)) {
      int lo = lo_b - L, hi = lo_b;  // first key of the previous run that is > key
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (in[pd<ITEMS>(mid)] <= key)
          lo = mid + 1;
        else
          hi = mid;
      }
      dst = k - L + (lo - (lo_b - L));
    }
    out[pd<ITEMS>(dst)] = key;
  }
}

// Merge sort of buf[0, n) (ascending) with tmp as the second buffer. With COUNT, each thread
// accumulates into `cnt` its share of the inversions (pairs i < j with buf[i] > buf[j]).
// run_cap < n (Step 1 only, without COUNT): the merge levels stop once the sorted runs reach
// run_cap, and team_group_fixup finishes the sort inside u-tie groups no longer than run_cap.
// Returns the buffer that holds the sorted sequence. Every thread of the team must call it.
// K: key type (32-bit, or 64-bit for rows with 32-bit ranks, whose per-thread counts also need 64
// bits).
template <int TEAM, int ITEMS, bool COUNT, typename K>
__device__ K* team_merge_sort(K* buf, K* tmp, int n, int lane, unsigned long long& cnt,
                              int run_cap) {
  using C = typename std::conditional<sizeof(K) == 4, unsigned, unsigned long long>::type;
  constexpr int CH = TEAM * ITEMS;
  constexpr K kSentinel = sentinel<K>();
  C c = 0;
  // Runs of ITEMS sorted in registers (inversions inside a run counted directly).
  for (int base = 0; base < n; base += CH) {
    const int s0 = base + lane * ITEMS;
    K r[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) r[i] = (s0 + i < n) ? buf[pd<ITEMS>(s0 + i)] : kSentinel;
    if (COUNT) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i)
#pragma unroll
        for (int j = i + 1; j < ITEMS; ++j) c += (r[i] > r[j]);
    }
#pragma unroll
    for (int p = 0; p < ITEMS; ++p) {
#pragma unroll
      for (int i = p & 1; i + 1 < ITEMS; i += 2) {
        const K a = min(r[i], r[i + 1]), b = max(r[i], r[i + 1]);
        r[i] = a;
        r[i + 1] = b;
      }
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)
      if (s0 + i < n) buf[pd<ITEMS>(s0 + i)] = r[i];
  }
  team_sync<TEAM>();
  K* in = buf;
  K* out = tmp;
  int s = ITEMS;
  for (; s < n && s < run_cap; s *= 2) {
    for (int base = 0; base < n; base += CH) {
      const int o = base + lane * ITEMS;
      const int A = (o / (2 * s)) * (2 * s);
      const int a_len = min(s, n - A);
      const int B = A + a_len;
      const int b_len = max(0, min(s, n - B));
      const int diag = o - A;
      // Predict and skip: when the left run's last key is not greater than the right run's
      // first, the two runs are already in order: the outputs are the inputs in place and no
      // pair is an inversion. Taken only when every thread of the warp can take it (a warp's
      // threads may belong to different merges), so that no warp runs both paths.
      const bool sorted =
          o >= n || b_len == 0 || in[pd<ITEMS>(A + a_len - 1)] <= in[pd<ITEMS>(B)];
      if (__all_sync(0xffffffffu, sorted)) {
        if (o < n) {
          const int todo = min(ITEMS, a_len + b_len - diag);
#pragma unroll
          for (int i = 0; i < ITEMS; ++i)
            if (i < todo) out[pd<ITEMS>(o + i)] = in[pd<ITEMS>(o + i)];
        }
        continue;
      }
      if (o < n) {
        // Merge-path co-rank: number of A elements among the first `diag` outputs of a stable
        // merge (equal keys: A first).
        int lo = max(0, diag - b_len), hi = min(diag, a_len);
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (in[pd<ITEMS>(A + mid)] <= in[pd<ITEMS>(B + diag - 1 - mid)])
            lo = mid + 1;
          else
            hi = mid;
        }
        // Serial merge of ITEMS outputs without branches: an exhausted run reads as the
        // sentinel (above every key), so "take the right run" is vb < va; one load refills the
        // side taken. Outputs past the merge's end are not stored.
        int ai = A + lo, bi = B + diag - lo;
        const int ae = A + a_len, be = B + b_len;
        const int todo = min(ITEMS, a_len + b_len - diag);
        K va = ai < ae ? in[pd<ITEMS>(ai)] : kSentinel;
        K vb = bi < be ? in[pd<ITEMS>(bi)] : kSentinel;
        // o is a multiple of ITEMS and, where pd pads (ITEMS 8 or 16), [o, o + ITEMS) stays
        // within one 32-element row: the outputs are consecutive words from pd(o).
        K* op = out + pd<ITEMS>(o);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          const bool take_b = vb < va;
          if (i < todo) op[i] = take_b ? vb : va;
          if (COUNT) c += take_b ? (C)(ae - ai) : (C)0;  // remaining left keys are larger
          ai += take_b ? 0 : 1;
          bi += take_b ? 1 : 0;
          const bool more = take_b ? bi < be : ai < ae;
          const K v = more ? in[pd<ITEMS>(take_b ? bi : ai)] : kSentinel;
          va = take_b ? va : v;
          vb = take_b ? v : vb;
        }
      }
    }
    team_sync<TEAM>();
    K* t = in;
    in = out;
    out = t;
  }
  if (!COUNT && s < n) {
    team_group_fixup<TEAM, ITEMS, K>(in, out, n, s, lane);
    team_sync<TEAM>();
    in = out;
  }
  cnt += c;
  return in;
}

struct MergeArgs {
  // row side (u): permutation, sorted ranks, tie counts, factors; column side (v): ranks. The
  // rank arrays are uint16, or uint32 for rows longer than 65535 samples (the kernel's RT).
  const void* perm;
  const void* srank;
  const int64_t* T;
  const int32_t* maxg;   // largest tie group of each row variable
  ktau_fac fac;
  const void* rank;      // column side
  const int64_t* Tc;
  ktau_fac facc;
  int64_t m;             // row variables
  int64_t mc;            // column variables
  int64_t n, ld;
  int rect;              // 0: upper triangle of one matrix, 1: every row x every column
  int64_t ncb;           // rect: column tiles
  int64_t ldo;           // rect: output row stride
  int64_t w;        // tiles per side
  int64_t tile_lo;  // tile-id range covering [p_begin, p_end)
  int64_t tile_hi;
  uint64_t p_begin, p_end;
  int tq;           // tile side
  int stage;        // rows of the tile staged in shared memory
  int cap;          // per-team buffer capacity (elements)
  void* gbuf;       // long rows: the CTA team's two buffers in global scratch (2 * cap keys per CTA)
  unsigned long long* counter;  // dynamic schedule: next tile id (nullptr = static)
  ktau_out out;
};

// Counts for one pair. perm_u/srank_u/rank_v point at the three rows (shared or global); RT is
// the rank type and K = KeyOf<RT> the key type of the team buffers.
template <int TEAM, int ITEMS, typename RT, typename K = KeyOf<RT>>
__device__ __forceinline__ void count_pair(const RT* perm_u, const RT* srank_u, const RT* rank_v,
                                           int n, bool u_ties, int maxg_u, K* buf, K* tmp,
                                           int lane, unsigned long long* red, long long& nd_out,
                                           long long& n3_out) {
  constexpr int sh = kGroupShift<K>;
  constexpr K kLow = ((K)1 << sh) - 1;  // the w part of a packed key
  for (int k = lane; k < n; k += TEAM) {
    const K w = rank_v[perm_u[k]];
    buf[pd<ITEMS>(k)] = u_ties ? (((K)srank_u[k] << sh) | w) : w;
  }
  team_sync<TEAM>();
  unsigned long long nd = 0, n3 = 0;
  if (u_ties) {
    unsigned long long unused = 0;
    // Step 1 sorts inside u-tie groups: with groups short next to n, the merge levels stop at
    // runs as long as the largest group and a fix-up pass finishes the groups across runs.
    const int cap = 4 * maxg_u <= n ? maxg_u : n;
    K* sorted = team_merge_sort<TEAM, ITEMS, false>(buf, tmp, n, lane, unused, cap);
    K* other = sorted == buf ? tmp : buf;
    // Step 2: joint ties. In the sorted keys, position k has (k - first index of its run of
    // equal keys) earlier equal keys.
    if (TEAM > 32) {
      // Long vectors: each lane takes a contiguous segment; the last run head of every earlier
      // segment (team max-scan) is where its first run started.
      const int per = (n + TEAM - 1) / TEAM;
      const int kb = min(n, lane * per), ke = min(n, kb + per);
      int last = -1;
      for (int k = kb; k < ke; ++k)
        if (k == 0 || sorted[pd<ITEMS>(k)] != sorted[pd<ITEMS>(k - 1)]) last = k;
      int first = team_excl_max<TEAM>(last, red);
      for (int k = kb; k < ke; ++k) {
        const K key = sorted[pd<ITEMS>(k)];
        if (k == 0 || key != sorted[pd<ITEMS>(k - 1)]) first = k;
        n3 += (unsigned long long)(k - first);
        other[pd<ITEMS>(k)] = key & kLow;
      }
    } else {
      // Short vectors, few ties: the first index of a tied key by binary search.
      for (int k = lane; k < n; k += TEAM) {
        const K key = sorted[pd<ITEMS>(k)];
        if (k > 0 && sorted[pd<ITEMS>(k - 1)] == key) {
          int lo = 0, hi = k;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sorted[pd<ITEMS>(mid)] < key)
              lo = mid + 1;
            else
              hi = mid;
          }
          n3 += (unsigned long long)(k - lo);
        }
        other[pd<ITEMS>(k)] = key & kLow;
      }
    }
    team_sync<TEAM>();
    team_merge_sort<TEAM, ITEMS, true>(other, sorted, n, lane, nd, n);
  } else {
    team_merge_sort<TEAM, ITEMS, true>(buf, tmp, n, lane, nd, n);
  }
  nd_out = (long long)team_sum<TEAM>(nd, red);
  n3_out = (long long)team_sum<TEAM>(n3, red);
  team_sync<TEAM>();
}

// Stages rows [first_row, first_row + rows) of a rank array in shared memory with asynchronous
// 16-byte copies (cp.async, L2 only: every row is read once per tile); rows past m are not
// copied (no pair reads them). ld is a multiple of 16 ranks, so every row starts on 32 bytes.
// The caller waits with cp_async_wait_all() and a CTA barrier.
template <typename RT>
__device__ __forceinline__ void copy_rows(RT* dst, const RT* src, int64_t first_row, int rows,
                                          int64_t m, int64_t ld) {
  const int vec_per_row = (int)(ld * (int64_t)sizeof(RT) / 16);
  const int valid = (int)max((int64_t)0, min((int64_t)rows, m - first_row));
  const int total = valid * vec_per_row;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int r = i / vec_per_row, c = i % vec_per_row;
    const void* g = reinterpret_cast<const uint4*>(src + (first_row + r) * ld) + c;
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(
        reinterpret_cast<uint4*>(dst + (int64_t)r * ld) + c);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(g) : "memory");
  }
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// GBUF: the team buffers are in global scratch (long rows); otherwise they are carved from
// shared memory, a pointer the compiler can see is shared (shared-memory loads and stores).
// RT: rank type (uint16_t, or uint32_t for rows longer than 65535 samples). Registers are held
// to what a higher CTA count per SM needs where that measured faster: the CTA-per-pair form with
// 16 keys per lane at four CTAs (64 registers, a few spilled; 2048 x 4096 heavy ties: 105 -> 100
// ns per pair), warp-per-pair forms with up to 7 keys per lane at five CTAs (48 registers;
// 16384 x 128: 2.26 -> 1.76 ns per pair). With 8 keys per lane five CTAs spill and were slower at
// n = 900.
template <int TEAM, int ITEMS, bool GBUF, typename RT>
__global__ void __launch_bounds__(
    256, (TEAM == 256 && ITEMS == 16 && !GBUF) ? 4 : ((TEAM == 32 && ITEMS <= 7) ? 5 : 1))
    merge_pairs_kernel(const MergeArgs a) {
  using K = KeyOf<RT>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red[8];
  __shared__ long long next_tile;
  const int nteams = blockDim.x / TEAM;
  const int team = threadIdx.x / TEAM, lane = threadIdx.x % TEAM;
  const int tq = a.tq;
  const int64_t ld = a.ld;
  const RT* g_perm = static_cast<const RT*>(a.perm);
  const RT* g_srank = static_cast<const RT*>(a.srank);
  const RT* g_rank = static_cast<const RT*>(a.rank);
  RT* s_perm = reinterpret_cast<RT*>(smem);
  RT* s_srank = s_perm + (a.stage ? (int64_t)tq * ld : 0);
  RT* s_rank = s_srank + (a.stage ? (int64_t)tq * ld : 0);
  K* tbuf = GBUF ? static_cast<K*>(a.gbuf) + (size_t)blockIdx.x * 2 * a.cap
                 : reinterpret_cast<K*>(s_rank + (a.stage ? (int64_t)tq * ld : 0)) +
                       (size_t)team * 2 * a.cap;
  K* tbuf2 = tbuf + a.cap;
  const int n = (int)a.n;
  const int64_t n0 = a.n * (a.n - 1) / 2;

  int64_t t = a.tile_lo + blockIdx.x;
  while (true) {
    if (a.counter) {
      __syncthreads();
      if (threadIdx.x == 0) next_tile = a.tile_lo + (long long)atomicAdd(a.counter, 1ull);
      __syncthreads();
      t = next_tile;
    }
    if (t >= a.tile_hi) break;
    int64_t yq, xq;
    if (a.rect) {
      yq = t / a.ncb;
      xq = t % a.ncb;
    } else {
      ktau_tile_coord(a.w, t, yq, xq);
    }
    const int64_t y0 = yq * tq, x0 = xq * tq;
    if (a.stage) {
      __syncthreads();
      copy_rows<RT>(s_perm, g_perm, y0, tq, a.m, ld);
      copy_rows<RT>(s_srank, g_srank, y0, tq, a.m, ld);
      copy_rows<RT>(s_rank, g_rank, x0, tq, a.mc, ld);
      cp_async_wait_all();
      __syncthreads();
    }
    for (int e = team; e < tq * tq; e += nteams) {
      const int64_t y = y0 + e / tq, x = x0 + e % tq;
      if (y >= a.m || x >= a.mc) continue;
      uint64_t k;
      if (a.rect) {
        k = (uint64_t)y * (uint64_t)a.ldo + (uint64_t)x;
      } else {
        if (x <= y) continue;
        const uint64_t p = ktau_pair_index(a.m, y, x);
        if (p < a.p_begin || p >= a.p_end) continue;
        k = p - a.p_begin;
      }
      const RT* pu = a.stage ? s_perm + (y - y0) * ld : g_perm + y * ld;
      const RT* su = a.stage ? s_srank + (y - y0) * ld : g_srank + y * ld;
      const RT* rv = a.stage ? s_rank + (x - x0) * ld : g_rank + x * ld;
      const int64_t Tu = a.T[y], Tv = a.Tc[x];
      long long nd, n3;
      count_pair<TEAM, ITEMS, RT>(pu, su, rv, n, Tu > 0, a.maxg[y], tbuf, tbuf2, lane, red, nd,
                                  n3);
      if (lane == 0) {
        const int64_t S = n0 - Tu - Tv + n3 - 2 * nd;
        if (a.out.tau64)
          a.out.tau64[k] = a.out.stat ? ktau_taua64(S, n0)
                                      : ktau_tau64(S, a.fac.rs64[y], a.facc.rs64[x]);
        if (a.out.tau32)
          a.out.tau32[k] = a.out.stat ? ktau_taua32(S, n0)
                                      : ktau_tau32(S, a.fac.rsff[y], a.facc.rsff[x], n0, Tu, Tv);
        if (a.out.count_bits == 64) {
          if (a.out.S) ((long long*)a.out.S)[k] = S;
          if (a.out.n3) ((long long*)a.out.n3)[k] = n3;
        } else {
          if (a.out.S) ((int*)a.out.S)[k] = (int)S;
          if (a.out.n3) ((int*)a.out.n3)[k] = (int)n3;
        }
      }
    }
    if (!a.counter) t += gridDim.x;
  }
}

template <int TEAM, int ITEMS, bool GBUF = false, typename RT = uint16_t>
ktau_status launch_one(const MergeArgs& args, int threads, size_t smem, int ctas_per_sm,
                       int64_t tiles, cudaStream_t st, int64_t max_grid = 0) {
  auto kern = merge_pairs_kernel<TEAM, ITEMS, GBUF, RT>;
  KTAU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  KTAU_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
  if (occ < 1) return ktau_fail(KTAU_ETOOLARGE, "merge kernel does not fit on an SM (smem %zu)", smem);
  if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
  int64_t grid = (int64_t)occ * ktau_sm_count();
  if (grid > tiles) grid = tiles;
  if (max_grid > 0 && grid > max_grid) grid = max_grid;
  if (grid < 1) grid = 1;
  KTAU_TRACE("merge_pairs_kernel", st);
  kern<<<(unsigned)grid, threads, smem, st>>>(args);
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

// Counts of one pair with the register run length chosen from n (warp team).
__device__ __forceinline__ void count_pair_any(int items, const uint16_t* pu, const uint16_t* su,
                                               const uint16_t* rv, int n, bool ties, int maxg,
                                               uint32_t* buf, uint32_t* tmp, int lane,
                                               long long& nd, long long& n3) {
  switch (items) {
    case 1: count_pair<32, 1>(pu, su, rv, n, ties, maxg, buf, tmp, lane, nullptr, nd, n3); break;
    case 2: count_pair<32, 2>(pu, su, rv, n, ties, maxg, buf, tmp, lane, nullptr, nd, n3); break;
    case 3: count_pair<32, 3>(pu, su, rv, n, ties, maxg, buf, tmp, lane, nullptr, nd, n3); break;
    case 4: count_pair<32, 4>(pu, su, rv, n, ties, maxg, buf, tmp, lane, nullptr, nd, n3); break;
    case 5: count_pair<32, 5>(pu, su, rv, n, ties, maxg, buf, tmp, lane, nullptr, nd, n3); break;
    case 6: count_pair<32, 6>(pu, su, rv, n, ties, maxg, buf, tmp, lane, nullptr, nd, n3); break;
    case 7: count_pair<32, 7>(pu, su, rv, n, ties, maxg, buf, tmp, lane, nullptr, nd, n3); break;
    default: count_pair<32, 8>(pu, su, rv, n, ties, maxg, buf, tmp, lane, nullptr, nd, n3); break;
  }
}

// Batched form: the tiles of every merge-path dataset form one list (prefix over ids[]); a
// persistent CTA takes tile ids with a static stride, finds the dataset by binary search, and
// walks the dataset's own tile triangle (Eq. 13-14) one warp per pair.
template <int TEAM>
__global__ void __launch_bounds__(256) batch_merge_kernel(const ktau_bds* __restrict__ ds,
                                                          const int32_t* __restrict__ ids, int nids,
                                                          const int64_t* __restrict__ tile_prefix,
                                                          int64_t total_tiles, int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long red[8];
  const int nteams = blockDim.x / TEAM;
  const int team = threadIdx.x / TEAM, lane = threadIdx.x % TEAM;
  uint32_t* tbuf = reinterpret_cast<uint32_t*>(smem) + (size_t)team * 2 * cap;
  uint32_t* tbuf2 = tbuf + cap;
  for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    int lo = 0, hi = nids - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_prefix[mid] <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    const ktau_bds& D = ds[ids[lo]];
    int64_t yq, xq;
    ktau_tile_coord(D.w, t - tile_prefix[lo], yq, xq);
    const int tq = D.tq;
    const int64_t y0 = yq * tq, x0 = xq * tq;
    const int n = (int)D.n;
    const int items = n <= 256 ? (n + 31) / 32 : 8;
    const int64_t n0 = D.n * (D.n - 1) / 2;
    const ktau_fac fac{D.rs64, D.rsff, D.T};
    for (int e = team; e < tq * tq; e += nteams) {
      const int64_t y = y0 + e / tq, x = x0 + e % tq;
      if (y >= D.m || x >= D.m || x <= y) continue;
      const int64_t Tu = D.T[y], Tv = D.T[x];
      long long nd, n3;
      if (TEAM == 32)
        count_pair_any(items, D.perm + y * D.ld, D.srank + y * D.ld, D.rank + x * D.ld, n, Tu > 0,
                       D.maxg[y], tbuf, tbuf2, lane, nd, n3);
      else
        count_pair<TEAM, 8>(D.perm + y * D.ld, D.srank + y * D.ld, D.rank + x * D.ld, n, Tu > 0,
                            D.maxg[y], tbuf, tbuf2, lane, red, nd, n3);
      if (lane == 0) {
        const int64_t S = n0 - Tu - Tv + n3 - 2 * nd;
        ktau_store(D.out, ktau_pair_index(D.m, y, x), S, n3, n0, fac, y, x);
      }
    }
  }
}

}  // namespace

ktau_status ktau_launch_batch_merge(const ktau_bds* ds, const int32_t* ids, int nids,
                                    const int64_t* tile_prefix, int64_t total_tiles, int64_t max_n,
                                    int cta_team, cudaStream_t st) {
  if (nids == 0 || total_tiles == 0) return KTAU_OK;
  const int cap = (int)((max_n + (max_n >> 5) + 1 + 3) & ~3LL);  // pd<ITEMS>(n) + 1, rounded
  const size_t team_bytes = (size_t)2 * cap * sizeof(uint32_t);
  int teams = cta_team ? 1 : (int)std::min<size_t>(8, (200 * 1024) / team_bytes);
  if (teams < 1) return ktau_fail(KTAU_ETOOLARGE, "n=%lld too long for the batched merge path",
                                  (long long)max_n);
  const int threads = cta_team ? 256 : 32 * teams;
  const size_t smem = (size_t)teams * team_bytes;
  auto kern = cta_team ? batch_merge_kernel<256> : batch_merge_kernel<32>;
  KTAU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  KTAU_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
  int64_t grid = (int64_t)(occ > 0 ? occ : 1) * ktau_sm_count();
  if (grid > total_tiles) grid = total_tiles;
  KTAU_TRACE("batch_merge_kernel", st);
  kern<<<(unsigned)grid, threads, smem, st>>>(ds, ids, nids, tile_prefix, total_tiles, cap);
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

void ktau_merge_default_plan(int64_t n, ktau_merge_plan* plan) {
  // One warp per pair up to n = 1024, one CTA per pair above (autotuner, GB300: 86 vs 131 ns per
  // pair at n = 2000, 66 vs 66 at n = 1500).
  plan->mapping = n <= 1024 ? 1 : 2;
  plan->tile_q = n <= 256 ? 32 : (n <= 1024 ? 8 : 4);
  plan->schedule = 1;
  plan->ctas_per_sm = 0;
}

// Scratch for the dynamic schedule (one counter per device, reset before each launch).
static unsigned long long* g_counter[64];

static ktau_status launch_merge_impl(const ktau_ranked* R, const ktau_ranked* C, int rect,
                                     uint64_t p_begin, uint64_t p_end, int64_t ldo,
                                     const ktau_out& out, const ktau_merge_plan& plan,
                                     cudaStream_t st) {
  const int64_t m = R->m, n = R->n;
  const int tq = plan.tile_q > 0 ? plan.tile_q : 32;
  const int64_t w = (m + tq - 1) / tq;
  int64_t tile_lo = 0, tile_hi = 0, ncb = 0;
  if (rect) {
    ncb = (C->m + tq - 1) / tq;
    tile_hi = w * ncb;
  } else {
    // Rows of the first and last pair of the range -> covering tile-id range (Eq. 12 on tiles).
    int64_t i0, j0, i1, j1;
    ktau_tile_coord(m - 1, (int64_t)p_begin, i0, j0);
    ktau_tile_coord(m - 1, (int64_t)(p_end - 1), i1, j1);
    tile_lo = ktau_rowstart(w, i0 / tq);
    tile_hi = ktau_rowstart(w, i1 / tq + 1);
  }
  const int64_t tiles = tile_hi - tile_lo;

  if (R->wide != C->wide) return ktau_fail(KTAU_EINVAL, "rank widths of the two sides differ");
  MergeArgs a;
  a.perm = R->wide ? (const void*)R->perm32 : (const void*)R->perm;
  a.srank = R->wide ? (const void*)R->srank32 : (const void*)R->srank;
  a.T = R->T;
  a.maxg = R->maxg;
  a.fac = ktau_fac{R->rs64, R->rsff, R->T};
  a.rank = C->wide ? (const void*)C->rank32 : (const void*)C->rank;
  a.Tc = C->T;
  a.facc = ktau_fac{C->rs64, C->rsff, C->T};
  a.m = m;
  a.mc = C->m;
  a.rect = rect;
  a.ncb = ncb;
  a.ldo = ldo;
  a.n = n;
  a.ld = R->ld;
  a.w = w;
  a.tile_lo = tile_lo;
  a.tile_hi = tile_hi;
  a.p_begin = p_begin;
  a.p_end = p_end;
  a.tq = tq;
  a.out = out;
  a.counter = nullptr;
  if (plan.schedule == 2) {
    int dev = 0;
    KTAU_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return ktau_fail(KTAU_EINVAL, "device index out of range");
    if (!g_counter[dev]) KTAU_CUDA(cudaMalloc(&g_counter[dev], sizeof(unsigned long long)));
    KTAU_CUDA(cudaMemsetAsync(g_counter[dev], 0, sizeof(unsigned long long), st));
    a.counter = g_counter[dev];
  }

  const bool cta_team = plan.mapping == 2;
  if (R->wide && !cta_team)
    return ktau_fail(KTAU_EINVAL, "n=%lld > %d: the merge path takes one CTA per pair (mapping 2)",
                     (long long)n, KTAU_NARROW_MAX_N);
  const int items = cta_team ? (n > 2048 ? 16 : 8) : (n <= 256 ? (int)((n + 31) / 32) : 8);
  a.cap = (int)((n + (n >> 5) + 1 + 3) & ~3LL);  // pd<ITEMS>(n) + 1, rounded
  a.gbuf = nullptr;
  // keys of 4 bytes (16-bit ranks) or 8 bytes (32-bit ranks, the (group << 32 | w) packing)
  const size_t key_bytes = R->wide ? sizeof(unsigned long long) : sizeof(uint32_t);
  const size_t team_bytes = (size_t)2 * a.cap * key_bytes;
  // Stage the tile's rows in shared memory when they are small next to the per-pair work.
  const size_t stage_bytes = (size_t)3 * tq * R->ld * sizeof(uint16_t);
  a.stage = (!cta_team && stage_bytes <= 64 * 1024) ? 1 : 0;
  const size_t budget = 200 * 1024;
  int teams = 1, threads = 256;
  if (!cta_team) {
    const size_t avail = budget - (a.stage ? stage_bytes : 0);
    teams = (int)std::min<size_t>(8, avail / team_bytes);
    if (teams < 1) {
      a.stage = 0;
      teams = (int)std::min<size_t>(8, budget / team_bytes);
    }
    if (teams < 1)
      return ktau_fail(KTAU_ETOOLARGE, "n=%lld too long for one warp per pair; use mapping 2",
                       (long long)n);
    threads = 32 * teams;
  }
  const int cps = plan.ctas_per_sm;
  if (cta_team && team_bytes > budget) {
    // Long rows: the team's two merge buffers live in global scratch, one pair per SM at a time.
    // The scratch is released once the launch has finished, so this call returns after the work.
    const int64_t grid = ktau_sm_count();
    const size_t gbytes = (size_t)grid * team_bytes;
    void* g = nullptr;
    if (ktau_dmalloc(&g, gbytes) != KTAU_OK) return KTAU_ENOMEM;
    a.gbuf = g;
    ktau_status s = R->wide ? launch_one<256, 16, true, uint32_t>(a, threads, 0, cps, tiles, st, grid)
                            : launch_one<256, 16, true>(a, threads, 0, cps, tiles, st, grid);
    const cudaError_t e = cudaStreamSynchronize(st);
    ktau_dfree(g, gbytes);
    if (s == KTAU_OK && e != cudaSuccess) s = ktau_cuda_fail(e, "cudaStreamSynchronize");
    return s;
  }
  const size_t smem = (a.stage ? stage_bytes : 0) + (size_t)teams * team_bytes;
  if (cta_team)
    return items == 16 ? launch_one<256, 16>(a, threads, smem, cps, tiles, st)
                       : launch_one<256, 8>(a, threads, smem, cps, tiles, st);
  switch (items) {
    case 1: return launch_one<32, 1>(a, threads, smem, cps, tiles, st);
    case 2: return launch_one<32, 2>(a, threads, smem, cps, tiles, st);
    case 3: return launch_one<32, 3>(a, threads, smem, cps, tiles, st);
    case 4: return launch_one<32, 4>(a, threads, smem, cps, tiles, st);
    case 5: return launch_one<32, 5>(a, threads, smem, cps, tiles, st);
    case 6: return launch_one<32, 6>(a, threads, smem, cps, tiles, st);
    case 7: return launch_one<32, 7>(a, threads, smem, cps, tiles, st);
    default: return launch_one<32, 8>(a, threads, smem, cps, tiles, st);
  }
}

ktau_status ktau_launch_merge(const ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                              const ktau_out& out, const ktau_merge_plan& plan, cudaStream_t st) {
  if (p_end <= p_begin) return KTAU_OK;
  return launch_merge_impl(R, R, 0, p_begin, p_end, 0, out, plan, st);
}

ktau_status ktau_launch_merge_rect(const ktau_ranked* Q, const ktau_ranked* D, int64_t ldo,
                                   const ktau_out& out, const ktau_merge_plan& plan,
                                   cudaStream_t st) {
  return launch_merge_impl(Q, D, 1, 0, 0, ldo, out, plan, st);
}
