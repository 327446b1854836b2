// Bit-parallel dominance count: a third pair path for short rows (n <= KTAU_BITS_MAX_N), the sign
// form of Algorithm 1 (Sec. 3.1) evaluated 32 sample pairs per logic instruction.
//
// For every variable and every sample a, two n-bit masks are built once from the dense ranks r:
//   G[a] = {b : r[b] > r[a]}   and   L[a] = {b : r[b] < r[a]}.
// For a pair (u, v) and a fixed a, the sum over b of sign(u_b - u_a) * sign(v_b - v_a) is
//   |G_u n G_v| + |L_u n L_v| - |G_u n L_v| - |L_u n G_v|
//   = pop((G_u & G_v) | (L_u & L_v)) - pop((G_u & L_v) | (L_u & G_v))
// (each union joins disjoint sets). Summed over a it counts every unordered sample pair twice, so
// S = n_c - n_d is half the total. Joint ties (Table 1's n_3): the samples tied with a in u are
// E_u[a] = not(G_u[a] or L_u[a]) without a itself, and n_3 = (sum over a of |E_u[a] n E_v[a]|) / 2.
// All counts are exact integers; tau-b is formed by the same epilogue as the other paths.
//
// Masks: variable v at bits + v * stride (stride = 2 n W words rounded up to 4, so every variable
// starts on 16 bytes), W = ceil(n / 32) words per mask, word w of G[a] at w * n + a and of L[a] at
// (W + w) * n + a: the lanes of a warp (consecutive samples a) read consecutive words, free of
// shared-memory bank conflicts. Built by one warp per variable with ballots. Pairs: persistent CTAs walk the upper triangle in TQ x TQ
// tiles through the job-id bijection (Eq. 13-14), stage the tile's row and column masks in shared
// memory, and give one pair to one warp (lane l takes samples l, l + 32, ...).
#include <algorithm>

#include "ktau_impl.cuh"

namespace {

constexpr int kBitsThreads = 256;

// Masks of `m` variables (ranks rank[v * ld + b]) into bits; one warp per variable.
__global__ void __launch_bounds__(256) bits_masks_kernel(const uint16_t* __restrict__ rank,
                                                         int64_t ld, int n, int64_t m,
                                                         int64_t stride,
                                                         uint32_t* __restrict__ bits) {
  const int lane = threadIdx.x & 31;
  const int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (v >= m) return;  // whole warps leave together
  const int W = (n + 31) >> 5;
  const uint16_t* r = rank + v * ld;
  uint32_t mine[KTAU_BITS_MAX_N / 32];  // r[32 w + lane], or the largest value past n
#pragma unroll
  for (int w = 0; w < KTAU_BITS_MAX_N / 32; ++w) {
    const int b = 32 * w + lane;
    mine[w] = (w < W && b < n) ? (uint32_t)r[b] : 0xffffffffu;
  }
  uint32_t* out = bits + (size_t)v * stride;
  for (int a = 0; a < n; ++a) {
    const uint32_t ra = r[a];
#pragma unroll
    for (int w = 0; w < KTAU_BITS_MAX_N / 32; ++w) {
      if (w >= W) break;
      const bool valid = 32 * w + lane < n;
      const uint32_t g = __ballot_sync(0xffffffffu, valid && mine[w] > ra);
      const uint32_t l = __ballot_sync(0xffffffffu, valid && mine[w] < ra);
      if (lane == 0) {
        out[(size_t)w * n + a] = g;
        out[(size_t)(W + w) * n + a] = l;
      }
    }
  }
}

// Counts of one pair from the masks of u (mu) and v (mv) in shared memory; every lane returns
// the warp totals of 2 S and 2 n_3.
template <int W, bool N3>
__device__ __forceinline__ void bits_pair(const uint32_t* mu, const uint32_t* mv, int n, int lane,
                                          long long& s2, long long& t2) {
  int acc = 0, tie = 0;
  for (int a = lane; a < n; a += 32) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t Gu = mu[w * n + a], Lu = mu[(W + w) * n + a];
      const uint32_t Gv = mv[w * n + a], Lv = mv[(W + w) * n + a];
      acc += __popc((Gu & Gv) | (Lu & Lv)) - __popc((Gu & Lv) | (Lu & Gv));
      if (N3) {
        // tied with a in both, a itself and positions past n excluded
        uint32_t valid = 32 * w + 32 <= n ? 0xffffffffu : ((1u << (n - 32 * w)) - 1u);
        if ((a >> 5) == w) valid &= ~(1u << (a & 31));
        tie += __popc(~(Gu | Lu) & ~(Gv | Lv) & valid);
      }
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if (N3) tie += __shfl_xor_sync(0xffffffffu, tie, d);
  }
  s2 = acc;
  t2 = tie;
}

struct BitsArgs {
  const uint32_t* bits;
  int64_t stride;    // words per variable (a multiple of 4)
  ktau_fac fac;
  int64_t m;
  int n;
  int tq;            // tile side
  int64_t w;         // tiles per side
  int64_t tile_lo, tile_hi;
  uint64_t p_begin, p_end;
  ktau_out out;
};

template <int W, bool N3>
__global__ void __launch_bounds__(kBitsThreads) bits_pairs_kernel(const BitsArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int n = a.n, tq = a.tq;
  const size_t per_var = (size_t)a.stride;  // words of one variable's masks
  uint32_t* srow = sm;
  uint32_t* scol = sm + (size_t)tq * per_var;
  const int64_t n0 = (int64_t)n * (n - 1) / 2;
  for (int64_t t = a.tile_lo + blockIdx.x; t < a.tile_hi; t += gridDim.x) {
    int64_t yq, xq;
    ktau_tile_coord(a.w, t, yq, xq);
    const int64_t y0 = yq * tq, x0 = xq * tq;
    __syncthreads();  // the previous tile's masks are no longer read
    // stage the tile's rows and columns (variables past m are left unstaged and never read)
    const int64_t ny = min((int64_t)tq, a.m - y0), nx = min((int64_t)tq, a.m - x0);
    const uint4* gy = reinterpret_cast<const uint4*>(a.bits + (size_t)y0 * per_var);
    const uint4* gx = reinterpret_cast<const uint4*>(a.bits + (size_t)x0 * per_var);
    uint4* sy = reinterpret_cast<uint4*>(srow);
    uint4* sx = reinterpret_cast<uint4*>(scol);
    const size_t vy = (size_t)ny * per_var / 4, vx = (size_t)nx * per_var / 4;
    for (size_t i = threadIdx.x; i < vy; i += blockDim.x) sy[i] = __ldg(gy + i);
    for (size_t i = threadIdx.x; i < vx; i += blockDim.x) sx[i] = __ldg(gx + i);
    __syncthreads();
    for (int e = warp; e < tq * tq; e += nw) {
      const int64_t y = y0 + e / tq, x = x0 + e % tq;
      if (y >= a.m || x >= a.m || x <= y) continue;
      const uint64_t p = ktau_pair_index(a.m, y, x);
      if (p < a.p_begin || p >= a.p_end) continue;
      long long s2, t2;
      bits_pair<W, N3>(srow + (size_t)(y - y0) * per_var, scol + (size_t)(x - x0) * per_var, n,
                       lane, s2, t2);
      if (lane == 0) ktau_store(a.out, p - a.p_begin, s2 / 2, t2 / 2, n0, a.fac, y, x);
    }
  }
}

template <int W>
ktau_status launch_bits_w(const BitsArgs& args, size_t smem, int64_t tiles, bool n3,
                          cudaStream_t st) {
  auto kern = n3 ? bits_pairs_kernel<W, true> : bits_pairs_kernel<W, false>;
  KTAU_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  KTAU_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBitsThreads, smem));
  if (occ < 1) return ktau_fail(KTAU_ETOOLARGE, "bit-parallel tile does not fit on an SM");
  int64_t grid = (int64_t)occ * ktau_sm_count();
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  KTAU_TRACE("bits_pairs_kernel", st);
  kern<<<(unsigned)grid, kBitsThreads, smem, st>>>(args);
  KTAU_CUDA(cudaGetLastError());
  return KTAU_OK;
}

}  // namespace

ktau_status ktau_bits_allpairs(ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                               const ktau_out& out, cudaStream_t st) {
  const int64_t m = R->m, n = R->n;
  if (n > KTAU_BITS_MAX_N)
    return ktau_fail(KTAU_EINVAL, "bit-parallel path supports n <= %d", KTAU_BITS_MAX_N);
  const int W = (int)((n + 31) / 32);
  const int64_t stride = ((int64_t)n * 2 * W + 3) / 4 * 4;
  const size_t per_var = (size_t)stride * sizeof(uint32_t);
  if (!R->bits) {  // masks built once per handle, on the first call of this path
    R->bits_bytes = (size_t)m * per_var;
    void* p = nullptr;
    if (ktau_dmalloc(&p, R->bits_bytes) != KTAU_OK) return KTAU_ENOMEM;
    R->bits = (uint32_t*)p;
    const int64_t blocks = (m * 32 + 255) / 256;
    if (blocks > 0x7fffffffLL) return ktau_fail(KTAU_ETOOLARGE, "too many variables");
    KTAU_TRACE("bits_masks_kernel", st);
    bits_masks_kernel<<<(unsigned)blocks, 256, 0, st>>>(R->rank, R->ld, (int)n, m, stride,
                                                         R->bits);
    KTAU_CUDA(cudaGetLastError());
  }
  // tile side: the tile's row and column masks fill at most ~200 KB of shared memory
  int tq = (int)std::min<size_t>(16, (200 * 1024) / (2 * per_var));
  if (tq < 1) tq = 1;
  BitsArgs a;
  a.bits = R->bits;
  a.stride = stride;
  a.fac = ktau_fac{R->rs64, R->rsff, R->T};
  a.m = m;
  a.n = (int)n;
  a.tq = tq;
  a.w = (m + tq - 1) / tq;
  int64_t i0, j0, i1, j1;
  ktau_tile_coord(m - 1, (int64_t)p_begin, i0, j0);
  ktau_tile_coord(m - 1, (int64_t)(p_end - 1), i1, j1);
  a.tile_lo = ktau_rowstart(a.w, i0 / tq);
  a.tile_hi = ktau_rowstart(a.w, i1 / tq + 1);
  a.p_begin = p_begin;
  a.p_end = p_end;
  a.out = out;
  const size_t smem = (size_t)2 * tq * per_var;
  const int64_t tiles = a.tile_hi - a.tile_lo;
  const bool n3 = out.n3 != nullptr;
  switch (W) {
    case 1: return launch_bits_w<1>(a, smem, tiles, n3, st);
    case 2: return launch_bits_w<2>(a, smem, tiles, n3, st);
    case 3: return launch_bits_w<3>(a, smem, tiles, n3, st);
    case 4: return launch_bits_w<4>(a, smem, tiles, n3, st);
    case 5: return launch_bits_w<5>(a, smem, tiles, n3, st);
    case 6: return launch_bits_w<6>(a, smem, tiles, n3, st);
    case 7: return launch_bits_w<7>(a, smem, tiles, n3, st);
    default: return launch_bits_w<8>(a, smem, tiles, n3, st);
  }
}

void ktau_bits_release(ktau_ranked* R) {
  ktau_dfree(R->bits, R->bits_bytes);
  R->bits = nullptr;
}
