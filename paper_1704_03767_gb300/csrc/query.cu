// Query form (Sec. 1: query-based co-expression search): exact tau-b of every query profile
// against every database variable, plus the k database rows with the largest |tau-b| per query.
//
// Counts come from the rectangular sign contraction (n <= 1024) or the rectangular merge path;
// the top-k kernel then orders each query's row exactly:
//   |tau| = |S| / sqrt(D_u D_v) with D_u fixed per query, so the order is that of S^2 / D_v.
//   key(v) = floor(S^2 2^f / D_v) + 1 (0 for NaN, i.e. D_v = 0) is monotone in that rational;
//   f is the largest shift that keeps S^2 2^f below 2^62. When 2^f > n_0^2, distinct rationals
//   (which differ by at least 1 / (D_v D_v') >= 1 / n_0^2) get distinct keys, so equal keys are
//   exact ties (broken by the smaller row index); otherwise equal keys at the selection boundary
//   are ordered by exact 128-bit cross-multiplication S_a^2 D_b vs S_b^2 D_a.
//   A radix select over the 64-bit keys (8 passes of 8 bits over keys cached in shared memory)
//   finds the k-th largest key of a chunk of up to 4096 rows, one CTA per (query, chunk); each
//   chunk's top-k rows become the candidates of the next pass, until one CTA per query selects
//   among all of them. The selected rows are sorted (bitonic) with the exact comparator, and tau
//   is formed by the shared epilogue (bit-identical to the pair output).
#include <algorithm>
#include <mutex>

#include "ktau_impl.cuh"
#include "signgemm.cuh"

namespace {

constexpr int TK_THREADS = 512;
constexpr int TK_MAXK = 1024;
constexpr int TK_EQCAP = 2048;  // boundary ties collected for the exact comparator

struct TopkArgs {
  const void* S;  // [b][ldS], int32 or int64
  int s64;
  int64_t ldS;
  int64_t m_db, n0;
  const int64_t* Tdb;
  const int64_t* Tq;
  const double* rs_db;
  const double* rs_q;
  int k;
  int shift;      // f
  int injective;  // 2^f > n0^2
  int32_t* idx_out;
  double* tau_out;
  unsigned int* status;  // set to 1 when the boundary group exceeded TK_EQCAP
};

__device__ __forceinline__ long long load_S(const TopkArgs& a, int64_t q, int64_t j) {
  return a.s64 ? ((const long long*)a.S)[q * a.ldS + j] : (long long)((const int*)a.S)[q * a.ldS + j];
}

__device__ __forceinline__ unsigned long long topk_key(const TopkArgs& a, long long S, int64_t Dv,
                                                       bool qnan) {
  if (qnan || Dv == 0) return 0ull;
  const unsigned long long s2 = (unsigned long long)(S < 0 ? -S : S);
  return ((s2 * s2) << a.shift) / (unsigned long long)Dv + 1ull;
}

// a before b in the final order? (exact |tau| descending, NaN last, then smaller index)
struct Cand {
  int S;  // |S| <= n_0 < 2^27
  int D;  // D_v, 0 = NaN
  int j;
};
__device__ __forceinline__ bool cand_before(const Cand& x, const Cand& y) {
  if ((x.D == 0) != (y.D == 0)) return y.D == 0;
  if (x.D != 0) {
    const unsigned long long sx = (unsigned long long)(x.S < 0 ? -x.S : x.S);
    const unsigned long long sy = (unsigned long long)(y.S < 0 ? -y.S : y.S);
    const unsigned long long ax = sx * sx, ay = sy * sy;  // < 2^54
    // compare ax * y.D vs ay * x.D in 128 bits
    const unsigned long long lx = ax * (unsigned long long)y.D, hx = __umul64hi(ax, (unsigned long long)y.D);
    const unsigned long long ly = ay * (unsigned long long)x.D, hy = __umul64hi(ay, (unsigned long long)x.D);
    if (hx != hy) return hx > hy;
    if (lx != ly) return lx > ly;
  }
  return x.j < y.j;
}

// One CTA selects among at most TK_CHUNK items of one query: items [c * TK_CHUNK, ...) of the
// query's list, where item i is database row i (LIST false: the whole database) or row
// in[q * N + i] (LIST: the candidates of an earlier pass, in increasing row order). It finds the
// top kk = min(k, count) items under the exact order; FINAL writes them in that order with tau,
// otherwise their rows, in increasing row order, go to out[q * nout + c * k ..]. The global top-k
// is inside the union of every chunk's top-k, so passes of chunks reduce the candidates until one
// CTA per query holds them all.
constexpr int TK_CHUNK = 4096;

template <bool LIST, bool FINAL>
__global__ void __launch_bounds__(TK_THREADS) topk_kernel(const TopkArgs a,
                                                          const int32_t* __restrict__ in,
                                                          int64_t N, int32_t* __restrict__ out,
                                                          int64_t nout) {
  extern __shared__ unsigned long long skey[];  // [TK_CHUNK] keys of this CTA's items
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long s_prefix;
  __shared__ int s_remaining, s_cnt, s_eqcnt, s_wsum[TK_THREADS / 32];
  __shared__ Cand sel[TK_MAXK];
  __shared__ Cand eq[TK_EQCAP];
  const int64_t q = blockIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * TK_CHUNK;
  const int cnt = (int)min((int64_t)TK_CHUNK, N - i0);
  const int kk = min(a.k, cnt);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool qnan = a.Tq[q] == a.n0;  // constant query variable: every tau is NaN
  auto row_of = [&](int i) -> int64_t {
    return LIST ? (int64_t)in[q * N + i0 + i] : i0 + i;
  };
  __shared__ unsigned long long s_or;
  if (tid == 0) {
    s_prefix = 0ull;
    s_remaining = kk;
    s_cnt = 0;
    s_eqcnt = 0;
    s_or = 0ull;
  }
  __syncthreads();
  // Keys once (the radix passes read them from shared memory), and the OR of all of them: the
  // digits above its highest set bit are 0 in every key, so the passes start below them.
  unsigned long long any = 0ull;
  for (int i = tid; i < cnt; i += blockDim.x) {
    const int64_t j = row_of(i);
    const unsigned long long key = topk_key(a, load_S(a, q, j), a.n0 - a.Tdb[j], qnan);
    skey[i] = key;
    any |= key;
  }
  for (int d = 16; d > 0; d >>= 1) any |= __shfl_xor_sync(0xffffffffu, any, d);
  if (lane == 0 && any) atomicOr(&s_or, any);
  __syncthreads();
  const int top_pass = s_or ? (63 - __clzll((long long)s_or)) / 8 : 0;
  // Radix select of the kk-th largest key, most significant digit first.
  for (int pass = top_pass; pass >= 0; --pass) {
    for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const unsigned long long prefix = s_prefix;
    const unsigned long long hmask = pass == 7 ? 0ull : (~0ull << (8 * (pass + 1)));
    if (pass == top_pass) {
      // The top digit is shared by most keys: lanes with the same digit add once.
      for (int base = 0; base < cnt; base += blockDim.x) {
        const int i = base + tid;
        const unsigned bin = i < cnt ? (unsigned)((skey[i] >> (8 * pass)) & 255u) : 256u + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        if (i < cnt && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned)__popc(peers));
      }
    } else {
      for (int i = tid; i < cnt; i += blockDim.x) {
        const unsigned long long key = skey[i];
        if ((key & hmask) == prefix) atomicAdd(&hist[(key >> (8 * pass)) & 255u], 1u);
      }
    }
    __syncthreads();
    if (warp == 0) {
      // The digit d: the largest with (count of digits >= d) >= remaining. Lane l holds digits
      // 8l .. 8l + 7; a suffix sum over the lanes finds the lane that holds d.
      const int rem0 = s_remaining;
      unsigned c[8];
      unsigned tot = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        c[e] = hist[8 * lane + e];
        tot += c[e];
      }
      unsigned suf = tot;  // digits of this lane and every higher one
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned v = __shfl_down_sync(0xffffffffu, suf, d);
        if (lane + d < 32) suf += v;
      }
      const unsigned above = suf - tot;
      if ((int)above < rem0 && ((int)suf >= rem0 || lane == 0)) {
        int rem = rem0 - (int)above;
        int e = 7;
        for (; e > 0; --e) {
          if ((int)c[e] >= rem) break;
          rem -= (int)c[e];
        }
        s_remaining = rem;
        s_prefix = prefix | ((unsigned long long)(8 * lane + e) << (8 * pass));
      }
    }
    __syncthreads();
  }
  const unsigned long long t = s_prefix;
  const int need_eq = s_remaining;  // how many items with key == t are selected
  // Items with key > t are all selected; items with key == t: the lowest rows when keys are
  // exact (items are in increasing row order), otherwise all of them go through the exact
  // comparator.
  // An exact-key candidate pass writes its selection in item order straight from this scan (the
  // selected items before item i: the greater keys before it, plus its rank among equal keys,
  // up to need_eq), without collecting and sorting.
  const bool direct = !FINAL && a.injective;
  int eq_before = 0, gt_before = 0;
  for (int base = 0; base < cnt; base += blockDim.x) {
    const int i = base + tid;
    long long S = 0, Dv = 0;
    int64_t j = 0;
    unsigned long long key = 0;
    if (i < cnt) {
      key = skey[i];
      j = row_of(i);
    }
    const bool gt = i < cnt && key > t;
    const bool eqf = i < cnt && key == t;
    if (gt || eqf) {
      S = load_S(a, q, j);
      Dv = a.n0 - a.Tdb[j];
    }
    if (gt && !direct) {
      const int pos = atomicAdd(&s_cnt, 1);
      sel[pos] = Cand{(int)S, qnan ? 0 : (int)Dv, (int)j};
    }
    // ordered ranks among equal keys (low 16 bits) and among greater keys (high 16 bits):
    // block-wide exclusive scan in item order
    const int own = (eqf ? 1 : 0) + (gt ? 1 << 16 : 0);
    int incl = own;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += s_wsum[w];
    const int excl = before + incl - own;
    const int rank_eq = eq_before + (excl & 0xffff);
    if (direct) {
      if (gt || (eqf && rank_eq < need_eq))
        out[q * nout + (int64_t)blockIdx.y * a.k + gt_before + (excl >> 16) + min(rank_eq, need_eq)] =
            (int32_t)j;
    } else if (eqf) {
      if (a.injective) {
        if (rank_eq < need_eq) sel[kk - need_eq + rank_eq] = Cand{(int)S, qnan ? 0 : (int)Dv, (int)j};
      } else if (rank_eq < TK_EQCAP) {
        eq[rank_eq] = Cand{(int)S, qnan ? 0 : (int)Dv, (int)j};
      }
    }
    int tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_wsum[w];
    eq_before += tot & 0xffff;
    gt_before += tot >> 16;
    __syncthreads();
  }
  if (direct) return;
  if (!a.injective) {
    // exact order of the boundary group, keep the first need_eq
    const int g = min(eq_before, TK_EQCAP);
    if (eq_before > TK_EQCAP && tid == 0) atomicExch(a.status, 1u);
    int p2 = 1;
    while (p2 < g) p2 <<= 1;
    for (int i = g + tid; i < p2 && i < TK_EQCAP; i += blockDim.x) eq[i] = Cand{0, 0, 0x7fffffff};
    __syncthreads();
    for (int k2 = 2; k2 <= p2; k2 <<= 1)
      for (int jj = k2 >> 1; jj > 0; jj >>= 1) {
        for (int i = tid; i < p2; i += blockDim.x) {
          const int l = i ^ jj;
          if (l > i) {
            const bool up = (i & k2) == 0;
            const bool sw = up ? cand_before(eq[l], eq[i]) : cand_before(eq[i], eq[l]);
            if (sw) {
              const Cand tmp = eq[i];
              eq[i] = eq[l];
              eq[l] = tmp;
            }
          }
        }
        __syncthreads();
      }
    for (int i = tid; i < need_eq; i += blockDim.x) sel[kk - need_eq + i] = eq[i];
  }
  __syncthreads();
  // Order of the kk selected items: the exact order (final pass) or increasing row.
  int p2 = 1;
  while (p2 < kk) p2 <<= 1;
  for (int i = kk + tid; i < p2; i += blockDim.x) sel[i] = Cand{0, 0, 0x7fffffff};
  __syncthreads();
  for (int k2 = 2; k2 <= p2; k2 <<= 1)
    for (int jj = k2 >> 1; jj > 0; jj >>= 1) {
      for (int i = tid; i < p2; i += blockDim.x) {
        const int l = i ^ jj;
        if (l > i) {
          const bool up = (i & k2) == 0;
          const bool sw = FINAL ? (up ? cand_before(sel[l], sel[i]) : cand_before(sel[i], sel[l]))
                                : (up ? sel[l].j < sel[i].j : sel[i].j < sel[l].j);
          if (sw) {
            const Cand tmp = sel[i];
            sel[i] = sel[l];
            sel[l] = tmp;
          }
        }
      }
      __syncthreads();
    }
  if (FINAL) {
    for (int i = tid; i < kk; i += blockDim.x) {
      const Cand c = sel[i];
      a.idx_out[q * a.k + i] = c.j;
      a.tau_out[q * a.k + i] = ktau_tau64(c.S, a.rs_q[q], a.rs_db[c.j]);
    }
  } else {
    for (int i = tid; i < kk; i += blockDim.x)
      out[q * nout + (int64_t)blockIdx.y * a.k + i] = sel[i].j;
  }
}

__device__ unsigned int g_topk_status;

}  // namespace

ktau_status ktau_check_counts(int64_t n, int count_bits);
ktau_status ktau_check_options(const ktau_options* opt);
int ktau_choose_path(const ktau_ranked* R, const ktau_options* opt);

static size_t scratch_S_bytes(const ktau_ranked* db, int64_t b) {
  return ((size_t)b * db->m * sizeof(int) + 255) & ~(size_t)255;
}

extern "C" ktau_status ktau_query_scratch_bytes(const ktau_ranked* db, int64_t b, int32_t k,
                                                size_t* bytes) {
  if (!db || !bytes || b < 0) return ktau_fail(KTAU_EINVAL, "bad argument");
  *bytes = k > 0 ? scratch_S_bytes(db, b) : 0;
  if (ktau_signgemm_supported(db->n)) *bytes += (size_t)b * ((db->n * (db->n - 1) / 2 + 127) / 128 * 128);
  return KTAU_OK;
}

// Shared by ktau_query and its caller-scratch variant: counts for every (query, row) into `out`
// (S may be the scratch buffer), then the top-k when k > 0.
ktau_status ktau_query_run(const ktau_ranked* db, const ktau_ranked* queries, const ktau_out& out,
                           int32_t k, int32_t* topk_idx, double* topk_tau, const ktau_options* opt,
                           cudaStream_t st) {
  ktau_ranked* Q = const_cast<ktau_ranked*>(queries);
  ktau_ranked* D = const_cast<ktau_ranked*>(db);
  const int path = ktau_choose_path(db, opt);
  ktau_status s;
  // n_3 of the rectangular contraction comes from the tie-list tile kernel (n <= 3000).
  if (path == KTAU_PATH_SIGNGEMM && ktau_signgemm_supported(db->n) &&
      (!out.n3 || db->n <= KTAU_SIGNGEMM_TIES_MAX_N)) {
    s = ktau_signgemm_rect(Q, D, out, db->m, ktau_sign_obits(db->n, opt), st);
  } else {
    ktau_merge_plan plan;
    ktau_merge_default_plan(db->n, &plan);
    // one warp per pair; one CTA per pair (merge buffers in global scratch) for rows too long
    // for a warp's shared-memory buffers
    plan.mapping = db->n > KTAU_RANK_CHUNK ? 2 : 1;
    if (opt && opt->tile_q) plan.tile_q = opt->tile_q;
    s = ktau_launch_merge_rect(Q, D, db->m, out, plan, st);
  }
  if (s != KTAU_OK || k == 0) return s;
  TopkArgs a;
  a.S = out.S;
  a.s64 = out.count_bits == 64;
  a.ldS = db->m;
  a.m_db = db->m;
  a.n0 = db->n * (db->n - 1) / 2;
  a.Tdb = db->T;
  a.Tq = queries->T;
  a.rs_db = db->rs64;
  a.rs_q = queries->rs64;
  a.k = k;
  int bits = 0;
  const unsigned long long s2max = (unsigned long long)a.n0 * (unsigned long long)a.n0;
  while (bits < 64 && (s2max >> bits)) ++bits;
  a.shift = std::max(0, 62 - bits);
  a.injective = a.shift >= bits ? 1 : 0;  // 2^f >= 2^bits > n0^2
  a.idx_out = topk_idx;
  a.tau_out = topk_tau;
  unsigned int* st_ptr = nullptr;
  KTAU_CUDA(cudaGetSymbolAddress((void**)&st_ptr, g_topk_status));
  a.status = st_ptr;
  // Passes of chunks of TK_CHUNK items, one CTA per (query, chunk), each keeping its chunk's
  // top-k, until one chunk per query holds every candidate; then the final pass. Candidate lists
  // live in stream-ordered allocations (no synchronisation, safe across streams) from a pool of
  // the library's own that keeps its memory once reserved: with the default pool's release
  // threshold of zero, every stream synchronisation would hand the memory back to the system and
  // the next call would map it again.
  const size_t dyn = (size_t)TK_CHUNK * sizeof(unsigned long long);
  const int64_t b = queries->m;
  if (b > 0x7fffffffLL) return ktau_fail(KTAU_ETOOLARGE, "too many queries in one call");
  cudaMemPool_t pool = nullptr;
  {
    // the kernels' shared-memory limit and the scratch pool, once per device
    static std::mutex mu;
    static bool done[64] = {};
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    KTAU_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return ktau_fail(KTAU_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      KTAU_CUDA(cudaMemPoolCreate(&pools[dev], &props));
      uint64_t keep = ~0ull;
      KTAU_CUDA(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    pool = pools[dev];
    if (!done[dev]) {
      KTAU_CUDA(cudaFuncSetAttribute(topk_kernel<false, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
      KTAU_CUDA(cudaFuncSetAttribute(topk_kernel<true, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
      KTAU_CUDA(cudaFuncSetAttribute(topk_kernel<false, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
      KTAU_CUDA(cudaFuncSetAttribute(topk_kernel<true, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
      done[dev] = true;
    }
  }
  int64_t N = db->m;
  bool list = false;
  const int32_t* in = nullptr;
  int32_t* buf[2] = {nullptr, nullptr};
  ktau_status ts = KTAU_OK;
  for (int w = 0; N > TK_CHUNK; w ^= 1) {
    const int64_t C = (N + TK_CHUNK - 1) / TK_CHUNK;
    const int64_t nout = (C - 1) * k + std::min<int64_t>(k, N - (C - 1) * TK_CHUNK);
    if (C > 65535) {
      ts = ktau_fail(KTAU_ETOOLARGE, "database too large for the top-k passes");
      break;
    }
    if (!buf[w]) {
      const cudaError_t e = cudaMallocFromPoolAsync((void**)&buf[w],
                                                    (size_t)b * nout * sizeof(int32_t), pool, st);
      if (e != cudaSuccess) {
        buf[w] = nullptr;
        ts = ktau_cuda_fail(e, "cudaMallocFromPoolAsync(top-k candidates)");
        break;
      }
    }
    {
      KTAU_TRACE("topk_kernel", st);
      const dim3 grid((unsigned)b, (unsigned)C);
      if (list)
        topk_kernel<true, false><<<grid, TK_THREADS, dyn, st>>>(a, in, N, buf[w], nout);
      else
        topk_kernel<false, false><<<grid, TK_THREADS, dyn, st>>>(a, in, N, buf[w], nout);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      ts = ktau_cuda_fail(e, "topk_kernel");
      break;
    }
    in = buf[w];
    N = nout;
    list = true;
  }
  if (ts == KTAU_OK) {
    KTAU_TRACE("topk_kernel", st);
    const dim3 grid((unsigned)b, 1u);
    if (list)
      topk_kernel<true, true><<<grid, TK_THREADS, dyn, st>>>(a, in, N, nullptr, 0);
    else
      topk_kernel<false, true><<<grid, TK_THREADS, dyn, st>>>(a, in, N, nullptr, 0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) ts = ktau_cuda_fail(e, "topk_kernel");
  }
  for (int w = 0; w < 2; ++w)
    if (buf[w]) cudaFreeAsync(buf[w], st);
  return ts;
}

ktau_status ktau_query_validate(const ktau_ranked* db, const ktau_ranked* queries, int32_t count_bits,
                                int32_t k, int32_t* topk_idx, double* topk_tau,
                                const ktau_options* opt) {
  if (!db || !queries) return ktau_fail(KTAU_EINVAL, "handle is NULL");
  // The exact top-k compares S^2 / D_v in 64- and 128-bit integers, which holds n_0^2 for
  // n <= 65535 only.
  if (db->n > KTAU_NARROW_MAX_N)
    return ktau_fail(KTAU_ETOOLARGE, "the query form takes n <= %d", KTAU_NARROW_MAX_N);
  if (db->n != queries->n)
    return ktau_fail(KTAU_EINVAL, "queries have n=%lld samples, database n=%lld",
                     (long long)queries->n, (long long)db->n);
  ktau_status s = ktau_check_counts(db->n, count_bits);
  if (s != KTAU_OK) return s;
  if ((s = ktau_check_options(opt)) != KTAU_OK) return s;
  if ((s = ktau_ranked_stats(db)) != KTAU_OK || (s = ktau_ranked_stats(queries)) != KTAU_OK)
    return s;
  if (opt && opt->statistic != 0) return ktau_fail(KTAU_EINVAL, "the query form computes tau-b");
  if (opt && opt->path == KTAU_PATH_BITS)
    return ktau_fail(KTAU_EINVAL, "the bit-parallel path counts the triangle of one matrix only");
  if (k < 0 || k > TK_MAXK || k > db->m)
    return ktau_fail(KTAU_EINVAL, "k must be in [0, min(m_db, %d)]", TK_MAXK);
  if (k > 0 && (!topk_idx || !topk_tau)) return ktau_fail(KTAU_EINVAL, "top-k outputs are NULL");
  return KTAU_OK;
}

extern "C" ktau_status ktau_query(const ktau_ranked* db, const ktau_ranked* queries, double* tau,
                                  void* S, void* n3, int32_t count_bits, int32_t k,
                                  int32_t* topk_idx, double* topk_tau, const ktau_options* opt,
                                  void* stream) {
  ktau_status s = ktau_query_validate(db, queries, count_bits, k, topk_idx, topk_tau, opt);
  if (s != KTAU_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  ktau_out out{tau, nullptr, S, n3, count_bits};
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  if (k > 0 && !S) {
    // The top-k needs S: library scratch (cached), released to the cache when the work is done.
    scratch_bytes = scratch_S_bytes(db, queries->m);
    if ((s = ktau_dmalloc(&scratch, scratch_bytes)) != KTAU_OK) return s;
    out.S = scratch;
    out.count_bits = 32;
  }
  s = ktau_query_run(db, queries, out, k, topk_idx, topk_tau, opt, st);
  if (scratch) {
    cudaStreamSynchronize(st);
    ktau_dfree(scratch, scratch_bytes);
  }
  return s;
}

// Reports (and clears) a top-k boundary group that exceeded the exact-comparator capacity.
ktau_status ktau_query_check_status(cudaStream_t st) {
  unsigned int e = 0;
  KTAU_CUDA(cudaMemcpyFromSymbolAsync(&e, g_topk_status, sizeof(e), 0, cudaMemcpyDeviceToHost, st));
  KTAU_CUDA(cudaStreamSynchronize(st));
  if (e) {
    const unsigned int zero = 0;
    cudaMemcpyToSymbolAsync(g_topk_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
    return ktau_fail(KTAU_ETOOLARGE, "top-k: more than %d rows tied at the selection boundary",
                     TK_EQCAP);
  }
  return KTAU_OK;
}
