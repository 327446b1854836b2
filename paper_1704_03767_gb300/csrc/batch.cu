// Batched form: many independent matrices of uneven m and n in one persistent launch per
// kernel family, capturable in a CUDA graph (generalises the tile/pass scheduling of
// Sec. 4.2-4.3 from one job matrix to a list of job matrices).
//
// Plan (ktau_batch_create): every dataset gets a path (its descriptor, the options, or the
// built-in crossover by n); datasets are laid out in one library-owned workspace grouped by path
// (see GroupKind) so each group's variables are consecutive rows. Per group: a descriptor table in device memory and prefix sums of rows,
// tiles and units. Contraction groups stack their sign expansions into one operand tensor (one
// TMA descriptor per group, each dataset using only its own K blocks).
//
// Run (ktau_batch_run): per group, on the group's lane: rank kernel over the group's rows; per
// contraction group: sign expansion, tie lists, contraction, joint ties; one launch per merge group.
// Nothing is allocated and nothing waits on the host, so the sequence can be graph-captured.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ktau_impl.cuh"
#include "signgemm.cuh"

namespace {

constexpr int kMergeTq = 16;

// Group kinds: contraction groups (one per operand type and stride class, stride = operand bytes
// of a row rounded up to a power of two, so stacking wastes at most half of the operand memory),
// merge with one warp per pair (n <= 1024), merge with one CTA per pair (n > 1024).
enum GroupKind { kContract = 0, kMergeWarp = 1, kMergeCta = 2 };

struct GroupPlan {
  int kind = kContract;
  int64_t key = 0;           // contraction: (operand bits / 4) * 64 + log2(stride)
  std::vector<int32_t> ids;  // indices into the workspace-ordered descriptor table
  int32_t* d_ids = nullptr;
  int64_t* d_row_prefix = nullptr;
  int64_t* d_unit_prefix = nullptr;
  int64_t* d_jt_prefix = nullptr;
  int64_t* d_tile_prefix = nullptr;  // merge group
  int64_t* d_blk_prefix = nullptr;   // contraction group: sign-expansion blocks per dataset
  int64_t blocks = 0;
  int64_t row0 = 0, rows = 0, units = 0, jt_tiles = 0, tiles = 0, max_n = 0, stride = 0;
  int esize = 0, obits = 0;
  void* sgn = nullptr;
  alignas(64) unsigned char tmap_b[128];  // row-operand boxes (FP4: 120 rows)
  int64_t* tie_off = nullptr;
  uint32_t* tie_pairs = nullptr;
  int64_t tie_cap = 0;
  alignas(64) unsigned char tmap[128];
};

}  // namespace

struct ktau_batch {
  int count = 0;
  int device = 0;
  std::vector<ktau_bds> hds;  // workspace order
  ktau_bds* d_ds = nullptr;
  int64_t total_rows = 0, max_n = 0;
  uint64_t pairs = 0;
  std::vector<GroupPlan> g;  // in workspace order
  ktau_stats* d_stats = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // Groups run on kLanes streams forked from the caller's stream and joined back at the end, so that groups too small to fill the GPU overlap (every group owns its
  // operands, tie lists and outputs).
  static constexpr int kLanes = 8;
  std::vector<int> lane_of;  // lane of each group: largest groups first, each to the least loaded
  cudaStream_t lane[kLanes] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kLanes] = {};
  // Where device memory comes from: the library's allocator (a plan, ktau_batch_create), a
  // caller's workspace carved front to back (ktau_allpairs_batched), or nowhere (measure: only
  // the sizes are added up, for ktau_workspace_size). In the workspace modes nothing is
  // allocated, no stream is created, every group runs on the caller's stream and the descriptor
  // tables are copied with cudaMemcpyAsync on it.
  enum Source { kLibrary = 0, kWorkspace = 1, kMeasure = 2 };
  int source = kLibrary;
  char* arena = nullptr;
  size_t arena_cap = 0, arena_used = 0;
  cudaStream_t copy_st = nullptr;
};

// Host-to-device copy of a plan table without a memcpy: the bytes travel as the by-value
// parameter of a one-block kernel, 32 KB per launch. Launch parameters are copied when the launch
// is enqueued, so the call neither stages through pinned memory nor waits for the stream, and the
// host buffer may be released as soon as it returns.
constexpr int kUploadChunk = 32736;  // + 16 header bytes stays within the 32764-byte limit
struct UploadChunk {
  unsigned char* dst;
  unsigned int bytes;
  unsigned int pad;
  alignas(16) unsigned char data[kUploadChunk];
};

__global__ void upload_kernel(const __grid_constant__ UploadChunk c) {
  const unsigned full = c.bytes & ~15u;
  if (((uintptr_t)c.dst & 15) == 0) {
    for (unsigned i = threadIdx.x * 16; i < full; i += blockDim.x * 16)
      *reinterpret_cast<uint4*>(c.dst + i) = *reinterpret_cast<const uint4*>(c.data + i);
  } else {
    for (unsigned i = threadIdx.x; i < full; i += blockDim.x) c.dst[i] = c.data[i];
  }
  for (unsigned i = full + threadIdx.x; i < c.bytes; i += blockDim.x) c.dst[i] = c.data[i];
}

static ktau_status upload_by_launch(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  static thread_local UploadChunk* chunk = new UploadChunk();  // 32 KB, kept per host thread
  for (size_t off = 0; off < bytes; off += kUploadChunk) {
    const size_t len = bytes - off < (size_t)kUploadChunk ? bytes - off : (size_t)kUploadChunk;
    chunk->dst = (unsigned char*)dst + off;
    chunk->bytes = (unsigned int)len;
    memcpy(chunk->data, (const unsigned char*)src + off, len);
    upload_kernel<<<1, 256, 0, st>>>(*chunk);
    KTAU_CUDA(cudaGetLastError());
  }
  return KTAU_OK;
}

static ktau_status batch_alloc(ktau_batch* B, void** p, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  if (B->source == ktau_batch::kMeasure) {
    // A stand-in address, 256-byte aligned, that is never dereferenced.
    *p = (void*)((uintptr_t)0x100000 + B->arena_used);
    B->arena_used += bytes;
    return KTAU_OK;
  }
  if (B->source == ktau_batch::kWorkspace) {
    if (B->arena_used + bytes > B->arena_cap)
      return ktau_fail(KTAU_EINVAL, "workspace of %zu bytes is too small (ktau_workspace_size)",
                       B->arena_cap);
    *p = B->arena + B->arena_used;
    B->arena_used += bytes;
    return KTAU_OK;
  }
  ktau_status s = ktau_dmalloc(p, bytes);
  if (s == KTAU_OK) B->allocs.push_back({*p, bytes});
  return s;
}

template <class T>
static ktau_status batch_upload(ktau_batch* B, T** dst, const std::vector<T>& v) {
  ktau_status s = batch_alloc(B, (void**)dst, v.size() * sizeof(T));
  if (s != KTAU_OK || v.empty() || B->source == ktau_batch::kMeasure) return s;
  if (B->source == ktau_batch::kWorkspace)
    return upload_by_launch(*dst, v.data(), v.size() * sizeof(T), B->copy_st);
  else
    KTAU_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return KTAU_OK;
}

static int batch_path_for(const ktau_batch_desc& d, const ktau_options* opt) {
  if (d.path != KTAU_PATH_AUTO) return d.path;
  if (opt && opt->path != KTAU_PATH_AUTO) return opt->path;
  // The contraction wins wherever it applies (autotuner, GB300); its batched n_3 comes from the
  // tie-list tile kernel, which takes n <= KTAU_SIGNGEMM_TIES_MAX_N.
  return d.n <= (d.n3 ? KTAU_SIGNGEMM_TIES_MAX_N : KTAU_SIGNGEMM_MAX_N) ? KTAU_PATH_SIGNGEMM
                                                                        : KTAU_PATH_MERGE;
}

ktau_status ktau_check_counts(int64_t n, int count_bits);
ktau_status ktau_check_options(const ktau_options* opt);

extern "C" ktau_status ktau_batch_free(ktau_batch* B) {
  if (!B) return KTAU_OK;
  if (B->source != ktau_batch::kLibrary) {  // owns no device memory, stream or graph
    delete B;
    return KTAU_OK;
  }
  cudaDeviceSynchronize();
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (int l = 0; l < ktau_batch::kLanes; ++l) {
    if (B->lane[l]) cudaStreamDestroy(B->lane[l]);
    if (B->join[l]) cudaEventDestroy(B->join[l]);
  }
  if (B->fork) cudaEventDestroy(B->fork);
  for (auto& a : B->allocs) ktau_dfree(a.first, a.second);
  delete B;
  return KTAU_OK;
}

static ktau_status batch_build_checked(const ktau_batch_desc* descs, int32_t count,
                                       const ktau_options* opt, ktau_batch* B);

// Validates the descriptors and lays the plan out (B->source says where memory comes from). On
// failure B is released.
static ktau_status batch_build(const ktau_batch_desc* descs, int32_t count,
                               const ktau_options* opt, ktau_batch* B) {
  if (!descs || count <= 0) {
    ktau_batch_free(B);
    return ktau_fail(KTAU_EINVAL, "need count > 0 descriptors");
  }
  ktau_status s = batch_build_checked(descs, count, opt, B);
  if (s != KTAU_OK) ktau_batch_free(B);
  return s;
}

extern "C" ktau_status ktau_batch_create(const ktau_batch_desc* descs, int32_t count,
                                         const ktau_options* opt, ktau_batch** out) {
  if (!out) return ktau_fail(KTAU_EINVAL, "out is NULL");
  *out = nullptr;
  ktau_batch* B = new ktau_batch();
  ktau_status s = batch_build(descs, count, opt, B);
  if (s == KTAU_OK) *out = B;
  return s;
}

static ktau_status batch_build_checked(const ktau_batch_desc* descs, int32_t count,
                                       const ktau_options* opt, ktau_batch* B) {
  ktau_status s = ktau_check_options(opt);
  if (s != KTAU_OK) return s;
  if (opt && opt->statistic != 0) return ktau_fail(KTAU_EINVAL, "the batched form computes tau-b");
  if (opt && opt->path == KTAU_PATH_BITS)
    return ktau_fail(KTAU_EINVAL, "the batched form runs the merge path or the contraction");
  for (int i = 0; i < count; ++i) {
    const ktau_batch_desc& d = descs[i];
    if (!d.values) return ktau_fail(KTAU_EINVAL, "descriptor %d: values is NULL", i);
    if (d.dtype != KTAU_F32 && d.dtype != KTAU_I32)
      return ktau_fail(KTAU_EINVAL, "descriptor %d: bad dtype", i);
    if (d.m < 2 || d.n < 2 || d.ld < d.n)
      return ktau_fail(KTAU_EINVAL, "descriptor %d: need m >= 2, n >= 2, ld >= n", i);
    if (d.n > KTAU_BATCH_MAX_N || d.m > KTAU_MAX_M)
      return ktau_fail(KTAU_ETOOLARGE, "descriptor %d: shape beyond the limits (n <= %d)", i,
                       KTAU_BATCH_MAX_N);
    if ((s = ktau_check_counts(d.n, d.count_bits)) != KTAU_OK) return s;
    if (d.path < 0 || d.path > 2) return ktau_fail(KTAU_EINVAL, "descriptor %d: bad path", i);
    if (d.mapping < 0 || d.mapping > 2)
      return ktau_fail(KTAU_EINVAL, "descriptor %d: bad mapping", i);
    if (batch_path_for(d, opt) == KTAU_PATH_SIGNGEMM &&
        d.n > (d.n3 ? KTAU_SIGNGEMM_TIES_MAX_N : KTAU_SIGNGEMM_MAX_N))
      return ktau_fail(KTAU_EINVAL, "descriptor %d: contraction path needs n <= %d", i,
                       d.n3 ? KTAU_SIGNGEMM_TIES_MAX_N : KTAU_SIGNGEMM_MAX_N);
  }
  B->count = count;
  cudaGetDevice(&B->device);
  // Group of every dataset; workspace order = group order (contraction groups by stride class,
  // then the two merge groups).
  std::vector<int64_t> gkey(count);
  for (int i = 0; i < count; ++i) {
    const ktau_batch_desc& d = descs[i];
    if (batch_path_for(d, opt) == KTAU_PATH_MERGE) {
      const bool cta = d.mapping == 2 || (d.mapping == 0 && d.n > 1024);
      gkey[i] = (int64_t)1 << 40 | (cta ? 1 : 0);
    } else {
      const int ob = ktau_sign_obits(d.n, opt);
      const int64_t bytes = ktau_kpad(d.n * (d.n - 1) / 2, ob) * ob / 8;
      int lg = 6;
      while (((int64_t)1 << lg) < bytes) ++lg;
      gkey[i] = (ob / 4) * 64 + lg;
    }
  }
  std::vector<int64_t> keys(gkey);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  std::vector<int> order;
  std::vector<int> grp(count);
  B->g.resize(keys.size());
  for (size_t gi = 0; gi < keys.size(); ++gi) {
    GroupPlan& G = B->g[gi];
    G.key = keys[gi];
    G.kind = keys[gi] >> 40 ? (keys[gi] & 1 ? kMergeCta : kMergeWarp) : kContract;
    for (int i = 0; i < count; ++i)
      if (gkey[i] == keys[gi]) {
        grp[i] = (int)gi;
        order.push_back(i);
      }
  }

  // Per-dataset workspace sizes.
  std::vector<int64_t> row_prefix(count + 1, 0);
  size_t rank_bytes = 0;
  std::vector<size_t> rank_off(count);
  for (int k = 0; k < count; ++k) {
    const ktau_batch_desc& d = descs[order[k]];
    row_prefix[k + 1] = row_prefix[k] + d.m;
    const int64_t ld = (d.n + 15) & ~15LL;
    rank_off[k] = rank_bytes;
    rank_bytes += (((size_t)d.m * ld * 2 + 255) & ~(size_t)255) * 3;
    B->max_n = std::max<int64_t>(B->max_n, d.n);
    B->pairs += (uint64_t)(d.m * (d.m - 1) / 2);
  }
  B->total_rows = row_prefix[count];
  const int64_t R = B->total_rows;
  char* ws = nullptr;
  if ((s = batch_alloc(B, (void**)&ws, rank_bytes + (size_t)R * 32 + 4096)) != KTAU_OK) {
    return s;
  }
  int64_t* T_all = (int64_t*)(ws + rank_bytes);
  double* rs64_all = (double*)(T_all + R);
  float2* rsff_all = (float2*)(rs64_all + R);
  int32_t* ndist_all = (int32_t*)(rsff_all + R);
  int32_t* maxg_all = ndist_all + R;

  B->hds.resize(count);
  for (int k = 0; k < count; ++k) {
    const ktau_batch_desc& d = descs[order[k]];
    ktau_bds& D = B->hds[k];
    memset(&D, 0, sizeof(D));
    D.values = d.values;
    D.dtype = d.dtype;
    D.count_bits = d.count_bits;
    D.m = d.m;
    D.n = d.n;
    D.ld_in = d.ld;
    D.ld = (d.n + 15) & ~15LL;
    const size_t arr = ((size_t)d.m * D.ld * 2 + 255) & ~(size_t)255;
    D.perm = (uint16_t*)(ws + rank_off[k]);
    D.rank = (uint16_t*)(ws + rank_off[k] + arr);
    D.srank = (uint16_t*)(ws + rank_off[k] + 2 * arr);
    const int64_t r0 = row_prefix[k];
    D.T = T_all + r0;
    D.rs64 = rs64_all + r0;
    D.rsff = rsff_all + r0;
    D.ndist = ndist_all + r0;
    D.maxg = maxg_all + r0;
    D.out = ktau_out{d.tau64, d.tau32, d.S, d.n3, d.count_bits};
    D.path = B->g[grp[order[k]]].kind == kContract ? KTAU_PATH_SIGNGEMM : KTAU_PATH_MERGE;
    B->g[grp[order[k]]].ids.push_back(k);
  }
  // Group plans.
  for (size_t gi = 0; gi < B->g.size(); ++gi) {
    GroupPlan& G = B->g[gi];
    if (G.ids.empty()) continue;
    G.row0 = row_prefix[G.ids.front()];
    std::vector<int64_t> rp(1, 0), up(1, 0), jp(1, 0), tp(1, 0), bp(1, 0);
    int64_t kpad_max = 0;
    for (int k : G.ids) G.max_n = std::max<int64_t>(G.max_n, B->hds[k].n);
    const int erows = ktau_expand_rows(G.max_n);
    for (int k : G.ids) {
      ktau_bds& D = B->hds[k];
      rp.push_back(rp.back() + D.m);
      if (G.kind != kContract) {
        D.tq = G.kind == kMergeWarp ? kMergeTq : 4;
        D.w = (D.m + D.tq - 1) / D.tq;
        tp.push_back(tp.back() + D.w * (D.w + 1) / 2);
      } else {
        const int gobits = (int)(G.key / 64) * 4;
        D.esize = gobits == 16 ? 2 : 1;  // BF16 takes 2 bytes in shared memory
        bp.push_back(bp.back() + (D.m + erows - 1) / erows);
        const int64_t K = D.n * (D.n - 1) / 2;
        const int64_t K_pad = ktau_kpad(K, gobits);
        // stage rows of 128 bytes: 128 FP8 / 64 BF16 elements, or 256 packed FP4 elements
        D.num_kb = gobits == 4 ? K_pad / 256 : K_pad * D.esize / 128;
        kpad_max = std::max(kpad_max, K_pad);
        const int st = ktau_pair_tile(gobits);  // super-tile side of the pair contraction
        D.wS = (D.m + st - 1) / st;
        up.push_back(up.back() + D.wS * (D.wS + 1));
        const int64_t w = (D.m + 255) / 256;
        jp.push_back(jp.back() + w * (w + 1) / 2);
      }
    }
    G.rows = rp.back();
    if ((s = batch_upload(B, &G.d_ids, G.ids)) != KTAU_OK ||
        (s = batch_upload(B, &G.d_row_prefix, rp)) != KTAU_OK) {
      return s;
    }
    if (G.kind != kContract) {
      G.tiles = tp.back();
      if ((s = batch_upload(B, &G.d_tile_prefix, tp)) != KTAU_OK) {
        return s;
      }
      continue;
    }
    G.obits = (int)(G.key / 64) * 4;
    G.esize = G.obits == 16 ? 2 : 1;
    G.units = up.back();
    G.jt_tiles = jp.back();
    G.blocks = bp.back();
    G.stride = kpad_max * G.obits / 8;
    if ((s = batch_upload(B, &G.d_unit_prefix, up)) != KTAU_OK ||
        (s = batch_upload(B, &G.d_blk_prefix, bp)) != KTAU_OK ||
        (s = batch_upload(B, &G.d_jt_prefix, jp)) != KTAU_OK ||
        (s = batch_alloc(B, &G.sgn, (size_t)G.rows * G.stride)) != KTAU_OK ||
        (s = batch_alloc(B, (void**)&G.tie_off, ((size_t)G.rows + 1) * 8)) != KTAU_OK) {
      return s;
    }
    // Tie lists: room for 2n tied pairs per variable on average; variables beyond the capacity
    // are handled from their tie groups directly.
    G.tie_cap = 0;
    for (int k : G.ids) G.tie_cap += B->hds[k].m * 2 * B->hds[k].n;
    if ((s = batch_alloc(B, (void**)&G.tie_pairs, (size_t)G.tie_cap * 4)) != KTAU_OK) {
      return s;
    }
    int64_t srow = 0;
    for (int k : G.ids) {
      ktau_bds& D = B->hds[k];
      D.srow = srow;
      srow += D.m;
      D.tie_off = G.tie_off + (row_prefix[k] - G.row0);
      D.tie_pairs = G.tie_pairs;
      D.tie_cap = G.tie_cap;
    }
    if (B->source != ktau_batch::kMeasure &&
        ((s = ktau_signgemm_make_tmap(G.tmap, G.sgn, G.stride, G.rows, G.obits, 128)) != KTAU_OK ||
         (s = ktau_signgemm_make_tmap(G.tmap_b, G.sgn, G.stride, G.rows, G.obits,
                                      ktau_pair_tile(G.obits) / 2)) != KTAU_OK)) {
      return s;
    }
  }
  if ((s = batch_upload(B, &B->d_ds, B->hds)) != KTAU_OK ||
      (s = batch_alloc(B, (void**)&B->d_stats, sizeof(ktau_stats))) != KTAU_OK) {
    return s;
  }
  if (B->source == ktau_batch::kMeasure) return KTAU_OK;
  if (B->source == ktau_batch::kWorkspace) {
    // Groups run one after another on the caller's stream; the statistics start at zero.
    B->lane_of.assign(B->g.size(), 0);
    KTAU_CUDA(cudaMemsetAsync(B->d_stats, 0, sizeof(ktau_stats), B->copy_st));
    return KTAU_OK;
  }
  KTAU_CUDA(cudaMemset(B->d_stats, 0, sizeof(ktau_stats)));
  cudaError_t e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
  for (int l = 0; l < ktau_batch::kLanes && e == cudaSuccess; ++l) {
    e = cudaStreamCreateWithFlags(&B->lane[l], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join[l], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) return ktau_cuda_fail(e, "batch streams");
  // Lane assignment: work estimate of a group = contraction tiles x K blocks (+ merge tiles x n),
  // largest first to the least loaded lane.
  {
    std::vector<std::pair<double, int>> work;
    for (size_t gi = 0; gi < B->g.size(); ++gi) {
      const GroupPlan& G = B->g[gi];
      double w = 0;
      if (G.kind == kContract)
        w = (double)G.units * (double)G.stride + (double)G.rows * (double)G.stride;
      else
        w = (double)G.tiles * (double)G.max_n * 64.0;
      work.push_back({w, (int)gi});
    }
    std::sort(work.begin(), work.end(), [](const std::pair<double, int>& a,
                                           const std::pair<double, int>& b) { return a.first > b.first; });
    B->lane_of.assign(B->g.size(), 0);
    double load[ktau_batch::kLanes] = {0};
    for (const auto& wi : work) {
      int best = 0;
      for (int l = 1; l < ktau_batch::kLanes; ++l)
        if (load[l] < load[best]) best = l;
      load[best] += wi.first;
      B->lane_of[wi.second] = best;
    }
  }
  return KTAU_OK;
}

extern "C" ktau_status ktau_batch_run(ktau_batch* B, void* stream) {
  if (!B) return ktau_fail(KTAU_EINVAL, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  ktau_status s = KTAU_OK;
  const bool lanes = B->fork != nullptr;  // a plan made by ktau_batch_create
  // fork: every lane starts after the caller's earlier work
  if (lanes) {
    KTAU_CUDA(cudaEventRecord(B->fork, st));
    for (int l = 0; l < ktau_batch::kLanes; ++l)
      KTAU_CUDA(cudaStreamWaitEvent(B->lane[l], B->fork, 0));
  }
  for (size_t gi = 0; gi < B->g.size(); ++gi) {
    GroupPlan& G = B->g[gi];
    if (G.ids.empty() || s != KTAU_OK) continue;
    cudaStream_t ls = lanes ? B->lane[B->lane_of[gi]] : st;
    // Rank transform of the group's own variables on its lane (a group's datasets are consecutive
    // in the descriptor table), so that a lane's counting starts as soon as its own ranks are done.
    s = ktau_launch_batch_rank(B->d_ds + G.ids.front(), (int)G.ids.size(), G.d_row_prefix, G.rows,
                               G.max_n, B->d_stats, ls);
    if (s != KTAU_OK) continue;
    if (G.kind != kContract) {
      s = ktau_launch_batch_merge(B->d_ds, G.d_ids, (int)G.ids.size(), G.d_tile_prefix, G.tiles,
                                  G.max_n, G.kind == kMergeCta ? 1 : 0, ls);
      continue;
    }
    ktau_sg_group g;
    g.ds = B->d_ds;
    g.bids = G.d_ids;
    g.nb = (int)G.ids.size();
    g.esize = G.esize;
    g.obits = G.obits;
    g.row_prefix = G.d_row_prefix;
    g.blk_prefix = G.d_blk_prefix;
    g.blocks = G.blocks;
    g.unit_prefix = G.d_unit_prefix;
    g.jt_prefix = G.d_jt_prefix;
    g.rows = G.rows;
    g.units = G.units;
    g.jt_tiles = G.jt_tiles;
    g.max_n = G.max_n;
    g.T = B->hds[G.ids.front()].T;
    g.tie_off = G.tie_off;
    g.tie_pairs = G.tie_pairs;
    g.tie_cap = G.tie_cap;
    g.sgn = G.sgn;
    g.stride = G.stride;
    g.tmap = G.tmap;
    g.tmap_b = G.tmap_b;
    s = ktau_signgemm_batch(g, ls);
  }
  // join: the caller's stream waits for every lane (also after an error, so that no lane is left
  // forked, e.g. inside a graph capture)
  for (int l = 0; lanes && l < ktau_batch::kLanes; ++l) {
    cudaError_t e = cudaEventRecord(B->join[l], B->lane[l]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, B->join[l], 0);
    if (e != cudaSuccess && s == KTAU_OK) s = ktau_cuda_fail(e, "batch join");
  }
  return s;
}

extern "C" ktau_status ktau_batch_graph_launch(ktau_batch* B, void* stream) {
  if (!B) return ktau_fail(KTAU_EINVAL, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return ktau_fail(KTAU_EINVAL, "graph capture needs a non-default stream");
  if (!B->exec) {
    KTAU_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    ktau_status s = ktau_batch_run(B, stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s != KTAU_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return ktau_cuda_fail(e, "cudaStreamEndCapture");
    B->graph = graph;
    KTAU_CUDA(cudaGraphInstantiate(&B->exec, B->graph, 0));
  }
  KTAU_CUDA(cudaGraphLaunch(B->exec, st));
  return KTAU_OK;
}

extern "C" ktau_status ktau_batch_check(ktau_batch* B, void* stream) {
  if (!B) return ktau_fail(KTAU_EINVAL, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  ktau_stats h;
  KTAU_CUDA(cudaMemcpyAsync(&h, B->d_stats, sizeof(h), cudaMemcpyDeviceToHost, st));
  KTAU_CUDA(cudaStreamSynchronize(st));
  KTAU_CUDA(cudaMemsetAsync(B->d_stats, 0, sizeof(ktau_stats), st));
  ktau_status s = ktau_signgemm_check_error(st);
  if (s != KTAU_OK) return s;
  if (h.nan_flag) return ktau_fail(KTAU_ENAN, "NaN in a dataset of the batch");
  return KTAU_OK;
}

extern "C" ktau_status ktau_batch_paths(const ktau_batch* B, int32_t* n_merge, int32_t* n_signgemm) {
  if (!B) return ktau_fail(KTAU_EINVAL, "batch is NULL");
  int32_t nm = 0, ns = 0;
  for (const GroupPlan& G : B->g) (G.kind == kContract ? ns : nm) += (int32_t)G.ids.size();
  if (n_merge) *n_merge = nm;
  if (n_signgemm) *n_signgemm = ns;
  return KTAU_OK;
}

extern "C" ktau_status ktau_batch_pairs(const ktau_batch* B, uint64_t* pairs) {
  if (!B || !pairs) return ktau_fail(KTAU_EINVAL, "NULL argument");
  *pairs = B->pairs;
  return KTAU_OK;
}

// ---------------------------------------------------------------------------------------------
// One call over many datasets with the scratch in the caller's workspace.
// ---------------------------------------------------------------------------------------------
extern "C" ktau_status ktau_workspace_size(const ktau_batch_desc* descs, int32_t count,
                                           const ktau_options* opt, size_t* bytes) {
  if (!bytes) return ktau_fail(KTAU_EINVAL, "bytes is NULL");
  *bytes = 0;
  ktau_batch* B = new ktau_batch();
  B->source = ktau_batch::kMeasure;
  ktau_status s = batch_build(descs, count, opt, B);
  if (s != KTAU_OK) return s;
  *bytes = B->arena_used;
  ktau_batch_free(B);
  return KTAU_OK;
}

extern "C" ktau_status ktau_allpairs_batched(const ktau_batch_desc* descs, int32_t count,
                                             const ktau_options* opt, void* workspace,
                                             size_t workspace_bytes, uint32_t* nan_flag,
                                             void* stream) {
  if (!workspace) return ktau_fail(KTAU_EINVAL, "workspace is NULL");
  if ((uintptr_t)workspace & 255) return ktau_fail(KTAU_EINVAL, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ktau_batch* B = new ktau_batch();
  B->source = ktau_batch::kWorkspace;
  B->arena = (char*)workspace;
  B->arena_cap = workspace_bytes;
  B->copy_st = st;
  ktau_status s = batch_build(descs, count, opt, B);
  if (s != KTAU_OK) return s;
  s = ktau_batch_run(B, stream);
  if (s == KTAU_OK && nan_flag) {
    const cudaError_t e = cudaMemcpyAsync(nan_flag, &B->d_stats->nan_flag, sizeof(uint32_t),
                                          cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) s = ktau_cuda_fail(e, "cudaMemcpyAsync(nan_flag)");
  }
  ktau_batch_free(B);
  return s;
}
