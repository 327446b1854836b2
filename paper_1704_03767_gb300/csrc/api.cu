// C ABI entry points: argument validation, handle ownership, path dispatch, error reporting.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

#include "ktau_impl.cuh"
#include "signgemm.cuh"

static thread_local char t_err[512] = "no error";

ktau_status ktau_fail(ktau_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_err, sizeof(t_err), fmt, ap);
  va_end(ap);
  return s;
}

ktau_status ktau_cuda_fail(cudaError_t e, const char* what) {
  snprintf(t_err, sizeof(t_err), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // clear the sticky-free allocation error
    return KTAU_ENOMEM;
  }
  return KTAU_ECUDA;
}

int ktau_sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

namespace {
std::mutex g_alloc_mu;
struct FreeBlock {
  int dev;
  size_t bytes;
  void* p;
};
std::vector<FreeBlock>* g_free_blocks = new std::vector<FreeBlock>();  // never destroyed
}  // namespace

static std::atomic<int> g_fail_alloc_after{-1};

extern "C" ktau_status ktau_debug_fail_alloc(int32_t k) {
  g_fail_alloc_after.store(k < 0 ? -1 : k);
  return KTAU_OK;
}

// Blocks are cached by size class: requests are rounded up to the next of 2^k, 1.25 * 2^k,
// 1.5 * 2^k, 1.75 * 2^k (at most 25% slack), so work of varying size (query batches, batched
// datasets) reuses a bounded set of blocks instead of one per distinct size.
static size_t size_class(size_t bytes) {
  if (bytes <= 4096) return 4096;
  int k = 63 - __builtin_clzll((unsigned long long)(bytes - 1));  // 2^k < bytes <= 2^(k+1)
  const size_t base = (size_t)1 << k, step = base >> 2;
  return base + ((bytes - base + step - 1) / step) * step;
}

ktau_status ktau_dmalloc(void** p, size_t bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  bytes = size_class(bytes);
  // injected failure (tests of the error paths)
  int left = g_fail_alloc_after.load();
  while (left >= 0) {
    if (left == 0) {
      *p = nullptr;
      return ktau_fail(KTAU_ENOMEM, "device allocation of %zu bytes failed (injected)", bytes);
    }
    if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) break;
  }
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    for (size_t i = 0; i < g_free_blocks->size(); ++i) {
      FreeBlock& b = (*g_free_blocks)[i];
      if (b.dev == dev && b.bytes == bytes) {
        *p = b.p;
        (*g_free_blocks)[i] = g_free_blocks->back();
        g_free_blocks->pop_back();
        return KTAU_OK;
      }
    }
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    // Give cached blocks back to the driver and retry once.
    std::vector<FreeBlock> mine;
    {
      std::lock_guard<std::mutex> lk(g_alloc_mu);
      std::vector<FreeBlock> keep;
      for (auto& b : *g_free_blocks) (b.dev == dev ? mine : keep).push_back(b);
      *g_free_blocks = keep;
    }
    cudaGetLastError();
    for (auto& b : mine) cudaFree(b.p);
    e = cudaMalloc(p, bytes);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return ktau_cuda_fail(e, "cudaMalloc");
  }
  return KTAU_OK;
}

void ktau_dfree(void* p, size_t bytes) {
  if (!p) return;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_free_blocks->push_back(FreeBlock{dev, size_class(bytes), p});
}

extern "C" {

const char* ktau_last_error(void) { return t_err; }

const char* ktau_status_string(ktau_status s) {
  switch (s) {
    case KTAU_OK: return "KTAU_OK";
    case KTAU_EINVAL: return "KTAU_EINVAL";
    case KTAU_ENAN: return "KTAU_ENAN";
    case KTAU_ETOOLARGE: return "KTAU_ETOOLARGE";
    case KTAU_ENOMEM: return "KTAU_ENOMEM";
    case KTAU_ECUDA: return "KTAU_ECUDA";
    case KTAU_ETIMEOUT: return "KTAU_ETIMEOUT";
    case KTAU_EBUSY: return "KTAU_EBUSY";
  }
  return "KTAU_UNKNOWN";
}

int32_t ktau_abi_version(void) { return KTAU_ABI_VERSION; }

}  // extern "C"

// Pinned host slots for the statistics of asynchronously prepared handles (one page-locked
// allocation made on first use, slots recycled when their handle releases them).
namespace {
constexpr int kPinSlots = 4096;
std::mutex g_pin_mu;
ktau_stats* g_pin = nullptr;
std::vector<int> g_pin_free;

ktau_stats* pin_take() {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (!g_pin) {
    if (cudaHostAlloc((void**)&g_pin, kPinSlots * sizeof(ktau_stats), cudaHostAllocPortable) !=
        cudaSuccess) {
      cudaGetLastError();
      g_pin = nullptr;
      return nullptr;
    }
    for (int i = kPinSlots - 1; i >= 0; --i) g_pin_free.push_back(i);
  }
  if (g_pin_free.empty()) return nullptr;
  const int i = g_pin_free.back();
  g_pin_free.pop_back();
  return g_pin + i;
}

void pin_give(ktau_stats* p) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back((int)(p - g_pin));
}

// Releases the pinned slot and event of a handle whose copy has completed (or never started),
// and the long-row rank scratch (the rank transform precedes the statistics copy on its stream).
void stats_release(ktau_ranked* R) {
  if (R->stats_pin) pin_give(R->stats_pin);
  if (R->stats_ev) cudaEventDestroy(R->stats_ev);
  R->stats_pin = nullptr;
  R->stats_ev = nullptr;
  if (R->tmp_block) ktau_dfree(R->tmp_block, R->tmp_bytes);
  R->tmp_block = nullptr;
}

ktau_status rank_prepare_impl(const void* values, ktau_dtype dt, int64_t m, int64_t n,
                              int64_t ld, void* stream, bool async, ktau_ranked** out) {
  if (!out) return ktau_fail(KTAU_EINVAL, "out is NULL");
  *out = nullptr;
  if (!values) return ktau_fail(KTAU_EINVAL, "values is NULL");
  if (dt != KTAU_F32 && dt != KTAU_I32) return ktau_fail(KTAU_EINVAL, "unknown dtype %d", (int)dt);
  if (m < 1 || n < 2) return ktau_fail(KTAU_EINVAL, "need m >= 1 and n >= 2 (m=%lld n=%lld)",
                                       (long long)m, (long long)n);
  if (ld < n) return ktau_fail(KTAU_EINVAL, "ld (%lld) < n (%lld)", (long long)ld, (long long)n);
  if (n > KTAU_MAX_N) return ktau_fail(KTAU_ETOOLARGE, "n=%lld exceeds KTAU_MAX_N=%d",
                                       (long long)n, KTAU_MAX_N);
  if (m > KTAU_MAX_M) return ktau_fail(KTAU_ETOOLARGE, "m=%lld exceeds KTAU_MAX_M=%d",
                                       (long long)m, KTAU_MAX_M);
  cudaStream_t st = (cudaStream_t)stream;
  ktau_ranked* R = (ktau_ranked*)calloc(1, sizeof(ktau_ranked));
  if (!R) return ktau_fail(KTAU_ENOMEM, "host allocation failed");
  R->m = m;
  R->n = n;
  R->ld = (n + 15) & ~15LL;
  R->wide = n > KTAU_NARROW_MAX_N;
  cudaGetDevice(&R->device);
  const size_t esz = R->wide ? sizeof(uint32_t) : sizeof(uint16_t);
  const size_t arr = (size_t)m * R->ld * esz;
  const size_t arr_al = (arr + 255) & ~(size_t)255;
  const size_t t_bytes = ((size_t)m * 8 + 255) & ~(size_t)255;
  const size_t i_bytes = ((size_t)m * 4 + 255) & ~(size_t)255;
  const size_t total = 3 * arr_al + 3 * t_bytes + 2 * i_bytes + 256;
  R->block_bytes = total;
  if (ktau_dmalloc(&R->block, total) != KTAU_OK) {
    free(R);
    return KTAU_ENOMEM;
  }
  cudaError_t e;
  char* b = (char*)R->block;
  if (R->wide) {
    R->perm32 = (uint32_t*)b;
    R->rank32 = (uint32_t*)(b + arr_al);
    R->srank32 = (uint32_t*)(b + 2 * arr_al);
  } else {
    R->perm = (uint16_t*)b;
    R->rank = (uint16_t*)(b + arr_al);
    R->srank = (uint16_t*)(b + 2 * arr_al);
  }
  R->T = (int64_t*)(b + 3 * arr_al);
  R->ndist = (int32_t*)(b + 3 * arr_al + t_bytes);
  R->maxg = (int32_t*)(b + 3 * arr_al + t_bytes + i_bytes);
  R->rs64 = (double*)(b + 3 * arr_al + t_bytes + 2 * i_bytes);
  R->rsff = (float2*)(b + 3 * arr_al + 2 * t_bytes + 2 * i_bytes);
  R->stats_dev = (ktau_stats*)(b + 3 * arr_al + 3 * t_bytes + 2 * i_bytes);
  ktau_status s = KTAU_OK;
  if ((e = cudaMemsetAsync(R->stats_dev, 0, sizeof(ktau_stats), st)) != cudaSuccess) {
    s = ktau_cuda_fail(e, "cudaMemsetAsync");
  }
  if (s == KTAU_OK) s = ktau_launch_rank(values, (int)dt, m, n, ld, R, st);
  ktau_stats* pin = (s == KTAU_OK && async) ? pin_take() : nullptr;
  if (pin) {
    R->stats_pin = pin;
    if ((e = cudaEventCreateWithFlags(&R->stats_ev, cudaEventDisableTiming)) != cudaSuccess) {
      R->stats_ev = nullptr;
      s = ktau_cuda_fail(e, "cudaEventCreate");
    } else if ((e = cudaMemcpyAsync(pin, R->stats_dev, sizeof(ktau_stats),
                                    cudaMemcpyDeviceToHost, st)) != cudaSuccess) {
      s = ktau_cuda_fail(e, "cudaMemcpyAsync(stats)");
    } else if ((e = cudaEventRecord(R->stats_ev, st)) != cudaSuccess) {
      s = ktau_cuda_fail(e, "cudaEventRecord(stats)");
    }
  } else if (s == KTAU_OK) {
    if ((e = cudaMemcpyAsync(&R->stats, R->stats_dev, sizeof(ktau_stats), cudaMemcpyDeviceToHost,
                             st)) != cudaSuccess)
      s = ktau_cuda_fail(e, "cudaMemcpyAsync(stats)");
    else if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
      s = ktau_cuda_fail(e, "cudaStreamSynchronize");
    else if (R->stats.nan_flag)
      s = ktau_fail(KTAU_ENAN, "NaN in the input matrix");
    if (e == cudaSuccess) stats_release(R);  // the rank transform has run: its scratch is free
  }
  if (s != KTAU_OK) {
    cudaStreamSynchronize(st);
    stats_release(R);
    ktau_dfree(R->block, R->block_bytes);
    free(R);
    return s;
  }
  *out = R;
  return KTAU_OK;
}

}  // namespace

ktau_status ktau_rank_prepare(const void* values, ktau_dtype dt, int64_t m, int64_t n, int64_t ld,
                              void* stream, ktau_ranked** out) {
  return rank_prepare_impl(values, dt, m, n, ld, stream, false, out);
}

ktau_status ktau_rank_prepare_async(const void* values, ktau_dtype dt, int64_t m, int64_t n,
                                    int64_t ld, void* stream, ktau_ranked** out) {
  return rank_prepare_impl(values, dt, m, n, ld, stream, true, out);
}

ktau_status ktau_rank_prepare_host(const void* values_h, ktau_dtype dt, int64_t m, int64_t n,
                                   int64_t ld, void* stream, ktau_ranked** out) {
  if (!out) return ktau_fail(KTAU_EINVAL, "out is NULL");
  *out = nullptr;
  if (!values_h) return ktau_fail(KTAU_EINVAL, "values is NULL");
  if (dt != KTAU_F32 && dt != KTAU_I32) return ktau_fail(KTAU_EINVAL, "unknown dtype %d", (int)dt);
  if (m < 1 || n < 2 || ld < n)
    return ktau_fail(KTAU_EINVAL, "need m >= 1, n >= 2 and ld >= n");
  if (n > KTAU_MAX_N || m > KTAU_MAX_M)
    return ktau_fail(KTAU_ETOOLARGE, "m=%lld x n=%lld beyond the limits", (long long)m,
                     (long long)n);
  cudaStream_t st = (cudaStream_t)stream;
  // Staging copy of the values (4-byte elements, rows packed to n), released once the rank
  // transform has read it: ktau_rank_prepare synchronises the stream before returning.
  const size_t row = (size_t)n * 4, bytes = (size_t)m * row;
  void* dv = nullptr;
  ktau_status s = ktau_dmalloc(&dv, bytes);
  if (s != KTAU_OK) return s;
  const cudaError_t e = cudaMemcpy2DAsync(dv, row, values_h, (size_t)ld * 4, row, (size_t)m,
                                          cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess)
    s = ktau_cuda_fail(e, "cudaMemcpy2DAsync(values)");
  else
    s = rank_prepare_impl(dv, dt, m, n, n, stream, false, out);
  cudaStreamSynchronize(st);
  ktau_dfree(dv, bytes);
  return s;
}

ktau_status ktau_ranked_stats(const ktau_ranked* Rc) {
  if (!Rc) return ktau_fail(KTAU_EINVAL, "handle is NULL");
  ktau_ranked* R = const_cast<ktau_ranked*>(Rc);
  if (R->stats_pin) {
    const cudaError_t e = cudaEventSynchronize(R->stats_ev);
    if (e != cudaSuccess) return ktau_cuda_fail(e, "statistics copy");
    R->stats = *R->stats_pin;
    stats_release(R);
  }
  if (R->stats.nan_flag) return ktau_fail(KTAU_ENAN, "NaN in the input matrix");
  return KTAU_OK;
}

extern "C" {

ktau_status ktau_ranked_free(ktau_ranked* R) {
  if (!R) return KTAU_OK;
  cudaDeviceSynchronize();  // no kernel may still use the handle's memory when it is recycled
  stats_release(R);
  if (R->block) ktau_dfree(R->block, R->block_bytes);
  ktau_signgemm_release(R);
  ktau_bits_release(R);
  free(R);
  return KTAU_OK;
}

ktau_status ktau_ranked_free_on(ktau_ranked* R, void* stream) {
  if (!R) return KTAU_OK;
  KTAU_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  stats_release(R);
  if (R->block) ktau_dfree(R->block, R->block_bytes);
  ktau_signgemm_release(R);
  ktau_bits_release(R);
  free(R);
  return KTAU_OK;
}

ktau_status ktau_ranked_shape(const ktau_ranked* R, int64_t* m, int64_t* n) {
  if (!R) return ktau_fail(KTAU_EINVAL, "handle is NULL");
  if (m) *m = R->m;
  if (n) *n = R->n;
  return KTAU_OK;
}

ktau_status ktau_tie_counts(const ktau_ranked* R, int64_t* T_dev, void* stream) {
  if (!R || !T_dev) return ktau_fail(KTAU_EINVAL, "NULL argument");
  KTAU_CUDA(cudaMemcpyAsync(T_dev, R->T, (size_t)R->m * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
  return KTAU_OK;
}

ktau_status ktau_ranked_export(const ktau_ranked* R, uint16_t* perm, uint16_t* rank, void* stream) {
  if (!R) return ktau_fail(KTAU_EINVAL, "handle is NULL");
  if (R->wide)
    return ktau_fail(KTAU_EINVAL, "n=%lld > %d has 32-bit ranks: use ktau_ranked_export32",
                     (long long)R->n, KTAU_NARROW_MAX_N);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t pitch = (size_t)R->ld * sizeof(uint16_t), width = (size_t)R->n * sizeof(uint16_t);
  if (perm)
    KTAU_CUDA(cudaMemcpy2DAsync(perm, width, R->perm, pitch, width, (size_t)R->m,
                                cudaMemcpyDeviceToDevice, st));
  if (rank)
    KTAU_CUDA(cudaMemcpy2DAsync(rank, width, R->rank, pitch, width, (size_t)R->m,
                                cudaMemcpyDeviceToDevice, st));
  return KTAU_OK;
}

ktau_status ktau_ranked_export32(const ktau_ranked* R, uint32_t* perm, uint32_t* rank,
                                 void* stream) {
  if (!R) return ktau_fail(KTAU_EINVAL, "handle is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (!R->wide) return ktau_launch_widen(R, perm, rank, st);
  const size_t pitch = (size_t)R->ld * sizeof(uint32_t), width = (size_t)R->n * sizeof(uint32_t);
  if (perm)
    KTAU_CUDA(cudaMemcpy2DAsync(perm, width, R->perm32, pitch, width, (size_t)R->m,
                                cudaMemcpyDeviceToDevice, st));
  if (rank)
    KTAU_CUDA(cudaMemcpy2DAsync(rank, width, R->rank32, pitch, width, (size_t)R->m,
                                cudaMemcpyDeviceToDevice, st));
  return KTAU_OK;
}

}  // extern "C"

// Shared validation of count widths and options.
ktau_status ktau_check_counts(int64_t n, int count_bits) {
  if (count_bits != 32 && count_bits != 64)
    return ktau_fail(KTAU_EINVAL, "count_bits must be 32 or 64 (got %d)", count_bits);
  const int64_t n0 = n * (n - 1) / 2;
  if (count_bits == 32 && n0 >= (1LL << 31))
    return ktau_fail(KTAU_ETOOLARGE, "n_0=%lld does not fit 32-bit counts", (long long)n0);
  return KTAU_OK;
}

ktau_status ktau_check_options(const ktau_options* opt) {
  if (!opt) return KTAU_OK;
  if (opt->path < 0 || opt->path > 3) return ktau_fail(KTAU_EINVAL, "bad path %d", opt->path);
  if (opt->tile_q < 0 || opt->tile_q > 256)
    return ktau_fail(KTAU_EINVAL, "tile_q must be in [0, 256]");
  if (opt->mapping < 0 || opt->mapping > 2) return ktau_fail(KTAU_EINVAL, "bad mapping");
  if (opt->schedule < 0 || opt->schedule > 2) return ktau_fail(KTAU_EINVAL, "bad schedule");
  if (opt->ctas_per_sm < 0 || opt->ctas_per_sm > 32) return ktau_fail(KTAU_EINVAL, "bad ctas_per_sm");
  if (opt->operand_bits != 0 && opt->operand_bits != 4 && opt->operand_bits != 8 &&
      opt->operand_bits != 16)
    return ktau_fail(KTAU_EINVAL, "operand_bits must be 0, 4, 8 or 16");
  if (opt->statistic != 0 && opt->statistic != 1)
    return ktau_fail(KTAU_EINVAL, "statistic must be 0 (tau-b) or 1 (tau-a)");
  return KTAU_OK;
}

// Path choice for one matrix shape, from the autotuner's measurements on GB300 (ns per pair at
// m ~ 2000): the sign contraction wins at every n it takes (e.g. 0.05 vs 2.5 at n = 128, 2.7 vs
// 50 at n = 2000, with 5% or 30% duplicated values), so it is the default there. With FP8 or BF16
// operands a tie-heavy matrix (more than 4n tied sample pairs per variable on average) goes to
// the merge path instead: its n_3 would come from per-pair tie checks (about T_u per pair), which
// outgrow the merge path's n log2 n steps; FP4 operands take n_3 from the magnitude contraction.
int ktau_choose_path(const ktau_ranked* R, const ktau_options* opt) {
  if (opt && opt->path != KTAU_PATH_AUTO) return opt->path;
  if (ktau_signgemm_supported(R->n)) {
    const double mean_T = (double)R->stats.T_sum / (double)R->m;
    if (mean_T <= 4.0 * (double)R->n || ktau_sign_obits(R->n, opt) == 4)
      return KTAU_PATH_SIGNGEMM;
  }
  return KTAU_PATH_MERGE;
}

extern "C" ktau_status ktau_allpairs(const ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                                     double* tau64, float* tau32, void* S, void* n3,
                                     int32_t count_bits, const ktau_options* opt, void* stream) {
  if (!R) return ktau_fail(KTAU_EINVAL, "handle is NULL");
  ktau_status s = ktau_check_counts(R->n, count_bits);
  if (s != KTAU_OK) return s;
  if ((s = ktau_ranked_stats(R)) != KTAU_OK) return s;
  if ((s = ktau_check_options(opt)) != KTAU_OK) return s;
  const uint64_t P = (uint64_t)(R->m * (R->m - 1) / 2);
  if (p_begin > p_end || p_end > P)
    return ktau_fail(KTAU_EINVAL, "pair range [%llu, %llu) outside [0, %llu)",
                     (unsigned long long)p_begin, (unsigned long long)p_end,
                     (unsigned long long)P);
  if (p_begin == p_end) return KTAU_OK;
  ktau_out out{tau64, tau32, S, n3, count_bits, opt ? opt->statistic : 0};
  cudaStream_t st = (cudaStream_t)stream;
  const int path = ktau_choose_path(R, opt);
  if (path == KTAU_PATH_BITS)
    return ktau_bits_allpairs(const_cast<ktau_ranked*>(R), p_begin, p_end, out, st);
  if (path == KTAU_PATH_SIGNGEMM) {
    if (!ktau_signgemm_supported(R->n))
      return ktau_fail(KTAU_EINVAL, "sign-contraction path supports n <= %d", KTAU_SIGNGEMM_MAX_N);
    return ktau_signgemm_allpairs(const_cast<ktau_ranked*>(R), p_begin, p_end, out,
                                  ktau_sign_obits(R->n, opt), st);
  }
  ktau_merge_plan plan;
  ktau_merge_default_plan(R->n, &plan);
  if (opt) {
    if (opt->tile_q) plan.tile_q = opt->tile_q;
    if (opt->mapping) plan.mapping = opt->mapping;
    if (opt->schedule) plan.schedule = opt->schedule;
    if (opt->ctas_per_sm) plan.ctas_per_sm = opt->ctas_per_sm;
  }
  return ktau_launch_merge(R, p_begin, p_end, out, plan, st);
}

extern "C" ktau_status ktau_allpairs_path(const ktau_ranked* R, const ktau_options* opt,
                                          int32_t* path) {
  if (!R || !path) return ktau_fail(KTAU_EINVAL, "NULL argument");
  ktau_status s = ktau_check_options(opt);
  if (s != KTAU_OK) return s;
  if ((s = ktau_ranked_stats(R)) != KTAU_OK) return s;
  *path = ktau_choose_path(R, opt);
  return KTAU_OK;
}

extern "C" ktau_status ktau_prepare_signs(ktau_ranked* R, void* stream) {
  if (!R) return ktau_fail(KTAU_EINVAL, "handle is NULL");
  if (!ktau_signgemm_supported(R->n))
    return ktau_fail(KTAU_EINVAL, "sign contraction supports n <= %d", KTAU_SIGNGEMM_MAX_N);
  return ktau_signgemm_prepare(R, ktau_sign_obits(R->n, nullptr), (cudaStream_t)stream);
}

ktau_status ktau_query_check_status(cudaStream_t st);

extern "C" ktau_status ktau_device_status(void* stream) {
  ktau_status s = ktau_signgemm_check_error((cudaStream_t)stream);
  if (s != KTAU_OK) return s;
  return ktau_query_check_status((cudaStream_t)stream);
}

// ---------------------------------------------------------------------------------------------
// Kernel trace
// ---------------------------------------------------------------------------------------------
namespace {
struct TraceRec {
  char name[48];
  cudaEvent_t e0, e1;
};
std::mutex g_trace_mu;
bool g_trace_on = false;
std::vector<TraceRec>* g_trace = new std::vector<TraceRec>();
}  // namespace

static char g_trace_only[48] = "";  // ktau_trace_filter; empty = every launch

ktau_trace_scope::ktau_trace_scope(const char* name, cudaStream_t s) : slot(-1), st(s) {
  if (!g_trace_on) return;
  if (g_trace_only[0] && strncmp(name, g_trace_only, sizeof(g_trace_only)) != 0) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  TraceRec r;
  snprintf(r.name, sizeof(r.name), "%s", name);
  if (cudaEventCreate(&r.e0) != cudaSuccess) return;
  if (cudaEventCreate(&r.e1) != cudaSuccess) {
    cudaEventDestroy(r.e0);
    return;
  }
  cudaEventRecord(r.e0, s);
  std::lock_guard<std::mutex> lk(g_trace_mu);
  slot = (int)g_trace->size();
  g_trace->push_back(r);
}

ktau_trace_scope::~ktau_trace_scope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (slot < (int)g_trace->size()) cudaEventRecord((*g_trace)[slot].e1, st);
}

extern "C" ktau_status ktau_trace_enable(int32_t on) {
  g_trace_on = on != 0;
  return KTAU_OK;
}

extern "C" ktau_status ktau_trace_filter(const char* name) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  snprintf(g_trace_only, sizeof(g_trace_only), "%s", name ? name : "");
  return KTAU_OK;
}

extern "C" ktau_status ktau_trace_collect(ktau_trace_record* out, int32_t cap, int32_t* count) {
  std::vector<TraceRec> recs;
  {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    recs.swap(*g_trace);
  }
  int32_t n = 0;
  for (auto& r : recs) {
    float ms = 0.f;
    cudaEventSynchronize(r.e1);
    cudaEventElapsedTime(&ms, r.e0, r.e1);
    if (out && n < cap) {
      memcpy(out[n].name, r.name, sizeof(r.name));
      out[n].ms = ms;
    }
    ++n;
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  if (count) *count = n < cap ? n : cap;
  return KTAU_OK;
}

// ---------------------------------------------------------------------------------------------
// Passes with overlapped device-to-host copies (Sec. 4.3.1).
// ---------------------------------------------------------------------------------------------
extern "C" ktau_status ktau_allpairs_host(const ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                                          double* tau64_h, float* tau32_h, void* S_h, void* n3_h,
                                          int32_t count_bits, const ktau_options* opt,
                                          uint64_t pass_pairs, void* stream) {
  if (!R) return ktau_fail(KTAU_EINVAL, "handle is NULL");
  ktau_status s = ktau_check_counts(R->n, count_bits);
  if (s != KTAU_OK) return s;
  if ((s = ktau_ranked_stats(R)) != KTAU_OK) return s;
  if ((s = ktau_check_options(opt)) != KTAU_OK) return s;
  const uint64_t P = (uint64_t)(R->m * (R->m - 1) / 2);
  if (p_begin > p_end || p_end > P) return ktau_fail(KTAU_EINVAL, "pair range outside the triangle");
  if (p_begin == p_end) return KTAU_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t total = p_end - p_begin;
  if (pass_pairs == 0) {
    // about a quarter of the range, rounded to whole 256-row blocks of the triangle
    pass_pairs = (total + 3) / 4;
    const uint64_t rowblock = (uint64_t)R->m * 256;
    if (pass_pairs > rowblock) pass_pairs = (pass_pairs + rowblock - 1) / rowblock * rowblock;
  }
  if (pass_pairs > total) pass_pairs = total;
  const size_t cb = (size_t)count_bits / 8;
  const size_t esz[4] = {sizeof(double), sizeof(float), cb, cb};
  void* hst[4] = {tau64_h, tau32_h, S_h, n3_h};
  void* dev[2][4] = {{nullptr}};
  size_t bytes[4];
  for (int o = 0; o < 4; ++o) bytes[o] = (size_t)pass_pairs * esz[o];
  for (int b = 0; b < 2 && s == KTAU_OK; ++b)
    for (int o = 0; o < 4 && s == KTAU_OK; ++o)
      if (hst[o]) s = ktau_dmalloc(&dev[b][o], bytes[o]);
  // One copy stream per output array, so that several copy engines move data at once.
  cudaStream_t cs[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t computed[2] = {nullptr, nullptr}, copied[2][4] = {{nullptr}};
  cudaError_t e = cudaSuccess;
  if (s == KTAU_OK) {
    for (int o = 0; o < 4 && e == cudaSuccess; ++o)
      if (hst[o]) e = cudaStreamCreateWithFlags(&cs[o], cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaEventCreateWithFlags(&computed[b], cudaEventDisableTiming);
      for (int o = 0; o < 4 && e == cudaSuccess; ++o)
        if (hst[o]) e = cudaEventCreateWithFlags(&copied[b][o], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) s = ktau_cuda_fail(e, "stream/event creation");
  }
  int pass = 0;
  for (uint64_t lo = p_begin; lo < p_end && s == KTAU_OK; lo += pass_pairs, ++pass) {
    const uint64_t hi = lo + pass_pairs < p_end ? lo + pass_pairs : p_end;
    const int b = pass & 1;
    // the buffer's previous copies must be done before it is overwritten
    for (int o = 0; o < 4 && pass >= 2; ++o)
      if (hst[o] && (e = cudaStreamWaitEvent(st, copied[b][o], 0)) != cudaSuccess) {
        s = ktau_cuda_fail(e, "cudaStreamWaitEvent");
        break;
      }
    if (s != KTAU_OK) break;
    s = ktau_allpairs(R, lo, hi, (double*)dev[b][0], (float*)dev[b][1], dev[b][2], dev[b][3],
                      count_bits, opt, stream);
    if (s != KTAU_OK) break;
    if ((e = cudaEventRecord(computed[b], st)) != cudaSuccess) {
      s = ktau_cuda_fail(e, "event");
      break;
    }
    for (int o = 0; o < 4; ++o) {
      if (!hst[o]) continue;
      if ((e = cudaStreamWaitEvent(cs[o], computed[b], 0)) != cudaSuccess ||
          (e = cudaMemcpyAsync((char*)hst[o] + (lo - p_begin) * esz[o], dev[b][o],
                               (hi - lo) * esz[o], cudaMemcpyDeviceToHost, cs[o])) != cudaSuccess ||
          (e = cudaEventRecord(copied[b][o], cs[o])) != cudaSuccess) {
        s = ktau_cuda_fail(e, "device-to-host copy");
        break;
      }
    }
  }
  for (int o = 0; o < 4; ++o)
    if (cs[o]) cudaStreamSynchronize(cs[o]);
  cudaStreamSynchronize(st);
  for (int b = 0; b < 2; ++b) {
    if (computed[b]) cudaEventDestroy(computed[b]);
    for (int o = 0; o < 4; ++o) {
      if (copied[b][o]) cudaEventDestroy(copied[b][o]);
      if (dev[b][o]) ktau_dfree(dev[b][o], bytes[o]);
    }
  }
  for (int o = 0; o < 4; ++o)
    if (cs[o]) cudaStreamDestroy(cs[o]);
  return s;
}
