// ktau_allpairs_noalloc: the rank transform and the Knight merge path for one matrix, with every
// byte of working memory taken from a fixed array compiled into the library instead of being
// allocated. It exists for callers that cannot allocate device memory at the point where they
// need the result: plug-ins that must stay inside a memory budget owned by a host framework's
// allocator, and real-time loops that forbid cudaMalloc/cudaFree (which can synchronise the
// device). The call synchronises its stream once, to read the NaN flag of the rank transform.
//
// The working memory is the ranked matrix (permutation, dense ranks, ranks in sorted order, tie
// counts, denominator factors, statistics): for m variables of n samples it needs
// 3 * m * ld * 2 + 32 * m bytes (ld = n rounded up to 16, each array padded to 256 bytes) plus
// 256 bytes, at most KTAU_NOALLOC_SCRATCH_BYTES.
#include <cstring>
#include <mutex>

#include "ktau_impl.cuh"

// Shared by every call on a device; a GPU that loads the library keeps it until process exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[KTAU_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64];  // device address of g_noalloc_scratch, per device
}  // namespace

ktau_status ktau_check_counts(int64_t n, int count_bits);

// Device address of the scratch array on the current device. In host code the array's name is
// only a host-side stand-in, so the address is queried once per device (with that device
// current) and cached.
static ktau_status noalloc_scratch(void** out) {
  int dev = 0;
  KTAU_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return ktau_fail(KTAU_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return ktau_cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return KTAU_OK;
}

extern "C" ktau_status ktau_allpairs_noalloc(const void* values, ktau_dtype dt, int64_t m, int64_t n,
                                             int64_t ld, uint64_t p_begin, uint64_t p_end,
                                             double* tau64, float* tau32, void* S, void* n3,
                                             int32_t count_bits, void* stream) {
  if (!values) return ktau_fail(KTAU_EINVAL, "values is NULL");
  if (dt != KTAU_F32 && dt != KTAU_I32) return ktau_fail(KTAU_EINVAL, "unknown dtype %d", (int)dt);
  if (m < 2 || n < 2) return ktau_fail(KTAU_EINVAL, "need m >= 2 and n >= 2");
  if (ld < n) return ktau_fail(KTAU_EINVAL, "ld (%lld) < n (%lld)", (long long)ld, (long long)n);
  if (n > KTAU_BATCH_MAX_N)
    return ktau_fail(KTAU_ETOOLARGE, "n=%lld exceeds KTAU_BATCH_MAX_N=%d", (long long)n,
                     KTAU_BATCH_MAX_N);
  ktau_status s = ktau_check_counts(n, count_bits);
  if (s != KTAU_OK) return s;
  const uint64_t P = (uint64_t)(m * (m - 1) / 2);
  if (p_begin > p_end || p_end > P)
    return ktau_fail(KTAU_EINVAL, "pair range outside [0, %llu)", (unsigned long long)P);

  // Layout of the ranked matrix inside the scratch array (same arrays as a ktau_ranked handle).
  const int64_t ldr = (n + 15) & ~15LL;
  const size_t arr = ((size_t)m * ldr * sizeof(uint16_t) + 255) & ~(size_t)255;
  const size_t t8 = ((size_t)m * 8 + 255) & ~(size_t)255;
  const size_t t4 = ((size_t)m * 4 + 255) & ~(size_t)255;
  const size_t need = 3 * arr + 3 * t8 + 2 * t4 + 256;
  if (need > (size_t)KTAU_NOALLOC_SCRATCH_BYTES)
    return ktau_fail(KTAU_ETOOLARGE,
                     "m=%lld x n=%lld needs %zu bytes of scratch; the fixed scratch holds %u",
                     (long long)m, (long long)n, need, (unsigned)KTAU_NOALLOC_SCRATCH_BYTES);
  void* base = nullptr;
  if ((s = noalloc_scratch(&base)) != KTAU_OK) return s;
  if (p_begin == p_end) return KTAU_OK;

  ktau_ranked R;
  memset(&R, 0, sizeof(R));
  R.m = m;
  R.n = n;
  R.ld = ldr;
  cudaGetDevice(&R.device);
  char* b = (char*)base;
  R.perm = (uint16_t*)b;
  R.rank = (uint16_t*)(b + arr);
  R.srank = (uint16_t*)(b + 2 * arr);
  R.T = (int64_t*)(b + 3 * arr);
  R.rs64 = (double*)(b + 3 * arr + t8);
  R.rsff = (float2*)(b + 3 * arr + 2 * t8);
  R.ndist = (int32_t*)(b + 3 * arr + 3 * t8);
  R.maxg = (int32_t*)(b + 3 * arr + 3 * t8 + t4);
  R.stats_dev = (ktau_stats*)(b + 3 * arr + 3 * t8 + 2 * t4);

  cudaStream_t st = (cudaStream_t)stream;
  // The statistics accumulate with atomics: they must start at zero on every call. Everything
  // else in the scratch is fully overwritten by the rank kernel.
  KTAU_CUDA(cudaMemsetAsync(R.stats_dev, 0, sizeof(ktau_stats), st));
  if ((s = ktau_launch_rank(values, (int)dt, m, n, ld, &R, st)) != KTAU_OK) return s;
  ktau_stats h;
  KTAU_CUDA(cudaMemcpyAsync(&h, R.stats_dev, sizeof(h), cudaMemcpyDeviceToHost, st));
  KTAU_CUDA(cudaStreamSynchronize(st));
  if (h.nan_flag) return ktau_fail(KTAU_ENAN, "NaN in the input matrix");
  R.stats = h;
  ktau_merge_plan plan;
  ktau_merge_default_plan(n, &plan);
  plan.schedule = 1;  // static tile schedule: the dynamic one needs an allocated counter
  ktau_out out{tau64, tau32, S, n3, count_bits};
  return ktau_launch_merge(&R, p_begin, p_end, out, plan, st);
}
