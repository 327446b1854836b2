// Job-id <-> coordinate bijection of the upper triangle (Sec. 4.1, Eq. 4-10), applied to a w x w
// matrix of tiles (Sec. 4.2, Eq. 11-14) with the diagonal included, and the packed index of the
// strict upper triangle. Host and device; no CUDA runtime dependency (also built by g++ in tests).
#pragma once
#include <math.h>
#include <stdint.h>

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#endif

__host__ __device__ inline int64_t ktau_rowstart(int64_t w, int64_t y) {  // Eq. 5 / Eq. 12
  return y * (2 * w - y + 1) / 2;
}

// Eq. 6: move y until F(y) <= J < F(y+1).
__host__ __device__ inline void ktau_coord_fixup(int64_t w, int64_t J, int64_t yy, int64_t& y,
                                                 int64_t& x) {
  if (yy < 0) yy = 0;
  if (yy > w - 1) yy = w - 1;
  while (yy > 0 && ktau_rowstart(w, yy) > J) --yy;
  while (yy < w - 1 && ktau_rowstart(w, yy + 1) <= J) ++yy;
  y = yy;
  x = J + yy - ktau_rowstart(w, yy);
}

// Eq. 13-14: y = ceil(w - 1/2 - sqrt(w^2 + w + 1/4 - 2(J+1))), x = J + y - F(y). The square-root
// argument is formed exactly in integers, 4(w^2 + w + 1/4 - 2(J+1)) = (2w+1)^2 - 8(J+1), so only
// the root is rounded; a rounded root can land the ceiling one row off when z is (nearly) an
// integer, which the Eq. 6 check corrects.
__host__ __device__ inline void ktau_tile_coord_f32(int64_t w, int64_t J, int64_t& y, int64_t& x) {
  const int64_t arg = (2 * w + 1) * (2 * w + 1) - 8 * (J + 1);
  const float root = sqrtf((float)(arg > 0 ? arg : 0));
  ktau_coord_fixup(w, J, (int64_t)ceilf((float)w - 0.5f - 0.5f * root), y, x);
}
__host__ __device__ inline void ktau_tile_coord_f64(int64_t w, int64_t J, int64_t& y, int64_t& x) {
  const int64_t arg = (2 * w + 1) * (2 * w + 1) - 8 * (J + 1);
  const double root = sqrt((double)(arg > 0 ? arg : 0));
  ktau_coord_fixup(w, J, (int64_t)ceil((double)w - 0.5 - 0.5 * root), y, x);
}
// FP32 root on the device (FP64 is a slow pipe on GB300), FP64 on the host.
__host__ __device__ inline void ktau_tile_coord(int64_t w, int64_t J, int64_t& y, int64_t& x) {
#ifdef __CUDA_ARCH__
  ktau_tile_coord_f32(w, J, y, x);
#else
  ktau_tile_coord_f64(w, J, y, x);
#endif
}

// Packed index of pair (i, j), i < j, in the strict upper triangle of an m x m job matrix
// (Eq. 4 applied to the (m-1)-triangle: p = J_{m-1}(i, j-1)).
__host__ __device__ inline uint64_t ktau_pair_index(int64_t m, int64_t i, int64_t j) {
  return (uint64_t)(i * (2 * m - i - 1) / 2 + (j - i - 1));
}
