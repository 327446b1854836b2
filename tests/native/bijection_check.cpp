// Exhaustive check of the library's bijection (both square-root variants) against enumeration of
// the upper triangle in row-major order (the numbering policy of Sec. 4.1).
#include <cstdio>
#include <cstdlib>

#include "bijection.cuh"

static int check(int64_t w, int64_t J, int64_t y, int64_t x) {
  int64_t a, b, c, d;
  ktau_tile_coord_f32(w, J, a, b);
  ktau_tile_coord_f64(w, J, c, d);
  if (a != y || b != x || c != y || d != x) {
    printf("mismatch w=%lld J=%lld want (%lld,%lld) f32 (%lld,%lld) f64 (%lld,%lld)\n",
           (long long)w, (long long)J, (long long)y, (long long)x, (long long)a, (long long)b,
           (long long)c, (long long)d);
    return 1;
  }
  return 0;
}

int main() {
  int bad = 0;
  for (int64_t w = 1; w <= 700 && !bad; ++w) {
    int64_t J = 0;
    for (int64_t y = 0; y < w; ++y)
      for (int64_t x = y; x < w; ++x) bad |= check(w, J++, y, x);
  }
  // Row boundaries of large matrices: the first and last id of sampled rows.
  const int64_t big[] = {4096, 65535, 65536, 1000003, 4194304, 4194305};
  for (int64_t w : big) {
    for (int64_t k = 0; k < 4000 && !bad; ++k) {
      int64_t y = k < 2000 ? k : w - 1 - (k - 2000);
      if (k >= 1000 && k < 2000) y = (int64_t)((k * 2654435761ULL) % (uint64_t)w);
      const int64_t first = ktau_rowstart(w, y), last = first + (w - 1 - y);
      bad |= check(w, first, y, y);
      bad |= check(w, last, y, w - 1);
    }
  }
  // Packed strict-upper index against enumeration.
  for (int64_t m = 2; m <= 300 && !bad; ++m) {
    uint64_t p = 0;
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = i + 1; j < m; ++j)
        if (ktau_pair_index(m, i, j) != p++) bad = 1;
  }
  printf(bad ? "FAIL\n" : "OK\n");
  return bad;
}
