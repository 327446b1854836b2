// K-c: exact sign-matrix contraction (Sec. 3.1, Algorithm 1 recast as a matrix product).
//
// Algorithm 1 sums sign(u_a - u_b) * sign(v_a - v_b) over all sample pairs a < b, which is
// n_c - n_d. Writing A_u[k] = sign(r_u[a_k] - r_u[b_k]) for the k-th sample pair, the numerator of
// every pair of variables is one dot product: S(u, v) = A_u . A_v, i.e. S = A A^T over the upper
// triangle. The {-1, 0, +1} entries are exact in FP4 (e2m1), FP8 (e4m3) and BF16, every product
// is exact, and every partial sum is an integer of magnitude at most n_0 < 2^24 for n <= 5792,
// which an FP32 accumulator holds exactly; the tcgen05 paths were measured to return these sums
// exactly at |S| = n_0 (tests/test_gpu_signgemm.py). n_3 (joint ties) comes from the tie-pair
// lists of the variables (n_3(u, v) = number of sample pairs tied in u that are also tied in v),
// or, for tie-heavy matrices, from a second contraction of the magnitudes:
// |A_u| . |A_v| = n_c + n_d = n_0 - T_u - T_v + n_3.
#pragma once
#include "ktau_impl.cuh"

#define KTAU_SIGNGEMM_MAX_N 5792      // n_0 = n(n-1)/2 < 2^24: exact FP32 accumulation
#define KTAU_SIGNGEMM_FP8_MAX_N 5792
// Longest rows whose n_3 the tie-list tile kernel can count: it stages 33 columns' ranks
// (n x 33 uint16) beside 8192 listed tied pairs in one CTA's shared memory. Longer rows take
// n_3 from the magnitude contraction (FP4 operands, single matrix) or from the merge path.
#define KTAU_SIGNGEMM_TIES_MAX_N 3000
// Variables per CTA of the sign-expansion kernels (their shared memory grows with n).
__host__ __device__ inline int ktau_expand_rows(int64_t n) {
  return n <= 512 ? 8 : (n <= 1024 ? 4 : 2);
}
// Operand row length in elements: n_0 rounded up to whole stages of the contraction (128 elements
// of FP8 / BF16; 256 packed FP4 elements, one 128-byte row of a block-scaled FP4 stage).
__host__ __device__ inline int64_t ktau_kpad(int64_t K, int obits) {
  return obits == 4 ? (K + 255) / 256 * 256 : (K + 127) / 128 * 128;
}
// Operand bits used when the caller does not choose (operand_bits = 0).
#define KTAU_SIGNGEMM_DEFAULT_BITS 4

bool ktau_signgemm_supported(int64_t n);
// Operand bits of the single-matrix and query contraction: 4 (FP4 e2m1), 8 or 16.
int ktau_sign_obits(int64_t n, const ktau_options* opt);
// Builds (once per element size) the sign expansion, the tie-pair lists and the TMA descriptor.
ktau_status ktau_signgemm_prepare(ktau_ranked* R, int obits, cudaStream_t st);
ktau_status ktau_signgemm_allpairs(ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                                   const ktau_out& out, int obits, cudaStream_t st);
// Rectangular form: every row of Q against every row of D (outputs [b][m_db], row stride ldo).
ktau_status ktau_signgemm_rect(ktau_ranked* Q, ktau_ranked* D, const ktau_out& out, int64_t ldo,
                               int obits, cudaStream_t st);
void ktau_signgemm_release(ktau_ranked* R);

// Batched tensor-core group: datasets bids[0..nb) of ds (all FP8 or all BF16), whose rows are
// rows [row0, row0 + rows) of the batch and are stacked in `sgn` (row stride `stride` bytes).
struct ktau_sg_group {
  const ktau_bds* ds;
  const int32_t* bids;
  int nb;
  int esize;                   // operand bytes per element in shared memory (1, or 2 for BF16)
  int obits;                   // operand bits in global memory: 4, 8 or 16
  const int64_t* row_prefix;   // [nb + 1] over the group's rows
  const int64_t* blk_prefix;   // [nb + 1] blocks of ktau_expand_rows(max_n) rows per dataset
  int64_t blocks;
  const int64_t* unit_prefix;  // [nb + 1] contraction units
  const int64_t* jt_prefix;    // [nb + 1] joint-ties tiles
  int64_t rows, units, jt_tiles, max_n;
  const int64_t* T;            // T of the group's rows (contiguous)
  int64_t* tie_off;            // [rows + 1]
  uint32_t* tie_pairs;
  int64_t tie_cap;
  void* sgn;
  int64_t stride;
  const void* tmap;            // CUtensorMap of sgn (host memory, 128 bytes), 128-row boxes
  const void* tmap_b;          // FP4: 120-row boxes for the row operand (else = tmap)
};
// Tensor map of a group's stacked operands, boxes of box_rows rows.
ktau_status ktau_signgemm_make_tmap(void* tmap, void* base, int64_t row_bytes, int64_t rows,
                                    int obits, int box_rows);
// Super-tile side of the pair contraction for this operand type (240 for block-scaled FP4).
int ktau_pair_tile(int obits);
ktau_status ktau_signgemm_batch(const ktau_sg_group& g, cudaStream_t st);
// Device error word of the contraction kernels (bounded waits that gave up); 0 = none.
ktau_status ktau_signgemm_check_error(cudaStream_t st);
