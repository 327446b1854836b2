// K-c: exact sign-matrix contraction (Sec. 3.1, Algorithm 1 recast as a matrix product).
#pragma once
#include "ktau_impl.cuh"

#define KTAU_SIGNGEMM_MAX_N 1024

bool ktau_signgemm_supported(int64_t n);
ktau_status ktau_signgemm_allpairs(ktau_ranked* R, uint64_t p_begin, uint64_t p_end,
                                   const ktau_out& out, cudaStream_t st);
void ktau_signgemm_release(ktau_ranked* R);
