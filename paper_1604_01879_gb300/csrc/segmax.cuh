// Segmented-max contraction shared by the exact match and the projected match.
#pragma once
#include "gift_internal.cuh"

namespace gift {

// S[b, p] (and argmax) from the per-(view, shape) cells of queries [b0, b0 + nq)
void segmax_reduce(const unsigned long long* cell, int64_t n_shapes, const int32_t* d_qoff, int32_t b0, int32_t nq,
                   int32_t view0, float* S, int16_t* argmax, cudaStream_t s);

// Segmented max on the tensor cores from two-part BF16 operands (rows of A =
// query views, rows of B = database views, nv per shape); each operand has at
// least one TMA box of rows (a_rows_alloc, b_rows_alloc >= 128).
void segmax_tc(const __nv_bfloat16* a_hi, const __nv_bfloat16* a_lo, int64_t a_rows_alloc, const float* a_inv,
               const __nv_bfloat16* b_hi, const __nv_bfloat16* b_lo, int64_t b_rows_alloc, const float* b_inv,
               int64_t ncols, int nv, int D, const int32_t* d_qoff, const std::vector<int32_t>& h_qoff, int32_t B,
               float* S, int16_t* argmax, int* err, Scratch& sc, cudaStream_t s);

}  // namespace gift
