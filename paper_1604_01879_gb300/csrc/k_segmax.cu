// Per-query sums of the per-(query view, shape) maxima of Eq. 3: each cell holds
// a 64-bit key (order-preserving key of the max cosine, 0xFFFF - j of the first
// view attaining it), filled by the tensor-core segmented max; the reduction
// averages a query's cells into S(x_q, x_p) and writes the argmax views.
#include "gift_internal.cuh"
#include "segmax.cuh"

namespace gift {

namespace {

__global__ void k_segmax_reduce(const unsigned long long* __restrict__ cell, int64_t n_shapes,
                                const int32_t* __restrict__ qoff, int32_t qb0, int32_t nq,
                                int32_t view0, float* __restrict__ S, int16_t* __restrict__ argmax) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nq * n_shapes) return;
  const int32_t b = qb0 + (int32_t)(idx / n_shapes);
  const int64_t p = idx % n_shapes;
  const int32_t v0 = qoff[b], v1 = qoff[b + 1];
  float sum = 0.f;
  for (int32_t v = v0; v < v1; ++v) {
    const unsigned long long key = cell[(int64_t)(v - view0) * n_shapes + p];
    sum += key2f((uint32_t)(key >> 32));
    if (argmax) argmax[(int64_t)v * n_shapes + p] = (int16_t)(0xFFFFu - (unsigned)(key & 0xFFFFu));
  }
  S[(int64_t)b * n_shapes + p] = sum / (float)(v1 - v0);
}

}  // namespace

void segmax_reduce(const unsigned long long* cell, int64_t n_shapes, const int32_t* d_qoff, int32_t b0, int32_t nq,
                   int32_t view0, float* S, int16_t* argmax, cudaStream_t s) {
  const int64_t work = (int64_t)nq * n_shapes;
  if (work <= 0) return;
  k_segmax_reduce<<<(unsigned)cdiv(work, 256), 256, 0, s>>>(cell, n_shapes, d_qoff, b0, nq, view0, S, argmax);
  GIFT_LAUNCHED("k_segmax_reduce");
}

}  // namespace gift
