// Exact set-to-set match (Eq. 3): S(x_q, x_p) = (1/|V(x_q)|) sum_i max_j s(q_i, p_j).
//
// A tile GEMM of query views [rows] against database views [cols] produces
// cosines; the epilogue reduces each row over every run of columns that
// belongs to one database shape (N_v consecutive columns) and folds the
// partial maximum (and the first view attaining it) into a per-(view, shape)
// cell with a 64-bit atomicMax on (order-preserving key of s, 0xFFFF - j).
// A second kernel sums the cells over each query's views.
#include "gift_internal.cuh"
#include "segmax.cuh"
#include "sgemm_nt.cuh"

namespace gift {

namespace {

struct EpiSegmax {
  const float* inv_a;  // [M]
  const float* inv_b;  // [N]
  int64_t M, N;
  int nv;              // columns per shape
  int64_t n_shapes;
  unsigned long long* cell;  // [M, n_shapes]
  __device__ __forceinline__ void operator()(int64_t m0, int64_t n0, const SgemmFrag& f,
                                             float (&acc)[8][8]) const {
    extern __shared__ float T[];  // [128][129]
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = f.row(i);
      const int64_t m = m0 + r;
      const float ia = m < M ? inv_a[m] : 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = f.col(j);
        const int64_t n = n0 + c;
        T[r * 129 + c] = (m < M && n < N) ? acc[i][j] * ia * inv_b[n] : 0.f;
      }
    }
    __syncthreads();
    const int tid = threadIdx.x;
    const int r = tid & 127, half = tid >> 7;
    const int64_t m = m0 + r;
    if (m >= M) return;
    for (int c = half * 64; c < half * 64 + 64; ++c) {
      const int64_t n = n0 + c;
      if (n >= N) break;
      if (c != 0 && (n % nv) != 0) continue;  // not the start of a shape run
      const int64_t shape = n / nv;
      float best = T[r * 129 + c];
      int bj = (int)(n % nv);
      int c2 = c + 1;
      for (; c2 < 128; ++c2) {
        const int64_t n2 = n0 + c2;
        if (n2 >= N || (n2 % nv) == 0) break;
        const float v = T[r * 129 + c2];
        if (v > best) {
          best = v;
          bj = (int)(n2 % nv);
        }
      }
      const unsigned long long key =
          ((unsigned long long)f2key(best) << 32) | (unsigned long long)(0xFFFFu - (unsigned)bj);
      atomicMax(cell + m * n_shapes + shape, key);
    }
  }
};

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

void segmax_scores(const float* A, const float* inv_a, int64_t n_views, const float* Bm,
                   const float* inv_b, int64_t n_shapes, int nv, int D, const int32_t* d_qoff,
                   const std::vector<int32_t>& h_qoff, int32_t Bq, float* S, int16_t* argmax,
                   Scratch& sc, cudaStream_t s) {
  if (Bq <= 0 || n_shapes <= 0) return;
  const int64_t ncols = n_shapes * nv;
  // views per pass: the cell block stays under 1 GiB
  const int64_t cap = std::max<int64_t>(1, ((int64_t)1 << 27) / n_shapes);
  unsigned long long* cell = nullptr;
  int64_t cell_rows = 0;
  GIFT_CUDA(cudaFuncSetAttribute(k_sgemm_nt<EpiSegmax>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 128 * 129 * 4));
  int32_t b0 = 0;
  while (b0 < Bq) {
    int32_t b1 = b0 + 1;
    while (b1 < Bq && (int64_t)(h_qoff[b1 + 1] - h_qoff[b0]) <= cap) ++b1;
    const int32_t v0 = h_qoff[b0], v1 = h_qoff[b1];
    const int64_t rows = v1 - v0;
    if (rows > cell_rows) {
      cell = sc.get<unsigned long long>((size_t)rows * n_shapes);
      cell_rows = rows;
    }
    GIFT_CUDA(cudaMemsetAsync(cell, 0, (size_t)rows * n_shapes * 8, s));
    EpiSegmax epi{inv_a + v0, inv_b, rows, ncols, nv, n_shapes, cell};
    launch_sgemm_nt(A + (int64_t)v0 * D, rows, Bm, ncols, D, epi, 128 * 129 * 4, s);
    const int64_t work = (int64_t)(b1 - b0) * n_shapes;
    k_segmax_reduce<<<(unsigned)cdiv(work, 256), 256, 0, s>>>(cell, n_shapes, d_qoff, b0, b1 - b0, v0, S,
                                                             argmax);
    GIFT_LAUNCHED("k_segmax_reduce");
    b0 = b1;
  }
}

}  // namespace gift
