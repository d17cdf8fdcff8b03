// Plain GEMM on the tcgen05 engine: C[M, N] (+)= A[M, K] * B[N, K]^T with
// A, B K-major BF16 (SPLIT = 1), two-part BF16 (SPLIT = 3: hi*hi + hi*lo +
// lo*hi, FP32-level), or a two-part A with a B exact in BF16 (SPLIT = 2:
// hi*b + lo*b), FP32 output. The reduction runs in chunks of at most 16
// k-blocks, each accumulated in its own TMEM buffer and summed in FP32 by the
// epilogue (bounds the steps that feed one tensor-core accumulator).
// Work items run along the longer side: with more row tiles than column
// tiles they run row-tile-major, so the CTAs working at the same time share
// each A tile (read from memory once) and all of B; otherwise column-tile-
// major, sharing the B tile.
#pragma once
#include "tc_engine.cuh"

namespace gift {

template <int SPLIT_>
struct GemmPolicy {
  static constexpr int TN = 128, NBUF = 4, STAGES = SPLIT_ == 1 ? 6 : SPLIT_ == 2 ? 4 : 3, SPLIT = SPLIT_, EB = 2;
  static constexpr int kWarpSmem = 16;
  int64_t M, N;
  int nkb;
  float* C;
  int64_t ldc;
  int accumulate;
  bool row_major;  // item order: row tile slow (true) or column tile slow
  struct Item {
    int64_t r0, c0;
    int nr, nc;
  };
  struct Ctx {
    float sum[TN];
  };
  __device__ __forceinline__ int64_t n_mt() const { return cdiv(M, tc::kTM); }
  __device__ __forceinline__ int64_t total() const { return n_mt() * cdiv(N, TN); }
  __device__ __forceinline__ Item decode(int64_t item) const {
    Item it;
    const int64_t mt = n_mt(), nt = cdiv(N, TN);
    const int64_t ct = row_major ? item % nt : item / mt, rt = row_major ? item / nt : item % mt;
    it.r0 = rt * tc::kTM;
    it.c0 = ct * TN;
    it.nr = (int)min((int64_t)tc::kTM, M - it.r0);
    it.nc = (int)min((int64_t)TN, N - it.c0);
    return it;
  }
  // chunks bound the MMA steps feeding one accumulator (about 192, 3 products
  // x 4 sub-steps per k-block), however long the reduction (the weight
  // gradient reduces over every database view); short reductions use one chunk
  __device__ __forceinline__ int nch() const {
    const int want = (nkb * 12 + 191) / 192;
    return want < 1 ? 1 : want;
  }
  __device__ __forceinline__ int nchunks(const Item&) const { return nch(); }
  __device__ __forceinline__ void chunk(const Item& it, int c, int& br, int& kb0, int& kb1) const {
    const int nch = this->nch();
    br = (int)it.c0;
    kb0 = (int)((int64_t)nkb * c / nch);
    kb1 = (int)((int64_t)nkb * (c + 1) / nch);
  }
  __device__ __forceinline__ int a_row(const Item& it) const { return (int)it.r0; }
  __device__ __forceinline__ void epi_begin(const Item&, Ctx& x, int, int, uint8_t*) const {
#pragma unroll
    for (int j = 0; j < TN; ++j) x.sum[j] = 0.f;
  }
  __device__ __forceinline__ void epi_chunk(const Item&, int, uint32_t taddr, Ctx& x, int, uint8_t*) const {
#pragma unroll
    for (int pc = 0; pc < TN / 32; ++pc) {
      uint32_t r[32];
      tc::tmem_ld32(taddr + pc * 32, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 32; ++j) x.sum[pc * 32 + j] += __uint_as_float(r[j]);
    }
  }
  __device__ __forceinline__ void epi_end(const Item& it, Ctx& x, int m, uint8_t*) const {
    if (m >= it.nr) return;
    float* crow = C + (it.r0 + m) * ldc + it.c0;
    if (it.nc == TN && (ldc % 4) == 0 && ((it.c0 % 4) == 0)) {
#pragma unroll
      for (int j = 0; j < TN; j += 4) {
        float4 v = make_float4(x.sum[j], x.sum[j + 1], x.sum[j + 2], x.sum[j + 3]);
        float4* dst = reinterpret_cast<float4*>(crow + j);
        if (accumulate) {
          const float4 o = *dst;
          v.x += o.x;
          v.y += o.y;
          v.z += o.z;
          v.w += o.w;
        }
        *dst = v;
      }
    } else {
#pragma unroll
      for (int j = 0; j < TN; ++j)
        if (j < it.nc) crow[j] = accumulate ? crow[j] + x.sum[j] : x.sum[j];
    }
  }
};

// Two-part (SPLIT 3), two-part A with one-part B (SPLIT 2, b_lo null) or
// one-part (SPLIT 1, both lo parts null) BF16 operands; a_rows_alloc /
// b_rows_alloc are the rows the tensor maps cover (rows past M or N read as
// zeros); lda / ldb are row pitches in elements (0 = K): C[M, N] (+)= A * B^T.
void gemm_tc(const __nv_bfloat16* a_hi, const __nv_bfloat16* a_lo, int64_t M, int64_t a_rows_alloc, int64_t lda,
             const __nv_bfloat16* b_hi, const __nv_bfloat16* b_lo, int64_t N, int64_t b_rows_alloc, int64_t ldb, int K,
             float* C, int64_t ldc, int accumulate, int* err, cudaStream_t s);

}  // namespace gift
