// FP32 CUDA-core tile GEMM, C = A * B^T with A [M, K] and B [N, K] both
// row-major (K contiguous), 128x128 tiles, 256 threads, 8x8 outputs per
// thread, double-buffered shared memory. The epilogue is a functor that
// receives the thread's accumulators; it decides what is stored.
#pragma once
#include "gift_internal.cuh"

namespace gift {

struct SgemmFrag {
  // rows of the thread's outputs: m0 + row(i), i < 8; cols: n0 + col(j), j < 8
  int tx, ty;
  __device__ __forceinline__ int row(int i) const { return (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4); }
  __device__ __forceinline__ int col(int j) const { return (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4); }
};

// Requires K % 4 == 0 and 16-byte aligned rows.
template <class Epi>
__global__ __launch_bounds__(256, 2) void k_sgemm_nt(const float* __restrict__ A, int64_t M,
                                                      const float* __restrict__ B, int64_t N, int K,
                                                      Epi epi) {
  __shared__ __align__(16) float As[2][8][128];
  __shared__ __align__(16) float Bs[2][8][128];
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.y * 128;
  const int64_t n0 = (int64_t)blockIdx.x * 128;
  const int lr = tid >> 1, lk = (tid & 1) * 4;
  const bool aok = m0 + lr < M;
  const bool bok = n0 + lr < N;
  const float* Ap = A + (aok ? (m0 + lr) : 0) * (int64_t)K + lk;
  const float* Bp = B + (bok ? (n0 + lr) : 0) * (int64_t)K + lk;
  float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra;
  const float4 z4 = ra;

  auto gload = [&](int k0) {
    const bool kin = k0 + lk < K;
    ra = (aok && kin) ? __ldg(reinterpret_cast<const float4*>(Ap + k0)) : z4;
    rb = (bok && kin) ? __ldg(reinterpret_cast<const float4*>(Bp + k0)) : z4;
  };
  auto sstore = [&](int buf) {
    As[buf][lk + 0][lr] = ra.x;
    As[buf][lk + 1][lr] = ra.y;
    As[buf][lk + 2][lr] = ra.z;
    As[buf][lk + 3][lr] = ra.w;
    Bs[buf][lk + 0][lr] = rb.x;
    Bs[buf][lk + 1][lr] = rb.y;
    Bs[buf][lk + 2][lr] = rb.z;
    Bs[buf][lk + 3][lr] = rb.w;
  };

  SgemmFrag f{tid & 15, tid >> 4};
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  gload(0);
  sstore(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += 8) {
    const bool more = k0 + 8 < K;
    if (more) gload(k0 + 8);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][f.ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + f.ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][f.tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + f.tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      sstore(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  epi(m0, n0, f, acc);
}

template <class Epi>
inline void launch_sgemm_nt(const float* A, int64_t M, const float* B, int64_t N, int K, Epi epi,
                            size_t smem, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((unsigned)cdiv(N, 128), (unsigned)cdiv(M, 128));
  GIFT_REQUIRE(grid.y <= 65535u, "sgemm: too many row tiles");
  k_sgemm_nt<Epi><<<grid, 256, smem, s>>>(A, M, B, N, K, epi);
  GIFT_LAUNCHED("k_sgemm_nt");
}

}  // namespace gift
