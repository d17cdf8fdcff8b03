// Off-line vocabulary on the GPU: Lloyd's k-means (Sec. 2.3 trains the
// codebook of the first inverted file with k-means and gives no details).
//
// Iteration: every row goes to its nearest centre through the exact
// quantiser (tensor-core coarse scores + two-float refine, ties to the lowest
// index); rows are grouped by centre with a stable sort, and each centre
// becomes the mean of its rows, summed in two-float (compensated FP32)
// arithmetic in ascending row order (so the result does not depend on
// scheduling; no FP64 on the GPU). A centre left without rows takes
// the row farthest from the centre it was assigned to (distance desc, index
// asc), the empty centres served in ascending order.
#include "gift_internal.cuh"

namespace gift {

namespace {

// one block per centre: mean of its rows (perm[off[c] .. off[c+1]) ascending), two-float sums
__global__ void k_km_mean(const float* __restrict__ X, int D, const int32_t* __restrict__ perm,
                          const int64_t* __restrict__ off, const float* __restrict__ C_old,
                          float* __restrict__ C_new) {
  const int c = blockIdx.x;
  const int64_t r0 = off[c], r1 = off[c + 1];
  for (int d = threadIdx.x; d < D; d += blockDim.x) {
    if (r1 == r0) {  // empty: keep the old centre until it is re-seeded
      C_new[(int64_t)c * D + d] = C_old[(int64_t)c * D + d];
      continue;
    }
    F2 s;
    for (int64_t e = r0; e < r1; ++e) f2_add(s, X[(int64_t)perm[e] * D + d]);
    // (hi + lo) / n: the quotient of the two-float sum, rounded once more
    const float n = (float)(r1 - r0);
    const float q = __fdiv_rn(s.hi, n);
    const float rem = __fmaf_rn(-q, n, s.hi);  // s.hi - q n exactly (n < 2^24)
    C_new[(int64_t)c * D + d] = q + __fdiv_rn(rem + s.lo, n);
  }
}

// squared distance of every row to its assigned centre (warp per row, two-float):
// t = x - c exactly as th + tl (TwoSum), t^2 = th^2 + 2 th tl + tl^2 with the
// rounding error of th^2 recovered by an FMA
__global__ void k_km_dist(const float* __restrict__ X, int64_t n, int D, const float* __restrict__ C,
                          const int32_t* __restrict__ lab, float* __restrict__ dist) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const float* x = X + r * D;
  const float* c = C + (int64_t)lab[r] * D;
  F2 s;
  for (int d = lane; d < D; d += 32) {
    float th, tl;
    two_sum(x[d], -c[d], th, tl);
    const float p = th * th;
    const float pe = __fmaf_rn(th, th, -p);
    f2_add(s, p);
    s.lo += pe + tl * (2.f * th + tl);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = f2_merge(s, f2_shfl_xor(s, o));
  if (lane == 0) dist[r] = f2_value(s);
}

__global__ void k_km_rows(const float* __restrict__ X, int D, const int32_t* __restrict__ rows,
                          int64_t n_rows, float* __restrict__ out) {
  const int64_t i = blockIdx.x;
  if (i >= n_rows) return;
  for (int d = threadIdx.x; d < D; d += blockDim.x) out[i * D + d] = X[(int64_t)rows[i] * D + d];
}

}  // namespace

void kmeans(const float* X, int64_t n, int D, int K, const std::vector<int32_t>& init_rows, int iters, float* C_out,
            Scratch& sc, cudaStream_t s) {
  Index tmp;  // the quantiser's view of the current centres
  tmp.prm.n_codewords = K;
  tmp.prm.dim = D;
  GIFT_CUDA(cudaGetDevice(&tmp.device));
  tmp.codebook = tmp.alloc<float>((size_t)K * D);
  tmp.d_err = tmp.alloc<int>(1);
  GIFT_CUDA(cudaMemsetAsync(tmp.d_err, 0, sizeof(int), s));
  int32_t* d_init = sc.get<int32_t>(K);
  GIFT_CUDA(cudaMemcpyAsync(d_init, init_rows.data(), (size_t)K * 4, cudaMemcpyHostToDevice, s));
  k_km_rows<<<(unsigned)K, 256, 0, s>>>(X, D, d_init, K, tmp.codebook);
  GIFT_LAUNCHED("k_km_rows");
  float* x_inv = sc.get<float>(n);
  launch_row_invnorm(X, n, D, x_inv, s);
  float* C_new = sc.get<float>((size_t)K * D);
  int32_t* lab = sc.get<int32_t>(n);
  int32_t* perm = sc.get<int32_t>(n);
  int32_t* skeys = sc.get<int32_t>(n);
  int64_t* off = sc.get<int64_t>((size_t)K + 1);
  float* dist = sc.get<float>(n);
  std::vector<int64_t> h_off((size_t)K + 1);
  for (int it = 0; it < iters; ++it) {
    prepare_codebook(tmp, s);
    assign_codes(tmp, X, n, 1, lab, sc, s, x_inv);
    stable_sort_by_key(lab, n, K, perm, skeys, sc, s);
    bin_offsets(skeys, n, K, off, s);
    k_km_mean<<<(unsigned)K, 256, 0, s>>>(X, D, perm, off, tmp.codebook, C_new);
    GIFT_LAUNCHED("k_km_mean");
    GIFT_CUDA(cudaMemcpyAsync(h_off.data(), off, ((size_t)K + 1) * 8, cudaMemcpyDeviceToHost, s));
    GIFT_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> empty;
    for (int c = 0; c < K; ++c)
      if (h_off[c + 1] == h_off[c]) empty.push_back(c);
    if (!empty.empty()) {
      const int E = (int)empty.size();
      k_km_dist<<<(unsigned)cdiv(n, 8), 256, 0, s>>>(X, n, D, tmp.codebook, lab, dist);
      GIFT_LAUNCHED("k_km_dist");
      int32_t* far = sc.get<int32_t>(E);
      topk_rows_f32(dist, 1, n, E, far, nullptr, sc, s);  // distance desc, index asc
      std::vector<int32_t> h_far(E);
      GIFT_CUDA(cudaMemcpyAsync(h_far.data(), far, (size_t)E * 4, cudaMemcpyDeviceToHost, s));
      GIFT_CUDA(cudaStreamSynchronize(s));
      for (int e = 0; e < E; ++e)
        GIFT_CUDA(cudaMemcpyAsync(C_new + (int64_t)empty[e] * D, X + (int64_t)h_far[e] * D, (size_t)D * 4,
                                  cudaMemcpyDeviceToDevice, s));
    }
    GIFT_CUDA(cudaMemcpyAsync(tmp.codebook, C_new, (size_t)K * D * 4, cudaMemcpyDeviceToDevice, s));
  }
  GIFT_CUDA(cudaMemcpyAsync(C_out, tmp.codebook, (size_t)K * D * 4, cudaMemcpyDefault, s));
  GIFT_CUDA(cudaStreamSynchronize(s));
}

}  // namespace gift
