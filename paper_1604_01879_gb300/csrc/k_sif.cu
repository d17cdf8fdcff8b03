// Second inverted file (Fig. 3) and context re-ranking (Eqs. 7, 8, 13, 14).
//
// Build: every database shape p, matched as a query, gives its first k1
// neighbours N_k1(p) (itself included) with memberships F_p[i] = S(x_p, x_i)
// (Eq. 7). The pairs (p, i) are transposed by a stable counting sort keyed
// by i: entry i lists every p with F_p[i] != 0 in ascending p, with the
// membership as uint32 fixed point round(S * 2^31); ||F_p||_1 is the sum of
// p's k1 fixed-point memberships (uint64, exact).
//
// Re-rank: F_q comes from the first k1 candidates of the query. For each
// non-zero F_q[i] the entry i is walked and min(F_q[i], F_p[i]) is added to
// p's numerator (Eq. 13, uint64 atomics: exact and order-free). Then
// S' = num / (||F_q||_1 + ||F_p||_1 - num) (Eq. 14) in FP32, and the final
// order (S' desc, S desc, id asc) is a top-k over 64-bit keys
// (key(S') << 32 | key(S)) with ties to the lower id.
#include "gift_internal.cuh"

namespace gift {

namespace {

__device__ __forceinline__ uint32_t member_fix(float S) {
  const float c = fminf(fmaxf(S, 0.f), 1.f);
  return __float2uint_rn(c * 2147483648.0f);
}

__global__ void k_sif_keys(const int32_t* __restrict__ nbr_ids, int64_t n, int32_t N, int32_t* keys,
                           int* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t id = nbr_ids[i];
  if (id < 0 || id >= N) {
    atomicExch(bad, 1);
    keys[i] = 0;
  } else {
    keys[i] = id;
  }
}

__global__ void k_sif_fill(const int32_t* __restrict__ perm, int64_t n, int k1,
                           const float* __restrict__ nbr_scores, int32_t* __restrict__ ids,
                           uint32_t* __restrict__ mem) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int32_t pair = perm[e];
  ids[e] = pair / k1;
  mem[e] = member_fix(nbr_scores[pair]);
}

__global__ void k_sif_card(const float* __restrict__ nbr_scores, int32_t N, int k1,
                           unsigned long long* __restrict__ card) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  unsigned long long c = 0;
  for (int r = 0; r < k1; ++r) c += member_fix(nbr_scores[p * k1 + r]);
  card[p] = c;
}

__global__ void k_max_entry(const int64_t* __restrict__ off, int32_t N, int* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  atomicMax(out, (int)(off[i + 1] - off[i]));
}

// ||F_q||_1 per query and the dense S row of the candidates (-inf elsewhere)
__global__ void k_rerank_prep(const int32_t* __restrict__ cand_ids, const float* __restrict__ cand_scores,
                              int n_cand, int k1, int32_t N, float* __restrict__ Srow,
                              unsigned long long* __restrict__ fq_norm) {
  const int b = blockIdx.x;
  __shared__ unsigned long long tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < n_cand; t += blockDim.x) {
    const int32_t id = cand_ids[(int64_t)b * n_cand + t];
    const float sc = cand_scores[(int64_t)b * n_cand + t];
    if (id >= 0 && id < N) {
      Srow[(int64_t)b * N + id] = sc;
      if (t < k1) atomicAdd(&tot, (unsigned long long)member_fix(sc));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) fq_norm[b] = tot;
}

// one block per (query, neighbour i): walk S-IF entry i
__global__ void k_rerank_walk(const int32_t* __restrict__ cand_ids, const float* __restrict__ cand_scores,
                              int n_cand, int k1, int32_t N, const int64_t* __restrict__ sif_off,
                              const int32_t* __restrict__ sif_ids, const uint32_t* __restrict__ sif_mem,
                              unsigned long long* __restrict__ num) {
  const int b = blockIdx.x, r = blockIdx.y;
  const int32_t i = cand_ids[(int64_t)b * n_cand + r];
  if (i < 0 || i >= N) return;
  const uint32_t fq = member_fix(cand_scores[(int64_t)b * n_cand + r]);
  if (fq == 0) return;
  const int64_t e0 = sif_off[i], e1 = sif_off[i + 1];
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const uint32_t m = sif_mem[e];
    if (m == 0) continue;
    atomicAdd(num + (int64_t)b * N + sif_ids[e], (unsigned long long)min(fq, m));
  }
}

__global__ void k_rerank_keys(const unsigned long long* __restrict__ num,
                              const unsigned long long* __restrict__ fq_norm,
                              const unsigned long long* __restrict__ card, const float* __restrict__ Srow,
                              int32_t B, int32_t N, unsigned long long* __restrict__ keys) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * N) return;
  const int b = (int)(idx / N);
  const int p = (int)(idx % N);
  const unsigned long long nm = num[idx];
  float sp = 0.f;
  if (nm > 0) {
    const unsigned long long den = fq_norm[b] + card[p] - nm;
    sp = __fdiv_rn(__ull2float_rn(nm), __ull2float_rn(den));
  }
  keys[idx] = ((unsigned long long)f2key(sp) << 32) | (unsigned long long)f2key(Srow[idx]);
}

__global__ void k_keys_to_sprime(const unsigned long long* __restrict__ keys, int64_t n,
                                 float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = keys[i] == 0ull ? -INFINITY : key2f((uint32_t)(keys[i] >> 32));
}

__global__ void k_fill_f32(float* p, int64_t n, float v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

}  // namespace

void sif_build(Index& ix, const int32_t* nbr_ids, const float* nbr_scores, Scratch& sc, cudaStream_t s) {
  const int32_t N = ix.prm.n_shapes;
  const int k1 = ix.k1;
  const int64_t n = (int64_t)N * k1;
  int32_t* keys = sc.get<int32_t>(n);
  int* bad = sc.get<int>(1);
  GIFT_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  k_sif_keys<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(nbr_ids, n, N, keys, bad);
  GIFT_LAUNCHED("k_sif_keys");
  int32_t* perm = sc.get<int32_t>(n);
  int32_t* skeys = sc.get<int32_t>(n);
  stable_sort_by_key(keys, n, N, perm, skeys, sc, s);
  bin_offsets(skeys, n, N, ix.sif_off, s);
  k_sif_fill<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(perm, n, k1, nbr_scores, ix.sif_ids, ix.sif_mem);
  GIFT_LAUNCHED("k_sif_fill");
  k_sif_card<<<(unsigned)cdiv(N, 256), 256, 0, s>>>(nbr_scores, N, k1,
                                                      reinterpret_cast<unsigned long long*>(ix.sif_card));
  GIFT_LAUNCHED("k_sif_card");
  int* mx = sc.get<int>(1);
  GIFT_CUDA(cudaMemsetAsync(mx, 0, sizeof(int), s));
  k_max_entry<<<(unsigned)cdiv(N, 256), 256, 0, s>>>(ix.sif_off, N, mx);
  GIFT_LAUNCHED("k_max_entry");
  int h[2] = {0, 0};
  GIFT_CUDA(cudaMemcpyAsync(&h[0], bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  GIFT_CUDA(cudaMemcpyAsync(&h[1], mx, sizeof(int), cudaMemcpyDeviceToHost, s));
  GIFT_CUDA(cudaStreamSynchronize(s));
  if (h[0]) fail(GIFT_EINVAL, "S-IF build: a database shape has fewer than k1 neighbours");
  ix.max_sif_entry = h[1];
}

void sif_rerank(const Index& ix, const int32_t* cand_ids, const float* cand_scores, int32_t B, int32_t n_cand,
                int32_t k1, int32_t topk, int32_t* out_ids, float* out_sprime, Scratch& sc, cudaStream_t s) {
  const int32_t N = ix.prm.n_shapes;
  const int64_t BN = (int64_t)B * N;
  unsigned long long* num = sc.get<unsigned long long>(BN);
  GIFT_CUDA(cudaMemsetAsync(num, 0, BN * 8, s));
  float* Srow = sc.get<float>(BN);
  k_fill_f32<<<(unsigned)cdiv(BN, 256), 256, 0, s>>>(Srow, BN, -INFINITY);
  GIFT_LAUNCHED("k_fill_f32");
  unsigned long long* fqn = sc.get<unsigned long long>(B);
  k_rerank_prep<<<(unsigned)B, 256, 0, s>>>(cand_ids, cand_scores, n_cand, k1, N, Srow, fqn);
  GIFT_LAUNCHED("k_rerank_prep");
  k_rerank_walk<<<dim3((unsigned)B, (unsigned)k1), 128, 0, s>>>(cand_ids, cand_scores, n_cand, k1, N, ix.sif_off,
                                                             ix.sif_ids, ix.sif_mem, num);
  GIFT_LAUNCHED("k_rerank_walk");
  unsigned long long* keys = sc.get<unsigned long long>(BN);
  k_rerank_keys<<<(unsigned)cdiv(BN, 256), 256, 0, s>>>(num, fqn,
                                                          reinterpret_cast<const unsigned long long*>(ix.sif_card),
                                                          Srow, B, N, keys);
  GIFT_LAUNCHED("k_rerank_keys");
  unsigned long long* kout = sc.get<unsigned long long>((int64_t)B * topk);
  topk_rows_u64(reinterpret_cast<const uint64_t*>(keys), B, N, topk, out_ids,
                reinterpret_cast<uint64_t*>(kout), sc, s);
  k_keys_to_sprime<<<(unsigned)cdiv((int64_t)B * topk, 256), 256, 0, s>>>(kout, (int64_t)B * topk, out_sprime);
  GIFT_LAUNCHED("k_keys_to_sprime");
}

namespace {
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace

size_t sif_rerank_scratch_bytes(int32_t B, int32_t N, int32_t topk) {
  const size_t BN = (size_t)B * (size_t)N;
  return align256(BN * 8) + align256(BN * 4) + align256((size_t)B * 8) + align256(BN * 8) +
         align256((size_t)B * (size_t)topk * 8);
}

// The re-rank of sif_rerank on scratch the caller provides (no allocation):
// the same kernels, with the numerator cleared and the candidate row filled
// before use, so nothing depends on what the scratch held before.
void sif_rerank_into(const Index& ix, const int32_t* cand_ids, const float* cand_scores, int32_t B, int32_t n_cand,
                     int32_t k1, int32_t topk, int32_t* out_ids, float* out_sprime, void* scratch,
                     size_t scratch_bytes, cudaStream_t s) {
  const int32_t N = ix.prm.n_shapes;
  const int64_t BN = (int64_t)B * N;
  GIFT_REQUIRE(sif_rerank_scratch_bytes(B, N, topk) <= scratch_bytes, "re-rank scratch too small");
  uint8_t* p = static_cast<uint8_t*>(scratch);
  unsigned long long* num = reinterpret_cast<unsigned long long*>(p);
  p += align256((size_t)BN * 8);
  float* Srow = reinterpret_cast<float*>(p);
  p += align256((size_t)BN * 4);
  unsigned long long* fqn = reinterpret_cast<unsigned long long*>(p);
  p += align256((size_t)B * 8);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(p);
  p += align256((size_t)BN * 8);
  unsigned long long* kout = reinterpret_cast<unsigned long long*>(p);
  GIFT_CUDA(cudaMemsetAsync(num, 0, BN * 8, s));
  k_fill_f32<<<(unsigned)cdiv(BN, 256), 256, 0, s>>>(Srow, BN, -INFINITY);
  GIFT_LAUNCHED("k_fill_f32");
  k_rerank_prep<<<(unsigned)B, 256, 0, s>>>(cand_ids, cand_scores, n_cand, k1, N, Srow, fqn);
  GIFT_LAUNCHED("k_rerank_prep");
  k_rerank_walk<<<dim3((unsigned)B, (unsigned)k1), 128, 0, s>>>(cand_ids, cand_scores, n_cand, k1, N, ix.sif_off,
                                                             ix.sif_ids, ix.sif_mem, num);
  GIFT_LAUNCHED("k_rerank_walk");
  k_rerank_keys<<<(unsigned)cdiv(BN, 256), 256, 0, s>>>(num, fqn,
                                                          reinterpret_cast<const unsigned long long*>(ix.sif_card),
                                                          Srow, B, N, keys);
  GIFT_LAUNCHED("k_rerank_keys");
  Scratch none(s);  // the selection kernel takes a scratch handle but allocates nothing
  topk_rows_u64(reinterpret_cast<const uint64_t*>(keys), B, N, topk, out_ids, reinterpret_cast<uint64_t*>(kout),
                none, s);
  k_keys_to_sprime<<<(unsigned)cdiv((int64_t)B * topk, 256), 256, 0, s>>>(kout, (int64_t)B * topk, out_sprime);
  GIFT_LAUNCHED("k_keys_to_sprime");
}

}  // namespace gift
