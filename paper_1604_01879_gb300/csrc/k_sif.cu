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
//
// Two measures (Sec. 2.4, Eqs. 9-11): a block per shape (database or query)
// gathers the activations that make up its two contextual activations — its
// own Eq. 7 rows, or the Eq. 7 rows of its first k2 neighbours under the same
// measure (Eq. 10) or the other one (Eq. 11) — as (id, measure, source) keys,
// sorts them in shared memory, sums each (id, measure) group in source order
// and divides by k2, and fuses the two measures per id with the generalised
// mean of Eq. 9. The database activations are transposed into a second
// inverted file of their own; a query's activation is walked through it as in
// the one-measure re-rank.
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

// The shapes a query reaches -- through the S-IF walk (numerator > 0) or as a
// candidate (finite S) -- in ascending id order, with their ranking keys (as
// k_rerank_keys); every other shape has the same key, S' = 0 and S = -inf,
// below all of these, so the top-k of the dense row is the top-k of this
// compact row, followed (when fewer than min(topk, N) shapes are reached) by the
// unreached shapes in ascending id order. One block per query, rows of `cap`
// (padding: key 0, id -1).
constexpr int kCompactT = 1024;
__global__ __launch_bounds__(kCompactT) void k_rerank_compact(
    const unsigned long long* __restrict__ num, const unsigned long long* __restrict__ fq_norm,
    const unsigned long long* __restrict__ card, const float* __restrict__ Srow, int32_t N, int64_t cap, int need,
    int32_t* __restrict__ ids, unsigned long long* __restrict__ keys) {
  __shared__ int wtot[kCompactT / 32];
  __shared__ int s_count;
  const int b = blockIdx.x, t = threadIdx.x, w = t >> 5, lane = t & 31;
  const unsigned long long* nr = num + (int64_t)b * N;
  const float* sr = Srow + (int64_t)b * N;
  int32_t* oid = ids + (int64_t)b * cap;
  unsigned long long* okey = keys + (int64_t)b * cap;
  const unsigned long long fq = fq_norm[b];
  if (t == 0) s_count = 0;
  __syncthreads();
  // pass 0: the reached shapes; pass 1 (only when too few): the first unreached ones
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1 && s_count >= need) break;  // block-uniform (read after a barrier)
    for (int c0 = 0; c0 < N; c0 += kCompactT) {
      const int p = c0 + t;
      bool in = false;
      unsigned long long key = 0;
      if (p < N) {
        const unsigned long long nm = nr[p];
        const float sv = sr[p];
        const bool reached = nm != 0ull || sv != -INFINITY;
        in = pass == 0 ? reached : !reached;
        if (in) {
          float sp = 0.f;
          if (nm > 0) sp = __fdiv_rn(__ull2float_rn(nm), __ull2float_rn(fq + card[p] - nm));
          key = ((unsigned long long)f2key(sp) << 32) | (unsigned long long)f2key(sv);
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (lane == 0) wtot[w] = __popc(m);
      __syncthreads();
      if (w == 0) {  // exclusive scan of the warp totals
        const int x = wtot[lane];
        int y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int z = __shfl_up_sync(0xffffffffu, y, o);
          if (lane >= o) y += z;
        }
        wtot[lane] = y - x;
      }
      __syncthreads();
      const int base = s_count;
      const int pos = base + wtot[w] + __popc(m & ((1u << lane) - 1u));
      const int limit = pass == 0 ? (int)cap : need;
      if (in && pos < limit) {
        oid[pos] = p;
        okey[pos] = key;
      }
      __syncthreads();
      if (t == kCompactT - 1) s_count = min(limit, pos + (in ? 1 : 0));
      __syncthreads();
      if (pass == 1 && s_count >= need) break;  // block-uniform
    }
    __syncthreads();
  }
  for (int64_t j = s_count + t; j < cap; j += kCompactT) {
    oid[j] = -1;
    okey[j] = 0ull;
  }
}

// output of the selection over compact rows: positions -> shape ids, keys -> S'
__global__ void k_rerank_out(const int32_t* __restrict__ pos, const unsigned long long* __restrict__ kout,
                             const int32_t* __restrict__ ids, int64_t cap, int32_t B, int32_t topk,
                             int32_t* __restrict__ out_ids, float* __restrict__ out_sprime) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * topk) return;
  const int64_t b = i / topk;
  const int32_t q = pos[i];
  const bool ok = q >= 0 && kout[i] != 0ull;
  out_ids[i] = ok ? ids[b * cap + q] : -1;
  out_sprime[i] = ok ? key2f((uint32_t)(kout[i] >> 32)) : -INFINITY;
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

// ---------------------------------------------------------------- two measures
constexpr int kAcaT = 256;
constexpr int kAcaMaxP = 4096;  // sorted pairs per shape (shared memory: 16 B each)

struct AcaRowArgs {
  int mode, k1, k2, cap, nmax, P;
  float alpha;
  int32_t N;
  const int32_t* db_ids[2];  // [N, k1] ranked neighbours of every database shape, per measure
  const float* db_sc[2];     // [N, k1] their scores
  const int32_t* nb[2];      // ranking of this row under measure l (row stride ld)
  const float* own_sc[2];    // scores aligned with nb (mode 0)
  int64_t ld;
  int32_t* out_ids;          // [rows, cap] ascending ids of the non-zero coordinates
  uint32_t* out_mem;         // [rows, cap] fixed-point activation
  int32_t* out_cnt;          // [rows]
  unsigned long long* out_norm;  // [rows] ||F||_1, fixed point
};

__device__ __forceinline__ float gen_mean(float a, float b, float alpha) {
  if (alpha == 0.5f) {
    const float r = 0.5f * (sqrtf(a) + sqrtf(b));
    return r * r;
  }
  if (alpha == 1.f) return 0.5f * (a + b);
  const float m = 0.5f * (powf(a, alpha) + powf(b, alpha));
  return m > 0.f ? powf(m, 1.f / alpha) : 0.f;
}

__global__ __launch_bounds__(kAcaT) void k_aca_rows(const AcaRowArgs a) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint64_t* key = reinterpret_cast<uint64_t*>(sm);
  float* val = reinterpret_cast<float*>(key + a.P);
  int* pos = reinterpret_cast<int*>(val + a.P);
  __shared__ int part[kAcaT];
  __shared__ unsigned long long norm;
  const int64_t r = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) norm = 0ull;
  // gather: measure l occupies [l * nmax, (l + 1) * nmax)
  for (int t = tid; t < a.P; t += kAcaT) {
    uint64_t k = ~0ull;
    float v = 0.f;
    if (t < 2 * a.nmax) {
      const int l = t / a.nmax, u = t % a.nmax;
      int32_t id = -1;
      if (a.mode == 0) {
        id = a.nb[l][r * a.ld + u];
        v = a.own_sc[l][r * a.ld + u];
      } else {
        const int src_l = a.mode == 1 ? l : 1 - l;
        const int32_t src = a.nb[src_l][r * a.ld + u / a.k1];
        if (src >= 0 && src < a.N) {
          id = a.db_ids[l][(int64_t)src * a.k1 + u % a.k1];
          v = a.db_sc[l][(int64_t)src * a.k1 + u % a.k1];
        }
      }
      if (id >= 0 && id < a.N) k = ((uint64_t)(uint32_t)id << 32) | ((uint64_t)l << 31) | (uint64_t)u;
    }
    key[t] = k;
    val[t] = v;
  }
  __syncthreads();
  // bitonic sort of (key, val), ascending
  for (int size = 2; size <= a.P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = tid; t < a.P; t += kAcaT) {
        const int o = t ^ stride;
        if (o > t) {
          const bool up = (t & size) == 0;
          const uint64_t x = key[t], y = key[o];
          if ((x > y) == up) {
            key[t] = y;
            key[o] = x;
            const float tv = val[t];
            val[t] = val[o];
            val[o] = tv;
          }
        }
      }
      __syncthreads();
    }
  }
  // heads of id groups, block-wide exclusive scan over each thread's consecutive chunk
  const int per = a.P / kAcaT;
  const int c0 = tid * per;
  int cnt = 0;
  for (int t = c0; t < c0 + per; ++t) {
    const uint64_t k = key[t];
    const bool head = k != ~0ull && (t == 0 || (key[t - 1] >> 32) != (k >> 32));
    pos[t] = head ? 1 : 0;
    cnt += head;
  }
  part[tid] = cnt;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int i = 0; i < kAcaT; ++i) {
      const int c = part[i];
      part[i] = run;
      run += c;
    }
    a.out_cnt[r] = run;
  }
  __syncthreads();
  int o = part[tid];
  const float div = a.mode == 0 ? 1.f : (float)a.k2;
  for (int t = c0; t < c0 + per; ++t) {
    if (!pos[t]) continue;
    const uint64_t id = key[t] >> 32;
    float s0 = 0.f, s1 = 0.f;
    for (int e = t; e < a.P && key[e] != ~0ull && (key[e] >> 32) == id; ++e) {
      if ((key[e] >> 31) & 1ull) s1 += val[e];
      else s0 += val[e];
    }
    const uint32_t m = member_fix(gen_mean(s0 / div, s1 / div, a.alpha));
    a.out_ids[r * a.cap + o] = (int32_t)id;
    a.out_mem[r * a.cap + o] = m;
    atomicAdd(&norm, (unsigned long long)m);
    ++o;
  }
  __syncthreads();
  if (tid == 0) a.out_norm[r] = norm;
}

__global__ void k_aca_keys(const int32_t* __restrict__ ids, const int32_t* __restrict__ cnt, int32_t N, int cap,
                           int32_t* __restrict__ keys) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)N * cap) return;
  const int64_t p = e / cap;
  keys[e] = (e % cap) < cnt[p] ? ids[e] : N;
}

__global__ void k_aca_fill(const int32_t* __restrict__ perm, int64_t n, int cap, const uint32_t* __restrict__ mem_rows,
                           int32_t* __restrict__ ids, uint32_t* __restrict__ mem) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int32_t slot = perm[e];
  ids[e] = slot / cap;
  mem[e] = mem_rows[slot];
}

// one block per (query, non-zero coordinate i of its activation): walk entry i
__global__ void k_aca_walk(const int32_t* __restrict__ q_ids, const uint32_t* __restrict__ q_mem,
                           const int32_t* __restrict__ q_cnt, int cap, int32_t N, const int64_t* __restrict__ off,
                           const int32_t* __restrict__ ids, const uint32_t* __restrict__ mem,
                           unsigned long long* __restrict__ num) {
  const int b = blockIdx.x, j = blockIdx.y;
  if (j >= q_cnt[b]) return;
  const int32_t i = q_ids[(int64_t)b * cap + j];
  const uint32_t fq = q_mem[(int64_t)b * cap + j];
  if (fq == 0 || i < 0 || i >= N) return;
  for (int64_t e = off[i] + threadIdx.x; e < off[i + 1]; e += blockDim.x) {
    const uint32_t m = mem[e];
    if (m == 0) continue;
    atomicAdd(num + (int64_t)b * N + ids[e], (unsigned long long)min(fq, m));
  }
}

void launch_aca_rows(AcaRowArgs& a, int64_t rows, cudaStream_t s) {
  a.nmax = a.mode == 0 ? a.k1 : a.k2 * a.k1;
  int P = 2 * kAcaT;
  while (P < 2 * a.nmax) P <<= 1;
  GIFT_REQUIRE(P <= kAcaMaxP, "k2 * k1 (or k1 without augmentation) exceeds 2048");
  a.P = P;
  a.cap = 2 * a.nmax;
  const size_t smem = (size_t)P * 16;
  GIFT_CUDA(cudaFuncSetAttribute(k_aca_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (rows <= 0) return;
  k_aca_rows<<<(unsigned)rows, kAcaT, smem, s>>>(a);
  GIFT_LAUNCHED("k_aca_rows");
}

}  // namespace

template <class T>
T* Aca::alloc(size_t n) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(n * sizeof(T), 16);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    fail(GIFT_ENOMEM, "allocation of " + std::to_string(bytes) + " bytes failed");
  }
  owned.push_back(p);
  device_bytes += bytes;
  return static_cast<T*>(p);
}

Aca::~Aca() {
  for (void* p : owned) cudaFree(p);
}

void aca_build(Aca& a, Scratch& sc, cudaStream_t s) {
  const int32_t N = a.N;
  AcaRowArgs r{};
  r.mode = a.mode;
  r.k1 = a.k1;
  r.k2 = a.k2;
  r.alpha = a.alpha;
  r.N = N;
  for (int l = 0; l < 2; ++l) {
    r.db_ids[l] = a.m[l]->row_ids;
    r.db_sc[l] = a.m[l]->row_sc;
    r.nb[l] = a.m[l]->row_ids;  // a database shape's own ranking
    r.own_sc[l] = a.m[l]->row_sc;
  }
  r.ld = a.k1;
  r.nmax = a.mode == 0 ? a.k1 : a.k2 * a.k1;
  r.cap = 2 * r.nmax;
  const int64_t slots = (int64_t)N * r.cap;
  r.out_ids = sc.get<int32_t>(slots);
  r.out_mem = sc.get<uint32_t>(slots);
  r.out_cnt = sc.get<int32_t>(N);
  a.card = a.alloc<unsigned long long>(N);
  r.out_norm = a.card;
  launch_aca_rows(r, N, s);
  a.cap = r.cap;
  // transpose: entry i lists every p with a non-zero coordinate i, ascending p (stable sort by i)
  int32_t* keys = sc.get<int32_t>(slots);
  k_aca_keys<<<(unsigned)cdiv(slots, 256), 256, 0, s>>>(r.out_ids, r.out_cnt, N, r.cap, keys);
  GIFT_LAUNCHED("k_aca_keys");
  int32_t* perm = sc.get<int32_t>(slots);
  int32_t* skeys = sc.get<int32_t>(slots);
  stable_sort_by_key(keys, slots, N + 1, perm, skeys, sc, s);
  int64_t* off_all = sc.get<int64_t>((size_t)N + 2);
  bin_offsets(skeys, slots, N + 1, off_all, s);
  int64_t pairs = 0;
  GIFT_CUDA(cudaMemcpyAsync(&pairs, off_all + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GIFT_CUDA(cudaStreamSynchronize(s));
  a.pairs = pairs;
  a.off = a.alloc<int64_t>((size_t)N + 1);
  GIFT_CUDA(cudaMemcpyAsync(a.off, off_all, ((size_t)N + 1) * 8, cudaMemcpyDeviceToDevice, s));
  a.ids = a.alloc<int32_t>((size_t)std::max<int64_t>(pairs, 1));
  a.mem = a.alloc<uint32_t>((size_t)std::max<int64_t>(pairs, 1));
  if (pairs > 0) {
    k_aca_fill<<<(unsigned)cdiv(pairs, 256), 256, 0, s>>>(perm, pairs, r.cap, r.out_mem, a.ids, a.mem);
    GIFT_LAUNCHED("k_aca_fill");
  }
  int* mx = sc.get<int>(1);
  GIFT_CUDA(cudaMemsetAsync(mx, 0, sizeof(int), s));
  k_max_entry<<<(unsigned)cdiv(N, 256), 256, 0, s>>>(a.off, N, mx);
  GIFT_LAUNCHED("k_max_entry");
  GIFT_CUDA(cudaMemcpyAsync(&a.max_entry, mx, sizeof(int), cudaMemcpyDeviceToHost, s));
  GIFT_CUDA(cudaStreamSynchronize(s));
}

void aca_rerank(const Aca& a, const int32_t* cand1, const float* sc1, const int32_t* cand2, const float* sc2,
                int32_t B, int32_t n_cand, int32_t topk, int32_t* out_ids, float* out_sprime, Scratch& sc,
                cudaStream_t s) {
  const int32_t N = a.N;
  const int64_t BN = (int64_t)B * N;
  AcaRowArgs r{};
  r.mode = a.mode;
  r.k1 = a.k1;
  r.k2 = a.k2;
  r.alpha = a.alpha;
  r.N = N;
  for (int l = 0; l < 2; ++l) {
    r.db_ids[l] = a.m[l]->row_ids;
    r.db_sc[l] = a.m[l]->row_sc;
  }
  r.nb[0] = cand1;
  r.nb[1] = cand2;
  r.own_sc[0] = sc1;
  r.own_sc[1] = sc2;
  r.ld = n_cand;
  r.nmax = a.mode == 0 ? a.k1 : a.k2 * a.k1;
  r.cap = 2 * r.nmax;
  r.out_ids = sc.get<int32_t>((size_t)B * r.cap);
  r.out_mem = sc.get<uint32_t>((size_t)B * r.cap);
  r.out_cnt = sc.get<int32_t>(B);
  r.out_norm = sc.get<unsigned long long>(B);
  launch_aca_rows(r, B, s);
  unsigned long long* num = sc.get<unsigned long long>(BN);
  GIFT_CUDA(cudaMemsetAsync(num, 0, BN * 8, s));
  float* Srow = sc.get<float>(BN);
  k_fill_f32<<<(unsigned)cdiv(BN, 256), 256, 0, s>>>(Srow, BN, -INFINITY);
  GIFT_LAUNCHED("k_fill_f32");
  unsigned long long* unused = sc.get<unsigned long long>(B);
  k_rerank_prep<<<(unsigned)B, 256, 0, s>>>(cand1, sc1, n_cand, a.k1, N, Srow, unused);  // S^(1) tie key
  GIFT_LAUNCHED("k_rerank_prep");
  k_aca_walk<<<dim3((unsigned)B, (unsigned)r.cap), 128, 0, s>>>(r.out_ids, r.out_mem, r.out_cnt, r.cap, N, a.off,
                                                                a.ids, a.mem, num);
  GIFT_LAUNCHED("k_aca_walk");
  unsigned long long* keys = sc.get<unsigned long long>(BN);
  k_rerank_keys<<<(unsigned)cdiv(BN, 256), 256, 0, s>>>(num, r.out_norm, a.card, Srow, B, N, keys);
  GIFT_LAUNCHED("k_rerank_keys");
  unsigned long long* kout = sc.get<unsigned long long>((int64_t)B * topk);
  topk_rows_u64(reinterpret_cast<const uint64_t*>(keys), B, N, topk, out_ids, reinterpret_cast<uint64_t*>(kout),
                sc, s);
  k_keys_to_sprime<<<(unsigned)cdiv((int64_t)B * topk, 256), 256, 0, s>>>(kout, (int64_t)B * topk, out_sprime);
  GIFT_LAUNCHED("k_keys_to_sprime");
}

void sif_build(Index& ix, const int32_t* nbr_ids, const float* nbr_scores, Scratch& sc, cudaStream_t s) {
  const int32_t N = ix.sif_n;
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
  const int32_t N = ix.sif_n;
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
  // a query reaches at most n_cand candidates and k1 S-IF entries of at most
  // max_sif_entry shapes: the selection runs over those, not over all N
  const int need = std::min(topk, N);
  const int64_t cap = std::min<int64_t>(
      N, std::max<int64_t>(need, (int64_t)n_cand + (int64_t)k1 * std::max(1, ix.max_sif_entry)));
  int32_t* cids = sc.get<int32_t>((size_t)B * cap);
  unsigned long long* keys = sc.get<unsigned long long>((size_t)B * cap);
  k_rerank_compact<<<(unsigned)B, kCompactT, 0, s>>>(num, fqn, reinterpret_cast<const unsigned long long*>(ix.sif_card),
                                                      Srow, N, cap, need, cids, keys);
  GIFT_LAUNCHED("k_rerank_compact");
  int32_t* pos = sc.get<int32_t>((size_t)B * topk);
  unsigned long long* kout = sc.get<unsigned long long>((int64_t)B * topk);
  topk_rows_u64(reinterpret_cast<const uint64_t*>(keys), B, cap, topk, pos, reinterpret_cast<uint64_t*>(kout), sc,
                s);
  k_rerank_out<<<(unsigned)cdiv((int64_t)B * topk, 256), 256, 0, s>>>(pos, kout, cids, cap, B, topk, out_ids,
                                                                     out_sprime);
  GIFT_LAUNCHED("k_rerank_out");
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
  const int32_t N = ix.sif_n;
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
