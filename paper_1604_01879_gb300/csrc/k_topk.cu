// Block-wide top-k selection: one CTA per row.
//
// Values become order-preserving unsigned keys (larger value -> larger key).
// A radix select over the key bytes (most significant first) finds the k-th
// largest key T and how many of the k must come from keys equal to T; an
// ordered compaction (in index order) takes every key > T and the first such
// keys == T, so ties are resolved by the lower index; a bitonic sort in
// shared memory orders the k winners by (key desc, index asc).
#include "gift_internal.cuh"

namespace gift {

namespace {

constexpr int kT = 1024;
constexpr int kMaxK = 1024;
constexpr unsigned kFull = 0xffffffffu;

// block-wide exclusive scan of one int per thread (kT threads)
__device__ __forceinline__ int block_excl_scan(int v, int* wsum, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    const int y = wsum[lane];
    int z = y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int q = __shfl_up_sync(kFull, z, o);
      if (lane >= o) z += q;
    }
    wsum[lane] = z - y;
    if (lane == 31) wsum[32] = z;
  }
  __syncthreads();
  const int r = x - v + wsum[w];
  total = wsum[32];
  __syncthreads();
  return r;
}

// "a before b": larger key first, then lower index
__device__ __forceinline__ bool before(unsigned long long ka, int ia, unsigned long long kb, int ib) {
  return ka > kb || (ka == kb && ia < ib);
}

__device__ void bitonic_sort(unsigned long long* key, int* idx, int P) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < P / 2; t += kT) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const bool sw = up ? before(key[hi], idx[hi], key[lo], idx[lo])
                           : before(key[lo], idx[lo], key[hi], idx[hi]);
        if (sw) {
          const unsigned long long tk = key[lo];
          key[lo] = key[hi];
          key[hi] = tk;
          const int ti = idx[lo];
          idx[lo] = idx[hi];
          idx[hi] = ti;
        }
      }
      __syncthreads();
    }
  }
}

template <bool F32>
__device__ __forceinline__ unsigned long long get_key(const float* sr, const unsigned long long* kr,
                                                      int64_t i) {
  if (F32) return (unsigned long long)f2key(sr[i]);
  return kr[i];
}

template <bool F32>
__global__ __launch_bounds__(kT) void k_topk(const float* __restrict__ scores,
                                             const unsigned long long* __restrict__ keys, int64_t n,
                                             int k, int32_t* __restrict__ ids_out,
                                             float* __restrict__ val_out,
                                             unsigned long long* __restrict__ key_out) {
  __shared__ int hist[256];
  __shared__ int wsum[33];
  __shared__ unsigned long long s_key[kMaxK];
  __shared__ int s_idx[kMaxK];
  __shared__ unsigned long long sh_prefix;
  __shared__ int sh_need;
  const int b = blockIdx.x;
  const float* sr = F32 ? scores + (int64_t)b * n : nullptr;
  const unsigned long long* kr = F32 ? nullptr : keys + (int64_t)b * n;
  const int tid = threadIdx.x;
  const int nbytes = F32 ? 4 : 8;
  const int take = (int)std::min<int64_t>(n, k);

  unsigned long long T = 0;
  int need_eq = 0;  // how many keys == T are taken
  if (n > k) {
    unsigned long long prefix = 0, mask = 0;
    int remaining = k;
    for (int byte = nbytes - 1; byte >= 0; --byte) {
      if (tid < 256) hist[tid] = 0;
      __syncthreads();
      if (byte == nbytes - 1) {
        // the top byte (sign and high exponent bits) is the same for nearly every key: one
        // atomic per distinct bin per warp (lanes grouped by __match_any_sync)
        for (int64_t c0 = 0; c0 < n; c0 += kT) {
          const int64_t i = c0 + tid;
          const int bin = i < n ? (int)((get_key<F32>(sr, kr, i) >> (8 * byte)) & 255) : -1;
          const unsigned peers = __match_any_sync(kFull, bin);
          if (bin >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
        }
      } else {
        for (int64_t i = tid; i < n; i += kT) {
          const unsigned long long key = get_key<F32>(sr, kr, i);
          if ((key & mask) == prefix) atomicAdd(&hist[(key >> (8 * byte)) & 255], 1);
        }
      }
      __syncthreads();
      if (tid == 0) {
        int cum = 0, d = 255;
        for (; d > 0; --d) {
          if (cum + hist[d] >= remaining) break;
          cum += hist[d];
        }
        sh_need = remaining - cum;
        sh_prefix = prefix | ((unsigned long long)d << (8 * byte));
      }
      __syncthreads();
      prefix = sh_prefix;
      remaining = sh_need;
      mask |= 0xFFull << (8 * byte);
      __syncthreads();
    }
    T = prefix;
    need_eq = remaining;
  }
  // ordered compaction
  const int n_gt = take - need_eq;
  int base_gt = 0, base_eq = 0;
  for (int64_t c0 = 0; c0 < n; c0 += kT) {
    const int64_t i = c0 + tid;
    unsigned long long key = 0;
    bool gt = false, eq = false;
    if (i < n) {
      key = get_key<F32>(sr, kr, i);
      if (n > k) {
        gt = key > T;
        eq = key == T;
      } else {
        gt = true;
      }
    }
    int tot_gt, tot_eq;
    const int pg = block_excl_scan(gt ? 1 : 0, wsum, tot_gt);
    const int pe = block_excl_scan(eq ? 1 : 0, wsum, tot_eq);
    if (gt) {
      s_key[base_gt + pg] = key;
      s_idx[base_gt + pg] = (int)i;
    } else if (eq && base_eq + pe < need_eq) {
      s_key[n_gt + base_eq + pe] = key;
      s_idx[n_gt + base_eq + pe] = (int)i;
    }
    base_gt += tot_gt;
    base_eq += tot_eq;
  }
  __syncthreads();
  int P = 1;
  while (P < take) P <<= 1;
  for (int t = take + tid; t < P; t += kT) {
    s_key[t] = 0;
    s_idx[t] = 0x7fffffff;
  }
  __syncthreads();
  bitonic_sort(s_key, s_idx, P);
  for (int t = tid; t < k; t += kT) {
    const int64_t o = (int64_t)b * k + t;
    if (t < take) {
      ids_out[o] = s_idx[t];
      if (val_out) val_out[o] = key2f((uint32_t)s_key[t]);
      if (key_out) key_out[o] = s_key[t];
    } else {
      ids_out[o] = -1;
      if (val_out) val_out[o] = -INFINITY;
      if (key_out) key_out[o] = 0;
    }
  }
}

// rows of (id, score): sort by (score desc, id asc) and keep k
__global__ __launch_bounds__(kT) void k_sort_candidates(const int32_t* __restrict__ ids,
                                                        const float* __restrict__ scores, int r, int k,
                                                        int32_t* __restrict__ ids_out,
                                                        float* __restrict__ scores_out, int mode_ids) {
  __shared__ unsigned long long s_key[kMaxK];
  __shared__ int s_idx[kMaxK];
  const int b = blockIdx.x;
  int P = 1;
  while (P < r) P <<= 1;
  for (int t = threadIdx.x; t < P; t += kT) {
    if (t < r) {
      const int32_t id = ids[(int64_t)b * r + t];
      // mode_ids: ascending ids (invalid -1 last); else (score desc, id asc)
      if (mode_ids) {
        s_key[t] = (unsigned long long)(0xFFFFFFFFu - (uint32_t)(id < 0 ? 0x7fffffff : id));
      } else {
        s_key[t] = id < 0 ? 0ull : (unsigned long long)f2key(scores[(int64_t)b * r + t]);
      }
      s_idx[t] = id < 0 ? 0x7fffffff : id;
    } else {
      s_key[t] = 0;
      s_idx[t] = 0x7fffffff;
    }
  }
  __syncthreads();
  bitonic_sort(s_key, s_idx, P);
  for (int t = threadIdx.x; t < k; t += kT) {
    const int64_t o = (int64_t)b * k + t;
    const bool ok = t < r && s_idx[t] != 0x7fffffff;
    ids_out[o] = ok ? s_idx[t] : -1;
    if (scores_out) scores_out[o] = ok ? key2f((uint32_t)s_key[t]) : -INFINITY;
  }
}

// key of an (id, score) pair: larger = better by (score desc, id asc); 0 = none
__global__ void k_merge_keys(const int32_t* __restrict__ ids, const float* __restrict__ scores, int64_t n,
                             unsigned long long* __restrict__ keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t id = ids[i];
  keys[i] = id < 0 ? 0ull
                   : ((unsigned long long)f2key(scores[i]) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)id);
}

__global__ void k_merge_decode(const unsigned long long* __restrict__ keys, int64_t n, int32_t* __restrict__ ids,
                               float* __restrict__ scores) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long key = keys[i];
  ids[i] = key == 0ull ? -1 : (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
  scores[i] = key == 0ull ? -INFINITY : key2f((uint32_t)(key >> 32));
}

}  // namespace

void merge_topk_rows(const int32_t* ids, const float* scores, int32_t B, int64_t n, int32_t k, int32_t* ids_out,
                     float* scores_out, Scratch& sc, cudaStream_t s) {
  if (B <= 0 || k <= 0) return;
  const int64_t total = (int64_t)B * n;
  unsigned long long* keys = sc.get<unsigned long long>(total);
  k_merge_keys<<<(unsigned)cdiv(total, 256), 256, 0, s>>>(ids, scores, total, keys);
  GIFT_LAUNCHED("k_merge_keys");
  int32_t* pos = sc.get<int32_t>((size_t)B * k);
  uint64_t* kout = sc.get<uint64_t>((size_t)B * k);
  topk_rows_u64(reinterpret_cast<const uint64_t*>(keys), B, n, k, pos, kout, sc, s);
  k_merge_decode<<<(unsigned)cdiv((int64_t)B * k, 256), 256, 0, s>>>(reinterpret_cast<unsigned long long*>(kout),
                                                                     (int64_t)B * k, ids_out, scores_out);
  GIFT_LAUNCHED("k_merge_decode");
}

void topk_rows_f32(const float* scores, int32_t B, int64_t n, int32_t k, int32_t* ids_out, float* val_out,
                   Scratch&, cudaStream_t s) {
  if (B <= 0 || k <= 0) return;
  GIFT_REQUIRE(k <= kMaxK, "top-k is limited to 1024");
  GIFT_REQUIRE(n < (int64_t)INT32_MAX, "row too long for top-k");
  k_topk<true><<<(unsigned)B, kT, 0, s>>>(scores, nullptr, n, k, ids_out, val_out, nullptr);
  GIFT_LAUNCHED("k_topk<f32>");
}

void topk_rows_u64(const uint64_t* keys, int32_t B, int64_t n, int32_t k, int32_t* ids_out,
                   uint64_t* key_out, Scratch&, cudaStream_t s) {
  if (B <= 0 || k <= 0) return;
  GIFT_REQUIRE(k <= kMaxK, "top-k is limited to 1024");
  GIFT_REQUIRE(n < (int64_t)INT32_MAX, "row too long for top-k");
  k_topk<false><<<(unsigned)B, kT, 0, s>>>(nullptr, reinterpret_cast<const unsigned long long*>(keys), n,
                                          k, ids_out, nullptr,
                                          reinterpret_cast<unsigned long long*>(key_out));
  GIFT_LAUNCHED("k_topk<u64>");
}

void sort_candidates(const int32_t* ids, const float* scores, int32_t B, int32_t r, int32_t k,
                     int32_t* ids_out, float* scores_out, cudaStream_t s) {
  if (B <= 0 || k <= 0) return;
  GIFT_REQUIRE(r <= kMaxK, "candidate rows are limited to 1024");
  k_sort_candidates<<<(unsigned)B, kT, 0, s>>>(ids, scores, r, k, ids_out, scores_out, 0);
  GIFT_LAUNCHED("k_sort_candidates");
}

void sort_ids_rows(const int32_t* ids, int32_t B, int32_t r, int32_t* out, cudaStream_t s) {
  if (B <= 0 || r <= 0) return;
  GIFT_REQUIRE(r <= kMaxK, "candidate rows are limited to 1024");
  k_sort_candidates<<<(unsigned)B, kT, 0, s>>>(ids, nullptr, r, r, out, nullptr, 1);
  GIFT_LAUNCHED("k_sort_ids");
}

}  // namespace gift
