// Shared device utilities: row norms, exclusive scan, stable counting/radix
// sort by small integer keys, bin offsets, fills.
#include "gift_internal.cuh"

namespace gift {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// one warp per row: 1/||x|| (0 for a zero row)
__global__ void k_row_invnorm(const float* __restrict__ X, int64_t n, int D, float* __restrict__ inv) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float4* p = reinterpret_cast<const float4*>(X + row * (int64_t)D);
  float acc = 0.f;
  for (int i = lane; i < (D >> 2); i += 32) {
    const float4 v = p[i];
    acc = fmaf(v.x, v.x, acc);
    acc = fmaf(v.y, v.y, acc);
    acc = fmaf(v.z, v.z, acc);
    acc = fmaf(v.w, v.w, acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) inv[row] = acc > 0.f ? 1.0f / sqrtf(acc) : 0.f;
}

// one warp per row: 0.5 * ||x||^2 accumulated in two-float precision
__global__ void k_half_sq_norm(const float* __restrict__ X, int64_t n, int D, float* __restrict__ out) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* p = X + row * (int64_t)D;
  float hi = 0.f, lo = 0.f;
  for (int i = lane; i < D; i += 32) {
    const float x = p[i];
    const float pr = x * x;
    const float pe = fmaf(x, x, -pr);
    const float s = hi + pr;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (pr - bb) + pe;
    hi = s;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(kFull, hi, o);
    const float l2 = __shfl_xor_sync(kFull, lo, o);
    const float s = hi + h2;
    const float bb = s - hi;
    lo = lo + l2 + ((hi - (s - bb)) + (h2 - bb));
    hi = s;
  }
  if (lane == 0) out[row] = 0.5f * (hi + lo);
}

constexpr int kScanT = 256;
constexpr int kScanItems = 8;
constexpr int kScanPerBlock = kScanT * kScanItems;

__global__ __launch_bounds__(kScanT) void k_scan_blocks(const int64_t* __restrict__ in,
                                                         int64_t* __restrict__ out, int64_t n,
                                                         int64_t* __restrict__ block_sums) {
  __shared__ int64_t wtot[kScanT / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanPerBlock + (int64_t)tid * kScanItems;
  int64_t v[kScanItems];
  int64_t t = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    t += v[i];
  }
  int64_t x = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtot[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t y = lane < kScanT / 32 ? wtot[lane] : 0;
    int64_t z = y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t q = __shfl_up_sync(kFull, z, o);
      if (lane >= o) z += q;
    }
    if (lane < kScanT / 32) wtot[lane] = z - y;  // exclusive warp prefix
  }
  __syncthreads();
  int64_t run = x - t + wtot[w];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (tid == kScanT - 1) block_sums[blockIdx.x] = run;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += offs[i / kScanPerBlock];
}

// ---------------------------------------------------------------- radix sort
constexpr int kRadixT = 1024;

__global__ __launch_bounds__(kRadixT) void k_radix_hist(const int32_t* __restrict__ keys, int64_t n,
                                                         int shift, int64_t* __restrict__ hist,
                                                         int64_t ntiles) {
  __shared__ int h[256];
  const int tid = threadIdx.x;
  if (tid < 256) h[tid] = 0;
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * kRadixT + tid;
  if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1);
  __syncthreads();
  if (tid < 256) hist[(int64_t)tid * ntiles + blockIdx.x] = h[tid];
}

__global__ __launch_bounds__(kRadixT) void k_radix_scatter(
    const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in, int64_t n, int shift,
    const int64_t* __restrict__ offs, int64_t ntiles, int32_t* __restrict__ keys_out,
    int32_t* __restrict__ vals_out) {
  __shared__ int wcnt[32][257];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < 32 * 257; i += kRadixT) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * kRadixT + tid;
  const bool valid = idx < n;
  const int key = valid ? keys_in[idx] : 0;
  const int d = valid ? ((key >> shift) & 255) : 256;
  const unsigned peers = __match_any_sync(kFull, d);
  const unsigned lt = (1u << lane) - 1u;
  const int rank_w = __popc(peers & lt);
  if (valid && rank_w == 0) wcnt[w][d] = __popc(peers);
  __syncthreads();
  if (tid < 256) {
    int run = 0;
    for (int ww = 0; ww < 32; ++ww) {
      const int c = wcnt[ww][tid];
      wcnt[ww][tid] = run;
      run += c;
    }
  }
  __syncthreads();
  if (valid) {
    const int64_t dst = offs[(int64_t)d * ntiles + blockIdx.x] + wcnt[w][d] + rank_w;
    keys_out[dst] = key;
    vals_out[dst] = vals_in ? vals_in[idx] : (int32_t)idx;
  }
}

__global__ void k_bin_offsets(const int32_t* __restrict__ sk, int64_t n, int nbins,
                              int64_t* __restrict__ off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  const int prev = (i == 0) ? -1 : sk[i - 1];
  const int cur = (i == n) ? nbins : sk[i];
  for (int k = prev + 1; k <= cur; ++k) off[k] = i;
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

}  // namespace

void launch_row_invnorm(const float* X, int64_t n, int D, float* inv, cudaStream_t s) {
  if (n <= 0) return;
  k_row_invnorm<<<(unsigned)cdiv(n, 8), 256, 0, s>>>(X, n, D, inv);
  GIFT_LAUNCHED("k_row_invnorm");
}

void launch_half_sq_norm(const float* X, int64_t n, int D, float* out, cudaStream_t s) {
  if (n <= 0) return;
  k_half_sq_norm<<<(unsigned)cdiv(n, 8), 256, 0, s>>>(X, n, D, out);
  GIFT_LAUNCHED("k_half_sq_norm");
}

void launch_fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s) {
  if (n <= 0) return;
  k_fill_i32<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(p, n, v);
  GIFT_LAUNCHED("k_fill_i32");
}

void scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, Scratch& sc, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t nb = cdiv(n, kScanPerBlock);
  int64_t* sums = sc.get<int64_t>(nb);
  k_scan_blocks<<<(unsigned)nb, kScanT, 0, s>>>(in, out, n, sums);
  GIFT_LAUNCHED("k_scan_blocks");
  if (nb > 1) {
    int64_t* sums_x = sc.get<int64_t>(nb);
    scan_exclusive_i64(sums, sums_x, nb, sc, s);
    k_scan_add<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(out, n, sums_x);
    GIFT_LAUNCHED("k_scan_add");
  }
}

void stable_sort_by_key(const int32_t* keys, int64_t n, int32_t nbins, int32_t* perm_out,
                        int32_t* keys_out, Scratch& sc, cudaStream_t s) {
  if (n <= 0) return;
  GIFT_REQUIRE(n < (int64_t)INT32_MAX, "sort size exceeds int32 range");
  int bits = 1;
  while ((1ll << bits) < (int64_t)nbins) ++bits;
  const int passes = (bits + 7) / 8;
  const int64_t ntiles = cdiv(n, kRadixT);
  int64_t* hist = sc.get<int64_t>(256 * ntiles);
  int64_t* offs = sc.get<int64_t>(256 * ntiles);
  int32_t* kbuf[2] = {sc.get<int32_t>(n), sc.get<int32_t>(n)};
  int32_t* vbuf[2] = {sc.get<int32_t>(n), sc.get<int32_t>(n)};
  const int32_t* kin = keys;
  const int32_t* vin = nullptr;
  for (int p = 0; p < passes; ++p) {
    const bool last = p == passes - 1;
    int32_t* ko = last ? keys_out : kbuf[p & 1];
    int32_t* vo = last ? perm_out : vbuf[p & 1];
    k_radix_hist<<<(unsigned)ntiles, kRadixT, 0, s>>>(kin, n, 8 * p, hist, ntiles);
    GIFT_LAUNCHED("k_radix_hist");
    scan_exclusive_i64(hist, offs, 256 * ntiles, sc, s);
    k_radix_scatter<<<(unsigned)ntiles, kRadixT, 0, s>>>(kin, vin, n, 8 * p, offs, ntiles, ko, vo);
    GIFT_LAUNCHED("k_radix_scatter");
    kin = ko;
    vin = vo;
  }
}

void bin_offsets(const int32_t* sorted_keys, int64_t n, int32_t nbins, int64_t* off, cudaStream_t s) {
  k_bin_offsets<<<(unsigned)cdiv(n + 1, 256), 256, 0, s>>>(sorted_keys, n, nbins, off);
  GIFT_LAUNCHED("k_bin_offsets");
}

}  // namespace gift
