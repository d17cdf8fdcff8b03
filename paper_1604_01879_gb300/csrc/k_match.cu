// Matching score of Eq. 3 after a learned linear view projection u = W q,
// and its gradient through the argmax view pair, on the tensor cores.
//
// Forward: U = Q W^T and V = P W^T (engine GEMMs; BF16 inputs multiply
// exactly in one product, FP32 inputs in the two-part split), then the
// segmented-max contraction of U and V (two-part split, FP32-level) gives
// S and the first argmax j* of every (query view, shape).
// Backward, with c = grad_S[b, p] / |V(x_b)| and s = u_i.v_j*/(|u_i||v_j*|):
//   dU_i  = (1/|u_i|)  ( g_i - (g_i . u_i/|u_i|) u_i/|u_i| ),  g_i = sum_p c v_j*/|v_j*|
//   dV_r  = (1/|v_r|)  ( h_r - (h_r . v_r/|v_r|) v_r/|v_r| ),  h_r = sum_{(i,p): j*=r} c u_i/|u_i|
// (the projections use s = g-weighted cosines: sum_p c s = g_i . u_i/|u_i|).
// G = A V is a GEMM with the one-hot matrix A[i, r] = c v-norm-weight where r
// is the argmax view of (i, shape(r)); A is never stored: the engine's producer
// warp writes each A tile from the argmax (transposed to shape-major) into
// shared memory, and the tensor cores multiply it with two-part operands.
// H = A^T U is a segmented sum on the CUDA cores over the entries sorted by
// their argmax view (N_v times fewer multiply-adds than the dense product). Then
//   dW = dU^T Q + dV^T P,  dQ = dU W,  dP = dV W
// as engine GEMMs on transposed two-part operands.
#include "gift_internal.cuh"
#include "segmax.cuh"
#include "tc_gemm.cuh"

namespace gift {

namespace {

// element of an input in FP32 or BF16
template <typename T>
__device__ __forceinline__ float ld_f(const T* p, int64_t i);
template <>
__device__ __forceinline__ float ld_f<float>(const float* p, int64_t i) { return p[i]; }
template <>
__device__ __forceinline__ float ld_f<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

// two-part BF16 copy of a row-major [rows, cols] matrix (lo may be null)
template <typename T>
__global__ void k_split_any(const T* __restrict__ in, int64_t n, __nv_bfloat16* __restrict__ hi,
                            __nv_bfloat16* __restrict__ lo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = ld_f<T>(in, i);
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[i] = h;
  if (lo) lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// the same for FP32 input, four elements per thread (n % 4 == 0, 16-byte aligned input, 8-byte aligned output)
__global__ void k_split4(const float4* __restrict__ in, int64_t n4, uint2* __restrict__ hi, uint2* __restrict__ lo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = in[i];
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
    hi[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
    if (lo) lo[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
  }
}

template <typename T>
__global__ void k_to_float(const T* __restrict__ in, int64_t n, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = ld_f<T>(in, i);
}

// out[c, r] (two-part BF16, row pitch ld) = in[r, c] for r < rows; zero for rows <= r < ld
template <typename T>
__global__ void k_transpose_split(const T* __restrict__ in, int64_t rows, int64_t cols, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, int64_t ld) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < rows && c < cols) ? ld_f<T>(in, r * cols + c) : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t c = c0 + y, r = r0 + threadIdx.x;
    if (c < cols && r < ld) {
      const float v = t[threadIdx.x][y];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      hi[c * ld + r] = h;
      if (lo) lo[c * ld + r] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

// out[c, r] = in[r, c] for BF16 (one part), 64 x 64 tiles moved in 16-byte
// pieces (cols % 8 == 0, ld % 64 == 0, 16-byte aligned rows); zero for rows <= r < ld
__global__ __launch_bounds__(256) void k_transpose_bf16(const __nv_bfloat16* __restrict__ in, int64_t rows,
                                                        int64_t cols, __nv_bfloat16* __restrict__ out, int64_t ld) {
  __shared__ __nv_bfloat16 t[64][72];
  const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
  const int tid = threadIdx.x, part = tid & 7;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int row = (tid >> 3) + 32 * i;
    const int64_t r = r0 + row, c = c0 + part * 8;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r < rows && c < cols) v = *reinterpret_cast<const uint4*>(in + r * cols + c);
    *reinterpret_cast<uint4*>(&t[row][part * 8]) = v;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int oc = (tid >> 3) + 32 * i;
    const int64_t c = c0 + oc, r = r0 + part * 8;
    if (c >= cols || r >= ld) continue;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = t[part * 8 + k][oc];
    *reinterpret_cast<uint4*>(out + c * ld + r) = *reinterpret_cast<const uint4*>(v);
  }
}

// ---------------------------------------------------------------- one-hot gradient GEMMs
// k-blocks per accumulator chunk: 16 x 4 sub-steps x 3 products = 192 MMA steps
constexpr int kOneHotChunkKB = 16;

// G = A V: rows are query views i and the reduction runs over database views r;
// B is the transposed two-part operand of V.
struct OneHotPolicy {
  static constexpr int TN = 128, NBUF = 4, STAGES = 3, SPLIT = 3, EB = 2;
  static constexpr bool GEN_A = true;
  static constexpr int GEN_WARPS = 4;  // generator thread g: row g of the A tile
  static constexpr int kWarpSmem = 16;
  int64_t M, N;             // rows (query views), dout
  int nkb;                  // 64-wide k-blocks of the reduction
  int64_t nq, nr;           // query views, database views
  int Np, nv;               // shapes, views per shape
  const int16_t* amT;       // [Np, nq] argmax view of (i, p), shape-major
  const float* wT;          // [Np, nq] weight of that non-zero, c / |v_r|
  const float* gS;          // [B, Np]
  const int32_t* vquery;    // [nq] query of each view
  const float* vcoef;       // [nq] 1 / |V(x_b)| of the view's query
  const float* kinv;        // 1/|v_r| [nr]
  float* C;                 // [M, N]
  struct Item {
    int64_t r0, c0;
    int nr, nc;
  };
  struct Ctx {
    float sum[TN];
  };
  // the non-zero of one k-block prefetched by each generator thread (fast
  // layout, N_v a multiple of 64, one shape per k-block: thread g owns row g);
  // other layouts are written by warp 0 alone inside gen_store
  bool fast;
  int kb_per_shape;  // fast layout: N_v / 64 k-blocks per shape
  struct GenRegs {  // loaded argmax (-1: none) and weight of the thread's entry
    int j;
    float w;
  };
  struct GenPos {
    int pos;  // row * 64 + column in the A tile, -1 = none
  };
  __device__ __forceinline__ int64_t n_mt() const { return cdiv(M, tc::kTM); }
  __device__ __forceinline__ int64_t total() const { return n_mt() * cdiv(N, TN); }
  __device__ __forceinline__ Item decode(int64_t item) const {
    Item it;
    const int64_t mt = n_mt();
    const int64_t ct = item / mt, rt = item % mt;
    it.r0 = rt * tc::kTM;
    it.c0 = ct * TN;
    it.nr = (int)min((int64_t)tc::kTM, M - it.r0);
    it.nc = (int)min((int64_t)TN, N - it.c0);
    return it;
  }
  __device__ __forceinline__ int nchunks(const Item&) const { return (int)cdiv(nkb, kOneHotChunkKB); }
  __device__ __forceinline__ void chunk(const Item& it, int c, int& br, int& kb0, int& kb1) const {
    br = (int)it.c0;
    kb0 = c * kOneHotChunkKB;
    kb1 = min(nkb, kb0 + kOneHotChunkKB);
  }
  // the argmax and weight lines of k-block kb + kPrefetchKB are pulled into L2
  // while this k-block's are loaded
  static constexpr int kPrefetchKB = 8;
  // issue the loads of k-block kb (their values are first read by gen_store)
  __device__ __forceinline__ void gen_load(const Item& it, int kb, int g, GenRegs& r) const {
    r.j = -1;
    r.w = 0.f;
    if (!fast) return;
    const int64_t k0 = (int64_t)kb * 64;
    if (k0 >= nr) return;
    const int p = kb_per_shape == 1 ? kb : kb / kb_per_shape;
    {  // 128 rows: 256 bytes of argmax and 512 of weights, one line per thread 32..37
       // (not warp 0, which also starts the B copies)
      const int64_t kp = k0 + (int64_t)kPrefetchKB * 64;
      const int u = g - 32;
      if (kp < nr && u >= 0 && u < 6) {
        const int pp = kb_per_shape == 1 ? kb + kPrefetchKB : (kb + kPrefetchKB) / kb_per_shape;
        const int64_t e = (int64_t)pp * nq + it.r0;
        const int off = u < 2 ? u * 64 : (u - 2) * 32;  // first row of the line
        if (it.r0 + off < nq) {
          if (u < 2)
            tc::prefetch_l2(amT + e + off);
          else
            tc::prefetch_l2(wT + e + off);
        }
      }
    }
    if (g < it.nr) {  // read-only for the kernel's lifetime
      const int64_t e = (int64_t)p * nq + it.r0 + g;
      r.j = __ldg(amT + e);
      r.w = __ldg(wT + e);
    }
  }
  // one non-zero of the A tile, hi and lo parts, 128-byte swizzled K-major layout
  __device__ __forceinline__ static void put(uint8_t* a_hi, uint8_t* a_lo, int row, int col, float w) {
    const __nv_bfloat16 h = __float2bfloat16_rn(w);
    const __nv_bfloat16 l = __float2bfloat16_rn(w - __bfloat162float(h));
    const int off = row * 128 + ((((col >> 3) ^ (row & 7))) << 4) + ((col & 7) << 1);
    *reinterpret_cast<__nv_bfloat16*>(a_hi + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(a_lo + off) = l;
  }
  __device__ __forceinline__ void gen_store(const Item& it, int kb, int g, const GenRegs& r, const GenPos* prev,
                                            GenPos& now, uint8_t* a_hi, uint8_t* a_lo) const {
    now.pos = -1;
    if (fast) {
      // the tile is zero but for the entry this thread wrote into it last time
      // (a position belongs to one thread: its row)
      if (prev && prev->pos >= 0) put(a_hi, a_lo, prev->pos >> 6, prev->pos & 63, 0.f);
      const int64_t k0 = (int64_t)kb * 64;
      const int p = kb_per_shape == 1 ? kb : kb / kb_per_shape;
      const int j = r.j;
      if (j >= 0) {  // argmax comes from the forward; stay inside the shape
        const int64_t rr = (int64_t)p * nv + (j < nv ? j : 0);
        if (rr >= k0 && rr < k0 + 64) now.pos = g * 64 + (int)(rr - k0);
      }
      if (now.pos >= 0) put(a_hi, a_lo, now.pos >> 6, now.pos & 63, r.w);
      return;
    }
    if (g >= 32) return;  // warp 0 writes the general layouts
    const int lane = g;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int o = lane * 16; o < tc::kTM * 128; o += 32 * 16) {
      *reinterpret_cast<uint4*>(a_hi + o) = z;
      *reinterpret_cast<uint4*>(a_lo + o) = z;
    }
    __syncwarp();
    const int64_t k0 = (int64_t)kb * 64;
    {
      if (k0 >= nr) return;
      const int p0 = (int)(k0 / nv), p1 = (int)min((int64_t)Np - 1, (k0 + 63) / nv);
      for (int q = 0; q < 4; ++q) {
        const int row = lane + 32 * q;
        const int64_t i = it.r0 + row;
        if (row >= it.nr) continue;
        const int b = vquery[i];
        const float cb = vcoef[i];
        for (int p = p0; p <= p1; ++p) {
          int j = amT[(int64_t)p * nq + i];
          if (j < 0 || j >= nv) j = 0;  // argmax comes from the forward; stay inside the shape
          const int64_t rr = (int64_t)p * nv + j;
          if (rr < k0 || rr >= k0 + 64) continue;
          put(a_hi, a_lo, row, (int)(rr - k0), gS[(int64_t)b * Np + p] * cb * kinv[rr]);
        }
      }
    }
  }
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
    float* crow = C + (it.r0 + m) * N + it.c0;
#pragma unroll
    for (int j = 0; j < TN; ++j)
      if (j < it.nc) crow[j] = x.sum[j];
  }
};

// shape-major argmax and one-hot weights: for every (query view i, shape p),
// j = argmax[i, p], wU = c / |v_{p nv + j}|, wV = c / |u_i| with c = grad_S[b, p] / |V(x_b)|
__global__ void k_onehot_prep(const int16_t* __restrict__ argmax, int64_t nq, int Np, int nv,
                              const int32_t* __restrict__ vquery, const float* __restrict__ vcoef,
                              const float* __restrict__ gS, const float* __restrict__ vinv,
                              const float* __restrict__ uinv, int16_t* __restrict__ amT, float* __restrict__ wU,
                              float* __restrict__ wV) {
  __shared__ int16_t t[32][33];
  const int64_t p0 = (int64_t)blockIdx.x * 32, i0 = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = i0 + k, p = p0 + threadIdx.x;
    if (i < nq && p < Np) t[k][threadIdx.x] = argmax[i * Np + p];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t p = p0 + k, i = i0 + threadIdx.x;
    if (i >= nq || p >= Np) continue;
    int j = t[threadIdx.x][k];
    const int16_t js = (int16_t)j;
    if (j < 0 || j >= nv) j = 0;  // argmax comes from the forward; stay inside the shape
    const float c = gS[(int64_t)vquery[i] * Np + p] * vcoef[i];
    amT[p * nq + i] = js;
    wU[p * nq + i] = c * vinv[p * nv + j];
    wV[p * nq + i] = c * uinv[i];
  }
}

__global__ void k_view_coef(const int32_t* __restrict__ vquery, const int32_t* __restrict__ qoff, int64_t nq,
                            float* __restrict__ coef) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const int b = vquery[i];
  coef[i] = 1.f / (float)(qoff[b + 1] - qoff[b]);
}

// out_r = inv_r (g_r - (g_r . x_r inv_r) x_r inv_r): the gradient through x / |x| (warp per row)
__global__ void k_tangent(const float* __restrict__ X, const float* __restrict__ inv, const float* __restrict__ G,
                          int64_t n, int dout, float* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const float iv = inv[r];
  const float* x = X + r * dout;
  const float* g = G + r * dout;
  float dot = 0.f;
  for (int d = lane; d < dout; d += 32) dot = fmaf(x[d], g[d], dot);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  const float t = dot * iv * iv;
  for (int d = lane; d < dout; d += 32) out[r * dout + d] = iv * (g[d] - t * x[d]);
}

__global__ void k_view_query(const int32_t* __restrict__ qoff, int32_t* __restrict__ vq) {
  const int b = blockIdx.x;
  for (int v = qoff[b] + threadIdx.x; v < qoff[b + 1]; v += blockDim.x) vq[v] = b;
}

// ---------------------------------------------------------------- H = A^T U on the CUDA cores
// Every database view's row of H is the weighted sum of the query views whose
// argmax in its shape is that view:
//   H[p N_v + j] = sum_{i : j(i, p) = j} wV[p, i] U[i]
// The (shape, query view) entries are sorted by that database view (stably, so in
// ascending entry order), and one warp per database view sums its entries' rows of
// U (L2-resident) in FP32 in that order: N_v times fewer multiply-adds than the dense
// one-hot GEMM, and a result that does not depend on the launch.
// The entries of shape p grouped by their argmax view j, ascending query view
// within a group (a stable counting sort, one block per shape): perm[p nq + ...]
// holds the entry indices e = p nq + i, beg[p N_v + j] the first position of
// view j's group and cnt[p N_v + j] its size; entries without an argmax (j
// outside [0, N_v)) are left out. Shared memory: 32 x N_v per-warp counts and
// N_v running group ends.
constexpr int kCsrT = 1024;
constexpr int kCsrMaxNv = 1024;  // 33 x 1024 ints of shared memory
__global__ __launch_bounds__(kCsrT) void k_onehot_csr(const int16_t* __restrict__ amT, int64_t nq, int nv,
                                                      int32_t* __restrict__ perm, int64_t* __restrict__ beg,
                                                      int32_t* __restrict__ cnt) {
  extern __shared__ int csr_sm[];
  int* wc = csr_sm;            // [32][nv]
  int* base = csr_sm + 32 * nv;  // [nv]
  const int p = blockIdx.x, t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int16_t* a = amT + (int64_t)p * nq;
  const int64_t e0 = (int64_t)p * nq;
  for (int j = t; j < nv; j += kCsrT) base[j] = 0;
  __syncthreads();
  for (int64_t i = t; i < nq; i += kCsrT) {
    const int j = a[i];
    if (j >= 0 && j < nv) atomicAdd(&base[j], 1);
  }
  __syncthreads();
  if (t == 0) {  // exclusive prefix over the views (N_v steps)
    int run = 0;
    for (int j = 0; j < nv; ++j) {
      const int c = base[j];
      cnt[(int64_t)p * nv + j] = c;
      beg[(int64_t)p * nv + j] = e0 + run;
      base[j] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int64_t c0 = 0; c0 < nq; c0 += kCsrT) {
    const int64_t i = c0 + t;
    int j = -1;
    if (i < nq) {
      j = a[i];
      if (j < 0 || j >= nv) j = -1;
    }
    for (int k = t; k < 32 * nv; k += kCsrT) wc[k] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, j);
    const int rank = __popc(peers & ((1u << lane) - 1u));  // earlier lanes of this warp with view j
    if (j >= 0 && rank == 0) wc[w * nv + j] = __popc(peers);
    __syncthreads();
    for (int v = t; v < nv; v += kCsrT) {  // per view: the warps' starts, in warp order
      int run = base[v];
      for (int w2 = 0; w2 < 32; ++w2) {
        const int c = wc[w2 * nv + v];
        wc[w2 * nv + v] = run;
        run += c;
      }
      base[v] = run;
    }
    __syncthreads();
    if (j >= 0) perm[e0 + wc[w * nv + j] + rank] = (int32_t)(e0 + i);
    __syncthreads();  // before the counts are cleared for the next chunk
  }
}

// key of every (shape p, query view i) entry of the shape-major argmax: its database
// view r = p N_v + j (nr when the view has no argmax)
__global__ void k_onehot_keys(const int16_t* __restrict__ amT, int64_t nq, int Np, int nv,
                              int32_t* __restrict__ keys) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nq * (int64_t)Np) return;
  const int p = (int)(e / nq);
  const int j = amT[e];
  keys[e] = (j >= 0 && j < nv) ? p * nv + j : Np * nv;
}

// group bounds from sorted-key offsets
__global__ void k_off_to_groups(const int64_t* __restrict__ off, int64_t nr, int64_t* __restrict__ beg,
                                int32_t* __restrict__ cnt) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nr) return;
  beg[r] = off[r];
  cnt[r] = (int32_t)(off[r + 1] - off[r]);
}

// H[r] = sum of wV[e] U[e mod nq] over the entries e of row r (perm[beg[r]] ..
// perm[beg[r] + cnt[r]]), in ascending e: one warp per database view, lane c owns columns
// 4 c + 128 t, up to kHCols columns per pass (dout % 4 == 0)
constexpr int kHCols = 512;
__global__ __launch_bounds__(256) void k_segment_rows_sum(const float* __restrict__ U, const int32_t* __restrict__ perm,
                                                          const int64_t* __restrict__ beg,
                                                          const int32_t* __restrict__ cnt,
                                                          const float* __restrict__ wT, int64_t nq, int64_t nr,
                                                          int dout, float* __restrict__ H) {
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nr) return;
  constexpr int kT = kHCols / 128;  // float4 pieces per lane and pass
  const int64_t e0 = beg[r], e1 = e0 + cnt[r];
  for (int cb = 0; cb < dout; cb += kHCols) {
    float acc[kT][4];
#pragma unroll
    for (int t = 0; t < kT; ++t)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[t][q] = 0.f;
    for (int64_t eb = e0; eb < e1; eb += 32) {
      const int n = (int)min((int64_t)32, e1 - eb);
      int64_t src = 0;
      float wl = 0.f;
      if (lane < n) {
        const int32_t e = perm[eb + lane];
        src = (int64_t)(e % nq) * dout;
        wl = wT[e];
      }
#pragma unroll 4
      for (int k = 0; k < n; ++k) {  // unrolled: several entries' row loads in flight
        const int64_t sk = __shfl_sync(0xffffffffu, src, k);
        const float wk = __shfl_sync(0xffffffffu, wl, k);
        const float* u = U + sk + cb;
#pragma unroll
        for (int t = 0; t < kT; ++t) {
          const int c = 4 * lane + 128 * t;
          if (cb + c < dout) {
            const float4 x = *reinterpret_cast<const float4*>(u + c);
            acc[t][0] = fmaf(wk, x.x, acc[t][0]);
            acc[t][1] = fmaf(wk, x.y, acc[t][1]);
            acc[t][2] = fmaf(wk, x.z, acc[t][2]);
            acc[t][3] = fmaf(wk, x.w, acc[t][3]);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < kT; ++t) {
      const int c = 4 * lane + 128 * t;
      if (cb + c < dout)
        *reinterpret_cast<float4*>(H + r * dout + cb + c) = make_float4(acc[t][0], acc[t][1], acc[t][2], acc[t][3]);
    }
  }
}

// two-part BF16 operand with one TMA box of padding rows
struct Operand {
  __nv_bfloat16* hi = nullptr;
  __nv_bfloat16* lo = nullptr;  // null: one-part (exact BF16 input)
  int64_t rows_alloc = 0;
};

Operand make_operand(const void* x, int dtype, int64_t rows, int cols, bool force_split, Scratch& sc, cudaStream_t s) {
  Operand o;
  if (dtype != GIFT_F32 && !force_split && rows >= tc::kTM && reinterpret_cast<uintptr_t>(x) % 16 == 0) {
    // a BF16 input is its own one-part operand: the tensor map covers its rows
    o.hi = const_cast<__nv_bfloat16*>(static_cast<const __nv_bfloat16*>(x));
    o.rows_alloc = rows;
    return o;
  }
  o.rows_alloc = rows + 128;
  const int64_t n = rows * cols;
  o.hi = sc.get<__nv_bfloat16>((size_t)o.rows_alloc * cols);
  const bool split = dtype == GIFT_F32 || force_split;
  if (split) o.lo = sc.get<__nv_bfloat16>((size_t)o.rows_alloc * cols);
  const bool vec = dtype == GIFT_F32 && n % 4 == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(o.hi) % 8 == 0 && reinterpret_cast<uintptr_t>(o.lo) % 8 == 0;
  if (vec) {
    const int64_t n4 = n / 4;
    const unsigned grid = (unsigned)std::min<int64_t>(cdiv(n4, 256), (int64_t)device_sm_count() * 16);
    k_split4<<<grid, 256, 0, s>>>(static_cast<const float4*>(x), n4, reinterpret_cast<uint2*>(o.hi),
                                  reinterpret_cast<uint2*>(o.lo));
    GIFT_LAUNCHED("k_split4");
    return o;
  }
  if (dtype == GIFT_F32)
    k_split_any<float><<<(unsigned)cdiv(n, 256), 256, 0, s>>>(static_cast<const float*>(x), n, o.hi, o.lo);
  else
    k_split_any<__nv_bfloat16><<<(unsigned)cdiv(n, 256), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(x), n,
                                                                        o.hi, o.lo);
  GIFT_LAUNCHED("k_split_any");
  return o;
}

// transposed operand: out [cols, ld] with ld = rows rounded up to 64; two-part
// for FP32 input, one-part (lo null) for BF16 input, which BF16 holds exactly
Operand make_transposed(const void* x, int dtype, int64_t rows, int64_t cols, int64_t& ld, Scratch& sc,
                        cudaStream_t s) {
  Operand o;
  ld = cdiv(rows, 64) * 64;
  o.rows_alloc = cols + 128;
  o.hi = sc.get<__nv_bfloat16>((size_t)o.rows_alloc * ld);
  if (dtype == GIFT_F32) o.lo = sc.get<__nv_bfloat16>((size_t)o.rows_alloc * ld);
  if (dtype != GIFT_F32 && cols % 8 == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0 &&
      reinterpret_cast<uintptr_t>(o.hi) % 16 == 0) {
    const dim3 g64((unsigned)cdiv(cols, 64), (unsigned)cdiv(ld, 64));
    k_transpose_bf16<<<g64, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(x), rows, cols, o.hi, ld);
    GIFT_LAUNCHED("k_transpose_bf16");
    return o;
  }
  const dim3 grid((unsigned)cdiv(cols, 32), (unsigned)cdiv(ld, 32)), blk(32, 8);
  if (dtype == GIFT_F32)
    k_transpose_split<float><<<grid, blk, 0, s>>>(static_cast<const float*>(x), rows, cols, o.hi, o.lo, ld);
  else
    k_transpose_split<__nv_bfloat16><<<grid, blk, 0, s>>>(static_cast<const __nv_bfloat16*>(x), rows, cols, o.hi,
                                                          o.lo, ld);
  GIFT_LAUNCHED("k_transpose_split");
  return o;
}

float* as_float(const void* x, int dtype, int64_t n, Scratch& sc, cudaStream_t s) {
  if (dtype == GIFT_F32) return const_cast<float*>(static_cast<const float*>(x));
  float* f = sc.get<float>((size_t)n);
  k_to_float<__nv_bfloat16><<<(unsigned)cdiv(n, 256), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(x), n, f);
  GIFT_LAUNCHED("k_to_float");
  return f;
}

struct Proj {
  float* U;
  float* V;
  float* uinv;
  float* vinv;
};

Proj project(const void* q, int64_t nq, const void* p, int64_t nr, const void* W, int din, int dout, int dtype,
             int* err, Scratch& sc, cudaStream_t s) {
  Proj P;
  if (W) {
    const Operand Qo = make_operand(q, dtype, nq, din, false, sc, s);
    const Operand Po = make_operand(p, dtype, nr, din, false, sc, s);
    const Operand Wo = make_operand(W, dtype, dout, din, false, sc, s);
    P.U = sc.get<float>((size_t)nq * dout);
    P.V = sc.get<float>((size_t)nr * dout);
    gemm_tc(Qo.hi, Qo.lo, nq, Qo.rows_alloc, 0, Wo.hi, Wo.lo, dout, Wo.rows_alloc, 0, din, P.U, dout, 0, err, s);
    gemm_tc(Po.hi, Po.lo, nr, Po.rows_alloc, 0, Wo.hi, Wo.lo, dout, Wo.rows_alloc, 0, din, P.V, dout, 0, err, s);
  } else {
    P.U = as_float(q, dtype, nq * din, sc, s);
    P.V = as_float(p, dtype, nr * din, sc, s);
  }
  P.uinv = sc.get<float>(nq);
  P.vinv = sc.get<float>(nr);
  launch_row_invnorm(P.U, nq, dout, P.uinv, s);
  launch_row_invnorm(P.V, nr, dout, P.vinv, s);
  return P;
}

int32_t* device_offsets(const std::vector<int32_t>& h_qoff, Scratch& sc, cudaStream_t s) {
  int32_t* d = sc.get<int32_t>(h_qoff.size());
  GIFT_CUDA(cudaMemcpyAsync(d, h_qoff.data(), h_qoff.size() * 4, cudaMemcpyHostToDevice, s));
  return d;
}

int* device_flag(Scratch& sc, cudaStream_t s) {
  int* f = sc.get<int>(1);
  GIFT_CUDA(cudaMemsetAsync(f, 0, sizeof(int), s));
  return f;
}

}  // namespace

void match_forward(const void* q, const std::vector<int32_t>& h_qoff, int32_t Bq, const void* p, int32_t Np,
                   int32_t nv, const void* W, int32_t din, int32_t dout, int32_t dtype, float* S, int16_t* argmax,
                   Scratch& sc, cudaStream_t s) {
  const int64_t nq = h_qoff[Bq];
  const int64_t nr = (int64_t)Np * nv;
  int* err = device_flag(sc, s);
  const Proj P = project(q, nq, p, nr, W, din, dout, dtype, err, sc, s);
  const Operand Uo = make_operand(P.U, GIFT_F32, nq, dout, true, sc, s);
  const Operand Vo = make_operand(P.V, GIFT_F32, nr, dout, true, sc, s);
  int32_t* d_qoff = device_offsets(h_qoff, sc, s);
  segmax_tc(Uo.hi, Uo.lo, Uo.rows_alloc, P.uinv, Vo.hi, Vo.lo, Vo.rows_alloc, P.vinv, nr, nv, dout, d_qoff, h_qoff,
            Bq, S, argmax, err, sc, s);
}

void match_backward(const void* q, const std::vector<int32_t>& h_qoff, int32_t Bq, const void* p, int32_t Np,
                    int32_t nv, const void* W, int32_t din, int32_t dout, int32_t dtype, const float* gS,
                    const int16_t* argmax, float* dW, float* dQ, float* dP, Scratch& sc, cudaStream_t s) {
  const int64_t nq = h_qoff[Bq];
  const int64_t nr = (int64_t)Np * nv;
  int* err = device_flag(sc, s);
  const Proj P = project(q, nq, p, nr, W, din, dout, dtype, err, sc, s);
  int32_t* d_qoff = device_offsets(h_qoff, sc, s);
  int32_t* vquery = sc.get<int32_t>(nq);
  k_view_query<<<(unsigned)Bq, 128, 0, s>>>(d_qoff, vquery);
  GIFT_LAUNCHED("k_view_query");
  // gradients w.r.t. the projected views (without a projection these are dQ, dP)
  float* dU = (W || !dQ) ? sc.get<float>((size_t)nq * dout) : dQ;
  float* dV = (W || !dP) ? sc.get<float>((size_t)nr * dout) : dP;
  float* vcoef = sc.get<float>(nq);
  k_view_coef<<<(unsigned)cdiv(nq, 256), 256, 0, s>>>(vquery, d_qoff, nq, vcoef);
  GIFT_LAUNCHED("k_view_coef");
  int16_t* amT = sc.get<int16_t>((size_t)nq * Np);
  float* wU = sc.get<float>((size_t)nq * Np);
  float* wV = sc.get<float>((size_t)nq * Np);
  k_onehot_prep<<<dim3((unsigned)cdiv(Np, 32), (unsigned)cdiv(nq, 32)), dim3(32, 8), 0, s>>>(
      argmax, nq, Np, nv, vquery, vcoef, gS, P.vinv, P.uinv, amT, wU, wV);
  GIFT_LAUNCHED("k_onehot_prep");
  float* G = sc.get<float>((size_t)std::max(nq, nr) * dout);  // G = A V, then H = A^T U
  GIFT_REQUIRE(dout % 4 == 0, "projected width must be a multiple of 4");
  const int sms = device_sm_count();
  {
    int64_t ldr = 0;
    const Operand Vt = make_transposed(P.V, GIFT_F32, nr, dout, ldr, sc, s);  // [dout, ldr], K = database views
    OneHotPolicy pol;
    pol.M = nq;
    pol.N = dout;
    pol.nkb = (int)(ldr / 64);
    pol.nq = nq;
    pol.nr = nr;
    pol.Np = Np;
    pol.nv = nv;
    pol.amT = amT;
    pol.gS = gS;
    pol.vquery = vquery;
    pol.vcoef = vcoef;
    pol.kinv = P.vinv;
    pol.wT = wU;
    pol.C = G;
    pol.fast = nv % 64 == 0 && nr < ((int64_t)1 << 31);
    pol.kb_per_shape = nv / 64;
    const CUtensorMap tB = make_tmap_bf16(Vt.hi, Vt.rows_alloc, ldr, 128);
    const CUtensorMap tB2 = make_tmap_bf16(Vt.lo, Vt.rows_alloc, ldr, 128);
    tc::launch_engine(tB, tB, tB2, tB2, pol, err, (int)std::min<int64_t>(sms, cdiv(nq, tc::kTM) * cdiv(dout, 128)),
                      s);
    k_tangent<<<(unsigned)cdiv(nq, 8), 256, 0, s>>>(P.U, P.uinv, G, nq, dout, dU);
    GIFT_LAUNCHED("k_tangent");
  }
  {
    // the (shape, query view) entries grouped by their argmax database view, in
    // ascending entry order (stable sorts), then one warp per database view
    const int64_t ne = nq * (int64_t)Np;
    GIFT_REQUIRE(ne < (int64_t)INT32_MAX && nr + 1 < (int64_t)INT32_MAX,
                 "query views x database shapes must stay below 2^31 for the gradient");
    int32_t* perm = sc.get<int32_t>((size_t)ne);
    int64_t* beg = sc.get<int64_t>((size_t)nr);
    int32_t* cnt = sc.get<int32_t>((size_t)nr);
    if (nv <= kCsrMaxNv) {  // per shape: a counting sort over its N_v views
      const size_t smem = (size_t)33 * nv * sizeof(int);
      GIFT_CUDA(cudaFuncSetAttribute(k_onehot_csr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_onehot_csr<<<(unsigned)Np, kCsrT, smem, s>>>(amT, nq, nv, perm, beg, cnt);
      GIFT_LAUNCHED("k_onehot_csr");
    } else {  // many views per shape: one radix sort of all entries by database view
      int32_t* keys = sc.get<int32_t>((size_t)ne);
      k_onehot_keys<<<(unsigned)cdiv(ne, (int64_t)256), 256, 0, s>>>(amT, nq, Np, nv, keys);
      GIFT_LAUNCHED("k_onehot_keys");
      int32_t* skeys = sc.get<int32_t>((size_t)ne);
      stable_sort_by_key(keys, ne, (int32_t)(nr + 1), perm, skeys, sc, s);
      int64_t* off = sc.get<int64_t>((size_t)nr + 2);
      bin_offsets(skeys, ne, (int32_t)(nr + 1), off, s);
      k_off_to_groups<<<(unsigned)cdiv(nr, (int64_t)256), 256, 0, s>>>(off, nr, beg, cnt);
      GIFT_LAUNCHED("k_off_to_groups");
    }
    k_segment_rows_sum<<<(unsigned)cdiv(nr, (int64_t)8), 256, 0, s>>>(P.U, perm, beg, cnt, wV, nq, nr, dout, G);
    GIFT_LAUNCHED("k_segment_rows_sum");
    k_tangent<<<(unsigned)cdiv(nr, 8), 256, 0, s>>>(P.V, P.vinv, G, nr, dout, dV);
    GIFT_LAUNCHED("k_tangent");
  }
  if (!W) return;
  if (dW) {
    int64_t ldq = 0, ldr = 0;
    const Operand dUt = make_transposed(dU, GIFT_F32, nq, dout, ldq, sc, s);
    const Operand Qt = make_transposed(q, dtype, nq, din, ldq, sc, s);
    gemm_tc(dUt.hi, dUt.lo, dout, dUt.rows_alloc, ldq, Qt.hi, Qt.lo, din, Qt.rows_alloc, ldq, (int)ldq, dW, din, 0,
            err, s);
    const Operand dVt = make_transposed(dV, GIFT_F32, nr, dout, ldr, sc, s);
    const Operand Pt = make_transposed(p, dtype, nr, din, ldr, sc, s);
    gemm_tc(dVt.hi, dVt.lo, dout, dVt.rows_alloc, ldr, Pt.hi, Pt.lo, din, Pt.rows_alloc, ldr, (int)ldr, dW, din, 1,
            err, s);
  }
  if (dQ || dP) {
    int64_t ldo = 0;
    const Operand Wt = make_transposed(W, dtype, dout, din, ldo, sc, s);  // [din, ldo], K = dout
    if (dQ) {
      const Operand dUo = make_operand(dU, GIFT_F32, nq, dout, true, sc, s);
      gemm_tc(dUo.hi, dUo.lo, nq, dUo.rows_alloc, dout, Wt.hi, Wt.lo, din, Wt.rows_alloc, ldo, dout, dQ, din, 0, err,
              s);
    }
    if (dP) {
      const Operand dVo = make_operand(dV, GIFT_F32, nr, dout, true, sc, s);
      gemm_tc(dVo.hi, dVo.lo, nr, dVo.rows_alloc, dout, Wt.hi, Wt.lo, din, Wt.rows_alloc, ldo, dout, dP, din, 0, err,
              s);
    }
  }
}

}  // namespace gift
