// Matching score of Eq. 3 after a learned linear view projection u = W q,
// and its gradient through the argmax view pair: products on the tensor
// cores, the gradient's one-hot gathers on the CUDA cores.
//
// Forward: U = Q W^T and V = P W^T (engine GEMMs; BF16 inputs multiply
// exactly in one product, FP32 inputs in the two-part split), then the
// segmented-max contraction of U and V (two-part split, FP32-level) gives
// S and the first argmax j* of every (query view, shape).
// Backward, with c = grad_S[b, p] / |V(x_b)| and s = u_i.v_j*/(|u_i||v_j*|):
//   dU_i  = (1/|u_i|)  ( g_i - (g_i . u_i/|u_i|) u_i/|u_i| ),  g_i = sum_p c v_j*/|v_j*|
//   dV_r  = (1/|v_r|)  ( h_r - (h_r . v_r/|v_r|) v_r/|v_r| ),  h_r = sum_{(i,p): j*=r} c u_i/|u_i|
// (the projections use s = g-weighted cosines: sum_p c s = g_i . u_i/|u_i|).
// G = A V and H = A^T U, with the one-hot matrix A[i, r] = c / |v_r| (c / |u_i| for
// H) where r is the argmax view of (i, shape(r)), are gathers on the CUDA cores: N_v
// times fewer multiply-adds than the dense products, FP32 sums in a fixed order. A
// block stages slices of V (of U for H) and of the shape-major argmax in shared
// memory and adds one staged row per (query view, shape) entry. Then
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

// ---------------------------------------------------------------- staged copies
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- G = A V on the CUDA cores
// G[i] = sum_p wU[p, i] V[p N_v + j(i, p)]: every (query view, shape) entry adds one
// row of V, so the product has N_v times fewer multiply-adds than the dense one-hot
// GEMM. A block owns 256 query views x 128 columns (16 warps of 16 views, 4 columns
// per lane, accumulators in registers) and walks the shapes in ascending order. A
// step stages, in shared memory (cp.async, three stages), the rows of up to 64
// database views restricted to the block's columns together with the entry records
// of the block's query views in those shapes: a row of V leaves L2 once per block
// instead of once per entry, and each entry is one broadcast record read, one
// 512-byte shared-memory read and four multiply-adds. A step is up to kGShapes whole
// shapes of at most 64 views together, or one 64-view piece of a larger shape. The
// steps may be split into parts (blockIdx.z) whose partial sums k_tangent adds in
// part order: the result does not depend on the launch.
constexpr int kGT = 512, kGRows = 256, kGCols = 128, kGStages = 3, kGViews = 64, kGShapes = 8;
constexpr int kGRecOff = (kGViews + 1) * kGCols * 4;            // 33,280: V rows + one zero row
constexpr int kGStageBytes = kGRecOff + kGShapes * kGRows * 8;  // 49,664: + records [kGShapes][kGRows]
static_assert(kGStageBytes % 16 == 0 && kGRecOff % 16 == 0, "stage alignment");

struct GatherSteps {
  int spc;  // whole shapes per step (N_v <= 64); 0: 64-view pieces of one shape
  int nch;  // pieces per shape (N_v > 64)
  int n;    // steps
};

// entry record of (query view i, shape p) for the gather: the weight wU and
//  - whole-shape steps (spc > 0): the staged row of the argmax view in float4
//    units, ((p mod spc) N_v + j) * 32, or the zero row kGViews * 32 (weight 0)
//    when the entry has no argmax;
//  - 64-view pieces (spc = 0): the argmax view j, or -1.
__device__ __forceinline__ float2 g_record(int spc, int64_t p, int nv, int j, float wu) {
  if (spc > 0) return make_float2(wu, __int_as_float(j >= 0 ? ((int)(p % spc) * nv + j) * 32 : kGViews * 32));
  return make_float2(wu, __int_as_float(j));
}

// shapes [p0, p0 + nps) and database views [vb, vb + nvs) of step s
__device__ __forceinline__ void g_step(const GatherSteps& st, int s, int nv, int Np, int& p0, int& nps, int64_t& vb,
                                       int& nvs) {
  if (st.spc > 0) {
    p0 = s * st.spc;
    nps = min(st.spc, Np - p0);
    vb = (int64_t)p0 * nv;
    nvs = nps * nv;
  } else {
    p0 = s / st.nch;
    const int ch = s - p0 * st.nch;
    nps = 1;
    vb = (int64_t)p0 * nv + ch * kGViews;
    nvs = min(kGViews, nv - ch * kGViews);
  }
}

// one entry: acc += w * staged row
__device__ __forceinline__ void g_add(float (&acc)[4], float w, const float4 x) {
  acc[0] = fmaf(w, x.x, acc[0]);
  acc[1] = fmaf(w, x.y, acc[1]);
  acc[2] = fmaf(w, x.z, acc[2]);
  acc[3] = fmaf(w, x.w, acc[3]);
}

// gR: [Np, ldq] entry records (ldq a multiple of kGRows; no entry past nq);
// V: [nr, dout] (16-byte aligned, dout % 4 == 0); Gp: [parts, nq, dout]
__global__ __launch_bounds__(kGT, 1) void k_gather_views(const float* __restrict__ V, const float2* __restrict__ gR,
                                                         int64_t nq, int64_t ldq, int Np, int nv, int dout,
                                                         GatherSteps st, float* __restrict__ Gp) {
  extern __shared__ __align__(16) uint8_t g_sm[];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int64_t i0 = (int64_t)blockIdx.x * kGRows;
  const int c0 = blockIdx.y * kGCols;
  const int part = blockIdx.z, parts = gridDim.z;
  const int s0 = (int)((int64_t)st.n * part / parts), s1 = (int)((int64_t)st.n * (part + 1) / parts);
  for (int t = tid; t < kGStages * 32; t += kGT)  // the zero row of every stage (never a copy target)
    *reinterpret_cast<float4*>(g_sm + (t >> 5) * kGStageBytes + kGViews * kGCols * 4 + (t & 31) * 16) =
        make_float4(0.f, 0.f, 0.f, 0.f);
  auto issue = [&](int s) {
    if (s < s1) {
      uint8_t* buf = g_sm + ((s - s0) % kGStages) * kGStageBytes;
      int p0, nps, nvs;
      int64_t vb;
      g_step(st, s, nv, Np, p0, nps, vb, nvs);
      for (int t = tid; t < nvs * 32; t += kGT) {  // rows of V, 16-byte pieces of the column slice
        const int row = t >> 5, q = t & 31, c = c0 + 4 * q;
        if (c < dout) cp_async16(buf + (row * kGCols + 4 * q) * 4, V + (vb + row) * dout + c);
      }
      for (int t = tid; t < nps * 128; t += kGT) {  // per shape: 256 records, 128 pieces
        const int ps = t >> 7, q = t & 127;
        cp_async16(buf + kGRecOff + ps * (kGRows * 8) + 16 * q, gR + (int64_t)(p0 + ps) * ldq + i0 + 2 * q);
      }
    }
    cp_async_commit();  // empty groups past the last step keep the wait count uniform
  };
  float acc[16][4];
#pragma unroll
  for (int k = 0; k < 16; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[k][q] = 0.f;
#pragma unroll
  for (int k = 0; k < kGStages - 1; ++k) issue(s0 + k);
  for (int s = s0; s < s1; ++s) {
    cp_async_wait<kGStages - 2>();  // this step's copies have landed ...
    __syncthreads();                // ... for every thread, and the step before is done with its buffer
    issue(s + kGStages - 1);
    const uint8_t* buf = g_sm + ((s - s0) % kGStages) * kGStageBytes;
    const float4* vs = reinterpret_cast<const float4*>(buf) + lane;
    int p0, nps, nvs;
    int64_t vb;
    g_step(st, s, nv, Np, p0, nps, vb, nvs);
    for (int ps = 0; ps < nps; ++ps) {
      // the warp's 16 records, two per 16-byte broadcast read
      const float4* rp = reinterpret_cast<const float4*>(buf + kGRecOff + (ps * kGRows + 16 * w) * 8);
      if (st.spc > 0) {  // the record holds the staged row: no test
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 r = rp[q];
          g_add(acc[2 * q], r.x, vs[__float_as_int(r.y)]);
          g_add(acc[2 * q + 1], r.z, vs[__float_as_int(r.w)]);
        }
      } else {  // 64-view piece of a shape: the argmax view must fall inside it
        const int base = (int)((int64_t)p0 * nv - vb);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 r = rp[q];
          const int l0 = base + __float_as_int(r.y), l1 = base + __float_as_int(r.w);
          if ((unsigned)l0 < (unsigned)nvs) g_add(acc[2 * q], r.x, vs[l0 * 32]);
          if ((unsigned)l1 < (unsigned)nvs) g_add(acc[2 * q + 1], r.z, vs[l1 * 32]);
        }
      }
    }
  }
  cp_async_wait<0>();
  const int c = c0 + 4 * lane;
  if (c >= dout) return;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int64_t i = i0 + 16 * w + k;
    if (i < nq)
      *reinterpret_cast<float4*>(Gp + ((int64_t)part * nq + i) * dout + c) =
          make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
  }
}

// shape-major argmax and one-hot weights, rows padded to ldq: for every (query view i,
// shape p), j = argmax[i, p], the gather record of wU = c / |v_{p nv + j}| (g_record)
// and wV = c / |u_i|, with c = grad_S[b, p] / |V(x_b)|; j = -1 (no entry, zero
// weights) for an argmax outside [0, N_v) and for the padding views nq <= i < ldq
__global__ void k_onehot_prep(const int16_t* __restrict__ argmax, int64_t nq, int64_t ldq, int Np, int nv, int spc,
                              const int32_t* __restrict__ vquery, const float* __restrict__ vcoef,
                              const float* __restrict__ gS, const float* __restrict__ vinv,
                              const float* __restrict__ uinv, int16_t* __restrict__ amT, float2* __restrict__ gR,
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
    if (i >= ldq || p >= Np) continue;
    const int j = i < nq ? (int)t[threadIdx.x][k] : -1;
    const int64_t e = p * ldq + i;
    if (j < 0 || j >= nv) {
      amT[e] = -1;
      gR[e] = g_record(spc, p, nv, -1, 0.f);
      wV[e] = 0.f;
      continue;
    }
    const float c = gS[(int64_t)vquery[i] * Np + p] * vcoef[i];
    amT[e] = (int16_t)j;
    gR[e] = g_record(spc, p, nv, j, c * vinv[p * nv + j]);
    wV[e] = c * uinv[i];
  }
}

__global__ void k_view_coef(const int32_t* __restrict__ vquery, const int32_t* __restrict__ qoff, int64_t nq,
                            float* __restrict__ coef) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const int b = vquery[i];
  coef[i] = 1.f / (float)(qoff[b + 1] - qoff[b]);
}

// out_r = inv_r (g_r - (g_r . x_r inv_r) x_r inv_r): the gradient through x / |x| (warp per
// row); g_r is the sum of `parts` partial rows G[s pstride + r dout], added in part order
__global__ void k_tangent(const float* __restrict__ X, const float* __restrict__ inv, const float* __restrict__ G,
                          int parts, int64_t pstride, int64_t n, int dout, float* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const float iv = inv[r];
  const float* x = X + r * dout;
  const float* g = G + r * dout;
  auto g_at = [&](int d) {
    float v = g[d];
    for (int s = 1; s < parts; ++s) v += g[s * pstride + d];
    return v;
  };
  float dot = 0.f;
  for (int d = lane; d < dout; d += 32) dot = fmaf(x[d], g_at(d), dot);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  const float t = dot * iv * iv;
  for (int d = lane; d < dout; d += 32) out[r * dout + d] = iv * (g_at(d) - t * x[d]);
}

__global__ void k_view_query(const int32_t* __restrict__ qoff, int32_t* __restrict__ vq) {
  const int b = blockIdx.x;
  for (int v = qoff[b] + threadIdx.x; v < qoff[b + 1]; v += blockDim.x) vq[v] = b;
}

// ---------------------------------------------------------------- H = A^T U on the CUDA cores
// Every database view's row of H is the weighted sum of the query views whose
// argmax in its shape is that view:
//   H[p N_v + j] = sum_{i : j(i, p) = j} wV[p, i] U[i]
// (N_v times fewer multiply-adds than the dense one-hot GEMM), summed in ascending
// query view order: a result that does not depend on the launch.
//
// Shapes of up to 1,024 views: the entries of each shape are grouped by their argmax
// view (a counting sort per shape in shared memory), then one warp per database view
// sums its entries' rows of U, gathered from L2 (U is L2-resident).
// Larger shapes (the sort's per-warp counts would not fit in shared memory): a block
// owns 256 database views (flattened; at most kHShapes shapes, N_v >= 16) x 128
// columns, warp w the 16 views from 16 w on, 4 columns per lane with the accumulators
// in registers. A step stages 64 query views' rows of U (the column slice) and the
// argmax and weight of those query views in the block's shapes (cp.async, three
// stages); a warp finds the query views of each of its database views with two
// ballots over the staged argmax and adds their staged rows.
constexpr int kHT = 512, kHRows = 256, kHQ = 64, kHStages = 3, kHShapes = 18;
constexpr int kHMinNv = 16;                                  // kHRows / kHMinNv + 2 <= kHShapes
constexpr int kHAmOff = kHQ * kGCols * 4;                    // 32,768: argmax [kHShapes][kHQ] int16
constexpr int kHWOff = kHAmOff + kHShapes * kHQ * 2;         // 35,072: weight [kHShapes][kHQ] float
constexpr int kHStageBytes = kHWOff + kHShapes * kHQ * 4;    // 39,680
static_assert(kHStageBytes % 16 == 0 && kHWOff % 16 == 0, "stage alignment");
static_assert(kHRows / kHMinNv + 2 <= kHShapes, "shapes of one block");

// amT, wV: [Np, ldq] (ldq a multiple of kHQ; argmax -1 past nq); U: [nq, dout]
// (16-byte aligned, dout % 4 == 0); H: [nr, dout]
__global__ __launch_bounds__(kHT, 1) void k_gather_entries(const float* __restrict__ U, const int16_t* __restrict__ amT,
                                                           const float* __restrict__ wV, int64_t nq, int64_t ldq,
                                                           int64_t nr, int nv, int dout, float* __restrict__ H) {
  extern __shared__ __align__(16) uint8_t h_sm[];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int64_t r0 = (int64_t)blockIdx.x * kHRows;
  const int c0 = blockIdx.y * kGCols;
  const int64_t ps0 = r0 / nv;
  const int ns = (int)((min(r0 + kHRows, nr) - 1) / nv - ps0 + 1);  // shapes of the block (<= kHShapes)
  const int nsteps = (int)cdiv(nq, (int64_t)kHQ);
  auto issue = [&](int s) {
    if (s < nsteps) {
      uint8_t* buf = h_sm + (s % kHStages) * kHStageBytes;
      const int64_t i0 = (int64_t)s * kHQ;
      for (int t = tid; t < kHQ * 32; t += kHT) {  // rows of U, 16-byte pieces of the column slice
        const int row = t >> 5, q = t & 31, c = c0 + 4 * q;
        if (c < dout && i0 + row < nq) cp_async16(buf + (row * kGCols + 4 * q) * 4, U + (i0 + row) * dout + c);
      }
      for (int t = tid; t < ns * 24; t += kHT) {  // per shape: 8 pieces of argmax, 16 of weight
        const int ps = t / 24, q = t - ps * 24;
        const int64_t e = (ps0 + ps) * ldq + i0;
        if (q < 8)
          cp_async16(buf + kHAmOff + (ps * kHQ + 8 * q) * 2, amT + e + 8 * q);
        else
          cp_async16(buf + kHWOff + (ps * kHQ + 4 * (q - 8)) * 4, wV + e + 4 * (q - 8));
      }
    }
    cp_async_commit();  // empty groups past the last step keep the wait count uniform
  };
  // shape and view of the warp's first database view
  const int64_t rw = r0 + 16 * w;
  const int pw0 = (int)(rw / nv - ps0), jw0 = (int)(rw % nv);
  float acc[16][4];
#pragma unroll
  for (int k = 0; k < 16; ++k)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[k][q] = 0.f;
#pragma unroll
  for (int k = 0; k < kHStages - 1; ++k) issue(k);
  for (int s = 0; s < nsteps; ++s) {
    cp_async_wait<kHStages - 2>();  // this step's copies have landed ...
    __syncthreads();                // ... for every thread, and the step before is done with its buffer
    issue(s + kHStages - 1);
    const uint8_t* buf = h_sm + (s % kHStages) * kHStageBytes;
    const float4* us = reinterpret_cast<const float4*>(buf);
    const int16_t* as = reinterpret_cast<const int16_t*>(buf + kHAmOff);
    const float* ws = reinterpret_cast<const float*>(buf + kHWOff);
    int ps = pw0, j = jw0, cur = -1;
    int ja = -1, jb = -1;
    float wa = 0.f, wb = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (rw + k < nr) {  // uniform over the warp
        if (ps != cur) {  // lane l holds query views l and l + 32 of the step
          cur = ps;
          ja = as[ps * kHQ + lane];
          jb = as[ps * kHQ + 32 + lane];
          wa = ws[ps * kHQ + lane];
          wb = ws[ps * kHQ + 32 + lane];
        }
        unsigned m = __ballot_sync(0xffffffffu, ja == j);
        while (m) {
          const int l = __ffs(m) - 1;
          m &= m - 1;
          const float wk = __shfl_sync(0xffffffffu, wa, l);
          const float4 x = us[l * 32 + lane];
          acc[k][0] = fmaf(wk, x.x, acc[k][0]);
          acc[k][1] = fmaf(wk, x.y, acc[k][1]);
          acc[k][2] = fmaf(wk, x.z, acc[k][2]);
          acc[k][3] = fmaf(wk, x.w, acc[k][3]);
        }
        m = __ballot_sync(0xffffffffu, jb == j);
        while (m) {
          const int l = __ffs(m) - 1;
          m &= m - 1;
          const float wk = __shfl_sync(0xffffffffu, wb, l);
          const float4 x = us[(l + 32) * 32 + lane];
          acc[k][0] = fmaf(wk, x.x, acc[k][0]);
          acc[k][1] = fmaf(wk, x.y, acc[k][1]);
          acc[k][2] = fmaf(wk, x.z, acc[k][2]);
          acc[k][3] = fmaf(wk, x.w, acc[k][3]);
        }
      }
      if (++j == nv) {
        j = 0;
        ++ps;
      }
    }
  }
  cp_async_wait<0>();
  const int c = c0 + 4 * lane;
  if (c >= dout) return;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int64_t r = rw + k;
    if (r < nr)
      *reinterpret_cast<float4*>(H + r * dout + c) = make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
  }
}

// The entries of shape p grouped by their argmax view j, ascending query view within a
// group (a stable counting sort, one block per shape): perm[p ld + ...] holds the entry
// indices e = p ld + i, beg[p N_v + j] the first position of view j's group and
// cnt[p N_v + j] its size; entries without an argmax (j = -1) are left out. Shared
// memory: 32 x N_v per-warp counts and N_v running group ends.
constexpr int kCsrT = 1024;
constexpr int kCsrMaxNv = 1024;  // 33 x 1024 ints of shared memory
static_assert(kCsrMaxNv >= kHMinNv, "the staged gather takes the larger shapes");
__global__ __launch_bounds__(kCsrT) void k_onehot_csr(const int16_t* __restrict__ amT, int64_t nq, int64_t ld,
                                                      int nv,
                                                      int32_t* __restrict__ perm, int64_t* __restrict__ beg,
                                                      int32_t* __restrict__ cnt) {
  extern __shared__ int csr_sm[];
  int* wc = csr_sm;            // [32][nv]
  int* base = csr_sm + 32 * nv;  // [nv]
  const int p = blockIdx.x, t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int16_t* a = amT + (int64_t)p * ld;
  const int64_t e0 = (int64_t)p * ld;
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

// H[r] = sum of wV[e] U[e mod ld] over the entries e of row r (perm[beg[r]] ..
// perm[beg[r] + cnt[r]]), in ascending e: one warp per database view, lane c owns columns
// 4 c + 128 t, up to kHCols columns per pass (dout % 4 == 0)
constexpr int kHCols = 512;
__global__ __launch_bounds__(256) void k_segment_rows_sum(const float* __restrict__ U, const int32_t* __restrict__ perm,
                                                          const int64_t* __restrict__ beg,
                                                          const int32_t* __restrict__ cnt,
                                                          const float* __restrict__ wT, int64_t ld, int64_t nr,
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
        src = (int64_t)(e % ld) * dout;
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
  // steps of the query-side gather
  GatherSteps st;
  if (nv <= kGViews) {
    st.spc = std::min(kGShapes, kGViews / nv);
    st.nch = 1;
    st.n = (int)cdiv((int64_t)Np, (int64_t)st.spc);
  } else {
    st.spc = 0;
    st.nch = (int)cdiv((int64_t)nv, (int64_t)kGViews);
    GIFT_REQUIRE((int64_t)Np * st.nch < INT32_MAX, "too many database views for the gradient");
    st.n = Np * st.nch;
  }
  // shape-major argmax, gather records and weights, query views padded to a multiple of the gather blocks
  const int64_t ldq = cdiv(nq, (int64_t)kGRows) * kGRows;
  int16_t* amT = sc.get<int16_t>((size_t)ldq * Np);
  float2* gR = sc.get<float2>((size_t)ldq * Np);
  float* wV = sc.get<float>((size_t)ldq * Np);
  k_onehot_prep<<<dim3((unsigned)cdiv(Np, 32), (unsigned)cdiv(ldq, 32)), dim3(32, 8), 0, s>>>(
      argmax, nq, ldq, Np, nv, st.spc, vquery, vcoef, gS, P.vinv, P.uinv, amT, gR, wV);
  GIFT_LAUNCHED("k_onehot_prep");
  GIFT_REQUIRE(dout % 4 == 0, "projected width must be a multiple of 4");
  // the staged copies read 16-byte pieces of the rows of U and V
  auto aligned16 = [&](float* x, int64_t n) {
    if (reinterpret_cast<uintptr_t>(x) % 16 == 0) return x;
    float* y = sc.get<float>((size_t)n);
    GIFT_CUDA(cudaMemcpyAsync(y, x, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return y;
  };
  const float* U16 = aligned16(P.U, nq * dout);
  const float* V16 = aligned16(P.V, nr * dout);
  const int sms = device_sm_count();
  {  // G = A V, then dU
    // parts of the step range: a block's time is ~ steps / parts, the launch takes
    // ceil(blocks x parts / SMs) rounds of one block per SM; partial rows cost a little
    const int64_t units = cdiv(nq, (int64_t)kGRows) * cdiv((int64_t)dout, (int64_t)kGCols);
    int parts = 1;
    double best = 1e30;
    for (int pc = 1; pc <= 8 && pc <= st.n; ++pc) {
      const double cost = (double)cdiv(units * pc, (int64_t)sms) / pc + 0.02 * pc;
      if (cost < best - 1e-9) {
        best = cost;
        parts = pc;
      }
    }
    float* Gp = sc.get<float>((size_t)parts * nq * dout);
    const size_t smem = (size_t)kGStages * kGStageBytes;
    GIFT_CUDA(cudaFuncSetAttribute(k_gather_views, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const dim3 grid((unsigned)cdiv(nq, (int64_t)kGRows), (unsigned)cdiv((int64_t)dout, (int64_t)kGCols),
                    (unsigned)parts);
    k_gather_views<<<grid, kGT, smem, s>>>(V16, gR, nq, ldq, Np, nv, dout, st, Gp);
    GIFT_LAUNCHED("k_gather_views");
    k_tangent<<<(unsigned)cdiv(nq, 8), 256, 0, s>>>(P.U, P.uinv, Gp, parts, nq * dout, nq, dout, dU);
    GIFT_LAUNCHED("k_tangent");
  }
  {  // H = A^T U, then dV
    float* H = sc.get<float>((size_t)nr * dout);
    if (nv <= kCsrMaxNv) {  // entries grouped per shape, then one warp per database view
      const int64_t ne = ldq * (int64_t)Np;
      GIFT_REQUIRE(ne < (int64_t)INT32_MAX, "query views x database shapes must stay below 2^31 for the gradient");
      int32_t* perm = sc.get<int32_t>((size_t)ne);
      int64_t* beg = sc.get<int64_t>((size_t)nr);
      int32_t* cnt = sc.get<int32_t>((size_t)nr);
      const size_t smem = (size_t)33 * nv * sizeof(int);
      GIFT_CUDA(cudaFuncSetAttribute(k_onehot_csr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_onehot_csr<<<(unsigned)Np, kCsrT, smem, s>>>(amT, nq, ldq, nv, perm, beg, cnt);
      GIFT_LAUNCHED("k_onehot_csr");
      k_segment_rows_sum<<<(unsigned)cdiv(nr, (int64_t)8), 256, 0, s>>>(U16, perm, beg, cnt, wV, ldq, nr, dout, H);
      GIFT_LAUNCHED("k_segment_rows_sum");
    } else {  // larger shapes: the staged gather
      const size_t smem = (size_t)kHStages * kHStageBytes;
      GIFT_CUDA(cudaFuncSetAttribute(k_gather_entries, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      const dim3 grid((unsigned)cdiv(nr, (int64_t)kHRows), (unsigned)cdiv((int64_t)dout, (int64_t)kGCols));
      k_gather_entries<<<grid, kHT, smem, s>>>(U16, amT, wV, nq, ldq, nr, nv, dout, H);
      GIFT_LAUNCHED("k_gather_entries");
    }
    k_tangent<<<(unsigned)cdiv(nr, 8), 256, 0, s>>>(P.V, P.vinv, H, 1, 0, nr, dout, dV);
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
