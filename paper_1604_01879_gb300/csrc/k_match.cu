// Matching score of Eq. 3 after a learned linear view projection u = W q,
// and its gradient through the argmax view pair, on the tensor cores.
//
// Forward: U = Q W^T and V = P W^T (engine GEMMs; BF16 inputs multiply
// exactly in one product, FP32 inputs in the two-part split), then the
// segmented-max contraction of U and V (two-part split, FP32-level) gives
// S and the first argmax j* of every (query view, shape).
// Backward, with c = grad_S[b, p] / |V(x_b)| and s = u_i.v_j*/(|u_i||v_j*|):
//   dU_i  = (1/|u_i|)  ( sum_p c v_j*/|v_j*|  - (sum_p c s) u_i/|u_i| )
//   dV_r  = (1/|v_r|)  ( sum_{(i,p): j*=r} c u_i/|u_i| - (sum c s) v_r/|v_r| )
// gathered on the CUDA cores (one block per query view for dU; per shape, a
// shared-memory accumulation over query views for dV, no atomics), then
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

// dU_i and s[i, p] = cos(u_i, v_{p*nv + j*}) for one query view per block:
// each warp walks a subset of the shapes, keeps u_i and its share of the dU
// accumulator in registers (lane owns dims lane, lane+32, ...), and the
// warps' partials are summed through shared memory at the end.
template <int DPL>  // dims per lane: dout <= 32 * DPL
__global__ __launch_bounds__(256) void k_grad_u(const float* __restrict__ U, const float* __restrict__ uinv,
                                                 const float* __restrict__ V, const float* __restrict__ vinv,
                                                 const int16_t* __restrict__ argmax, const float* __restrict__ gS,
                                                 const int32_t* __restrict__ vquery, const int32_t* __restrict__ qoff,
                                                 int Np, int nv, int dout, float* __restrict__ s_out,
                                                 float* __restrict__ dU) {
  __shared__ float part[8][DPL * 32];
  __shared__ float tot_w[8];
  const int64_t i = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = vquery[i];
  const float invV = 1.f / (float)(qoff[b + 1] - qoff[b]);
  const float ui = uinv[i];
  float u[DPL], acc[DPL];
#pragma unroll
  for (int k = 0; k < DPL; ++k) {
    const int d = lane + 32 * k;
    u[k] = d < dout ? U[i * dout + d] : 0.f;
    acc[k] = 0.f;
  }
  float tot = 0.f;
#pragma unroll 2
  for (int p = w; p < Np; p += 8) {
    const int64_t wi = i * Np + p;
    int j = argmax[wi];
    if (j < 0 || j >= nv) j = 0;  // argmax comes from the forward; never index outside the shape
    const int64_t r = (int64_t)p * nv + j;
    const float* v = V + r * dout;
    float vv[DPL];
    float dot = 0.f;
#pragma unroll
    for (int k = 0; k < DPL; ++k) {
      const int d = lane + 32 * k;
      vv[k] = d < dout ? v[d] : 0.f;
      dot = fmaf(u[k], vv[k], dot);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    const float vi = vinv[r];
    const float sc = dot * ui * vi;
    if (lane == 0) s_out[wi] = sc;
    const float c = gS[(int64_t)b * Np + p] * invV;
    const float cv = c * vi;
#pragma unroll
    for (int k = 0; k < DPL; ++k) acc[k] = fmaf(cv, vv[k], acc[k]);
    tot = fmaf(c, sc, tot);
  }
#pragma unroll
  for (int k = 0; k < DPL; ++k) part[w][lane + 32 * k] = acc[k];  // lanes past dout hold 0
  if (lane == 0) tot_w[w] = tot;
  __syncthreads();
  float T = 0.f;
#pragma unroll
  for (int ww = 0; ww < 8; ++ww) T += tot_w[ww];
  for (int d = threadIdx.x; d < dout; d += 256) {
    float a = 0.f;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) a += part[ww][d];
    dU[i * dout + d] = ui * (a - T * U[i * dout + d] * ui);
  }
}

// dV rows of shape p: one block per shape, 16 warps; warp w owns the shape's
// rows j = w, w + 16, ... (accumulators in registers, lane owns dims lane,
// lane + 32, ...), scans the argmax column of the shape for the query views
// that selected one of its rows and adds c * u_i / |u_i| there. No atomics;
// every row of U is read once per shape, from L2.
template <int DPL>
__global__ __launch_bounds__(512) void k_grad_v(const float* __restrict__ U, const float* __restrict__ uinv,
                                                 const float* __restrict__ V, const float* __restrict__ vinv,
                                                 const int16_t* __restrict__ argmax, const float* __restrict__ s,
                                                 const float* __restrict__ gS, const int32_t* __restrict__ vquery,
                                                 const int32_t* __restrict__ qoff, int64_t nq, int Np, int nv,
                                                 int dout, float* __restrict__ dV) {
  constexpr int RPW = 4;  // rows per warp per pass
  const int p = blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j0 = w * RPW; j0 < nv; j0 += 16 * RPW) {
    float acc[RPW][DPL];
    float ct[RPW];
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
      ct[t] = 0.f;
#pragma unroll
      for (int k = 0; k < DPL; ++k) acc[t][k] = 0.f;
    }
    for (int64_t i0 = 0; i0 < nq; i0 += 32) {
      const int64_t i = i0 + lane;
      int j = -1;
      if (i < nq) {
        j = argmax[i * Np + p];
        if (j < 0 || j >= nv) j = 0;
      }
      unsigned hit = __ballot_sync(0xffffffffu, j >= j0 && j < j0 + RPW);
      while (hit) {
        const int src = __ffs(hit) - 1;
        hit &= hit - 1;
        const int64_t ii = i0 + src;
        const int jj = __shfl_sync(0xffffffffu, j, src) - j0;
        const int b = vquery[ii];
        const float c = gS[(int64_t)b * Np + p] / (float)(qoff[b + 1] - qoff[b]);
        const float cu = c * uinv[ii];
        const float sc = s[ii * Np + p];
        const float* u = U + ii * dout;
#pragma unroll
        for (int t = 0; t < RPW; ++t) {
          if (t == jj) {
#pragma unroll
            for (int k = 0; k < DPL; ++k) {
              const int d = lane + 32 * k;
              if (d < dout) acc[t][k] = fmaf(cu, u[d], acc[t][k]);
            }
            ct[t] = fmaf(c, sc, ct[t]);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < RPW; ++t) {
      const int j = j0 + t;
      if (j >= nv) continue;
      const int64_t r = (int64_t)p * nv + j;
      const float vi = vinv[r];
#pragma unroll
      for (int k = 0; k < DPL; ++k) {
        const int d = lane + 32 * k;
        if (d < dout) dV[r * dout + d] = vi * (acc[t][k] - ct[t] * V[r * dout + d] * vi);
      }
    }
  }
}

__global__ void k_view_query(const int32_t* __restrict__ qoff, int32_t* __restrict__ vq) {
  const int b = blockIdx.x;
  for (int v = qoff[b] + threadIdx.x; v < qoff[b + 1]; v += blockDim.x) vq[v] = b;
}

// two-part BF16 operand with one TMA box of padding rows
struct Operand {
  __nv_bfloat16* hi = nullptr;
  __nv_bfloat16* lo = nullptr;  // null: one-part (exact BF16 input)
  int64_t rows_alloc = 0;
};

Operand make_operand(const void* x, int dtype, int64_t rows, int cols, bool force_split, Scratch& sc, cudaStream_t s) {
  Operand o;
  o.rows_alloc = rows + 128;
  const int64_t n = rows * cols;
  o.hi = sc.get<__nv_bfloat16>((size_t)o.rows_alloc * cols);
  const bool split = dtype == GIFT_F32 || force_split;
  if (split) o.lo = sc.get<__nv_bfloat16>((size_t)o.rows_alloc * cols);
  if (dtype == GIFT_F32)
    k_split_any<float><<<(unsigned)cdiv(n, 256), 256, 0, s>>>(static_cast<const float*>(x), n, o.hi, o.lo);
  else
    k_split_any<__nv_bfloat16><<<(unsigned)cdiv(n, 256), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(x), n,
                                                                        o.hi, o.lo);
  GIFT_LAUNCHED("k_split_any");
  return o;
}

// transposed two-part operand: out [cols, ld] with ld = rows rounded up to 64
Operand make_transposed(const void* x, int dtype, int64_t rows, int64_t cols, int64_t& ld, Scratch& sc,
                        cudaStream_t s) {
  Operand o;
  ld = cdiv(rows, 64) * 64;
  o.rows_alloc = cols + 128;
  o.hi = sc.get<__nv_bfloat16>((size_t)o.rows_alloc * ld);
  o.lo = sc.get<__nv_bfloat16>((size_t)o.rows_alloc * ld);
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
  float* sv = sc.get<float>((size_t)nq * Np);
  // gradients w.r.t. the projected views (without a projection these are dQ, dP)
  float* dU = (W || !dQ) ? sc.get<float>((size_t)nq * dout) : dQ;
  float* dV = (W || !dP) ? sc.get<float>((size_t)nr * dout) : dP;
  const int dpl = (int)cdiv(dout, 32);
  switch (dpl <= 1 ? 1 : dpl <= 2 ? 2 : dpl <= 4 ? 4 : dpl <= 8 ? 8 : dpl <= 16 ? 16 : dpl <= 32 ? 32 : 0) {
#define GIFT_GRAD_U(n)                                                                                      \
  case n:                                                                                                   \
    k_grad_u<n><<<(unsigned)nq, 256, 0, s>>>(P.U, P.uinv, P.V, P.vinv, argmax, gS, vquery, d_qoff, Np, nv, \
                                             dout, sv, dU);                                                 \
    break;
    GIFT_GRAD_U(1)
    GIFT_GRAD_U(2)
    GIFT_GRAD_U(4)
    GIFT_GRAD_U(8)
    GIFT_GRAD_U(16)
    GIFT_GRAD_U(32)
#undef GIFT_GRAD_U
    default:
      fail(GIFT_EINVAL, "d_out must be at most 1024 for the backward");
  }
  GIFT_LAUNCHED("k_grad_u");
  switch (dpl <= 1 ? 1 : dpl <= 2 ? 2 : dpl <= 4 ? 4 : dpl <= 8 ? 8 : dpl <= 16 ? 16 : dpl <= 32 ? 32 : 0) {
#define GIFT_GRAD_V(n)                                                                                      \
  case n:                                                                                                   \
    k_grad_v<n><<<(unsigned)Np, 512, 0, s>>>(P.U, P.uinv, P.V, P.vinv, argmax, sv, gS, vquery, d_qoff, nq, Np, \
                                             nv, dout, dV);                                                 \
    break;
    GIFT_GRAD_V(1)
    GIFT_GRAD_V(2)
    GIFT_GRAD_V(4)
    GIFT_GRAD_V(8)
    GIFT_GRAD_V(16)
    GIFT_GRAD_V(32)
#undef GIFT_GRAD_V
    default:
      fail(GIFT_EINVAL, "d_out must be at most 1024 for the backward");
  }
  GIFT_LAUNCHED("k_grad_v");
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
