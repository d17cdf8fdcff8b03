// Matching score of Eq. 3 after a learned linear view projection u = W q,
// and its gradient through the argmax view pair.
//
// Forward: U = Q W^T, V = P W^T (tile GEMMs), S and the first argmax j* of
// every (query view, shape) by the segmented-max kernel of the exact match.
// Backward, with c = grad_S[b, p] / |V(x_b)| and s = u_i.v_j*/(|u_i||v_j*|):
//   dU_i  = (1/|u_i|)  ( sum_p c v_j*/|v_j*|  - (sum_p c s) u_i/|u_i| )
//   dV_r  = (1/|v_r|)  ( sum_{(i,p): j*=r} c u_i/|u_i| - (sum c s) v_r/|v_r| )
//   dW    = dU^T Q + dV^T P,  dQ = dU W,  dP = dV W.
// dU is a gather over shapes (one block per query view), dV a per-shape
// accumulation over query views in shared memory (no atomics).
#include "gift_internal.cuh"
#include "segmax.cuh"
#include "sgemm_nt.cuh"

namespace gift {

namespace {

struct EpiStore {
  float* C;
  int64_t M, N, ldc;
  int accumulate;
  __device__ __forceinline__ void operator()(int64_t m0, int64_t n0, const SgemmFrag& f,
                                             float (&acc)[8][8]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t m = m0 + f.row(i);
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t n = n0 + f.col(j);
        if (n < N) {
          float* c = C + m * ldc + n;
          *c = accumulate ? *c + acc[i][j] : acc[i][j];
        }
      }
    }
  }
};

// out[c * ldo + r] = in[r * cols + c] for r < rows, c < cols; zero pad up to ldo
__global__ void k_transpose(const float* __restrict__ in, int64_t rows, int64_t cols, float* __restrict__ out,
                            int64_t ldo) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    t[y][threadIdx.x] = (r < rows && c < cols) ? in[r * cols + c] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int64_t c = c0 + y, r = r0 + threadIdx.x;
    if (c < cols && r < ldo) out[c * ldo + r] = t[threadIdx.x][y];
  }
}

// s[i, p] = cos(u_i, v_{p*nv + j*}) , one warp per (i, p)
__global__ void k_pair_cos(const float* __restrict__ U, const float* __restrict__ uinv,
                           const float* __restrict__ V, const float* __restrict__ vinv,
                           const int16_t* __restrict__ argmax, int64_t nq, int Np, int nv, int dout,
                           float* __restrict__ s) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nq * Np) return;
  const int64_t i = w / Np, p = w % Np;
  int j = argmax[w];
  if (j < 0 || j >= nv) j = 0;  // argmax comes from the forward; never index outside the shape
  const int64_t r = p * nv + j;
  const float* u = U + i * dout;
  const float* v = V + r * dout;
  float acc = 0.f;
  for (int d = lane; d < dout; d += 32) acc = fmaf(u[d], v[d], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) s[w] = acc * uinv[i] * vinv[r];
}

// dU_i, one block per query view
__global__ void k_grad_u(const float* __restrict__ U, const float* __restrict__ uinv,
                         const float* __restrict__ V, const float* __restrict__ vinv,
                         const int16_t* __restrict__ argmax, const float* __restrict__ s,
                         const float* __restrict__ gS, const int32_t* __restrict__ vquery,
                         const int32_t* __restrict__ qoff, int Np, int nv, int dout, float* __restrict__ dU) {
  extern __shared__ float acc[];  // [dout]
  __shared__ float tot;
  const int64_t i = blockIdx.x;
  const int b = vquery[i];
  const float invV = 1.f / (float)(qoff[b + 1] - qoff[b]);
  for (int d = threadIdx.x; d < dout; d += blockDim.x) acc[d] = 0.f;
  if (threadIdx.x == 0) tot = 0.f;
  __syncthreads();
  float t_local = 0.f;
  for (int p = 0; p < Np; ++p) {
    const float c = gS[(int64_t)b * Np + p] * invV;
    if (c == 0.f) continue;
    const int64_t w = i * Np + p;
    int j = argmax[w];
    if (j < 0 || j >= nv) j = 0;
    const int64_t r = (int64_t)p * nv + j;
    const float cv = c * vinv[r];
    const float* v = V + r * dout;
    for (int d = threadIdx.x; d < dout; d += blockDim.x) acc[d] = fmaf(cv, v[d], acc[d]);
    if (threadIdx.x == 0) t_local = fmaf(c, s[w], t_local);
  }
  if (threadIdx.x == 0) tot = t_local;
  __syncthreads();
  const float ui = uinv[i];
  for (int d = threadIdx.x; d < dout; d += blockDim.x)
    dU[i * dout + d] = ui * (acc[d] - tot * U[i * dout + d] * ui);
}

// dV rows of shape p, columns [d0, d1); one block per (shape, column chunk)
__global__ void k_grad_v(const float* __restrict__ U, const float* __restrict__ uinv,
                         const float* __restrict__ V, const float* __restrict__ vinv,
                         const int16_t* __restrict__ argmax, const float* __restrict__ s,
                         const float* __restrict__ gS, const int32_t* __restrict__ vquery,
                         const int32_t* __restrict__ qoff, int64_t nq, int Np, int nv, int dout, int dchunk,
                         float* __restrict__ dV) {
  extern __shared__ float sm[];  // acc [nv][dchunk] then ctot [nv]
  float* acc = sm;
  float* ctot = sm + (int64_t)nv * dchunk;
  const int p = blockIdx.x;
  const int d0 = blockIdx.y * dchunk;
  const int dw = min(dchunk, dout - d0);
  for (int t = threadIdx.x; t < nv * dchunk; t += blockDim.x) acc[t] = 0.f;
  for (int t = threadIdx.x; t < nv; t += blockDim.x) ctot[t] = 0.f;
  __syncthreads();
  for (int64_t i = 0; i < nq; ++i) {
    const int b = vquery[i];
    const float c = gS[(int64_t)b * Np + p] / (float)(qoff[b + 1] - qoff[b]);
    if (c == 0.f) continue;
    const int64_t w = i * Np + p;
    int j = argmax[w];
    if (j < 0 || j >= nv) j = 0;
    const float cu = c * uinv[i];
    const float* u = U + i * dout + d0;
    float* a = acc + (int64_t)j * dchunk;
    for (int d = threadIdx.x; d < dw; d += blockDim.x) a[d] = fmaf(cu, u[d], a[d]);
    if (threadIdx.x == 0) ctot[j] = fmaf(c, s[w], ctot[j]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nv * dw; t += blockDim.x) {
    const int j = t / dw, d = t % dw;
    const int64_t r = (int64_t)p * nv + j;
    const float vi = vinv[r];
    dV[r * dout + d0 + d] = vi * (acc[(int64_t)j * dchunk + d] - ctot[j] * V[r * dout + d0 + d] * vi);
  }
}

__global__ void k_view_query(const int32_t* __restrict__ qoff, int B, int32_t* __restrict__ vq) {
  const int b = blockIdx.x;
  for (int v = qoff[b] + threadIdx.x; v < qoff[b + 1]; v += blockDim.x) vq[v] = b;
}

struct Proj {
  const float* U;
  const float* V;
  float* uinv;
  float* vinv;
};

Proj project(const float* q, int64_t nq, const float* p, int64_t nr, const float* W, int din, int dout,
             Scratch& sc, cudaStream_t s) {
  Proj P;
  if (W) {
    float* U = sc.get<float>((size_t)nq * dout);
    float* V = sc.get<float>((size_t)nr * dout);
    launch_sgemm_nt(q, nq, W, dout, din, EpiStore{U, nq, dout, dout, 0}, 0, s);
    launch_sgemm_nt(p, nr, W, dout, din, EpiStore{V, nr, dout, dout, 0}, 0, s);
    P.U = U;
    P.V = V;
  } else {
    P.U = q;
    P.V = p;
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

// C [M, N] (+)= A^T-free NT product of row-major A [M, K] and B [N, K]
void gemm_tn_via_transpose(const float* X, int64_t rows, int64_t colsX, const float* Y, int64_t colsY,
                           float* C, int accumulate, Scratch& sc, cudaStream_t s) {
  // C[o, k] = sum_r X[r, o] Y[r, k]: transpose both so the reduction is contiguous
  const int64_t ldr = cdiv(rows, 16) * 16;
  float* Xt = sc.get<float>((size_t)colsX * ldr);
  float* Yt = sc.get<float>((size_t)colsY * ldr);
  dim3 blk(32, 8);
  k_transpose<<<dim3((unsigned)cdiv(colsX, 32), (unsigned)cdiv(ldr, 32)), blk, 0, s>>>(X, rows, colsX, Xt, ldr);
  GIFT_LAUNCHED("k_transpose");
  k_transpose<<<dim3((unsigned)cdiv(colsY, 32), (unsigned)cdiv(ldr, 32)), blk, 0, s>>>(Y, rows, colsY, Yt, ldr);
  GIFT_LAUNCHED("k_transpose");
  launch_sgemm_nt(Xt, colsX, Yt, colsY, (int)ldr, EpiStore{C, colsX, colsY, colsY, accumulate}, 0, s);
}

}  // namespace

void match_forward(const float* q, const std::vector<int32_t>& h_qoff, int32_t Bq, const float* p, int32_t Np,
                   int32_t nv, const float* W, int32_t din, int32_t dout, float* S, int16_t* argmax, Scratch& sc,
                   cudaStream_t s) {
  const int64_t nq = h_qoff[Bq];
  const int64_t nr = (int64_t)Np * nv;
  Proj P = project(q, nq, p, nr, W, din, dout, sc, s);
  int32_t* d_qoff = device_offsets(h_qoff, sc, s);
  segmax_scores(P.U, P.uinv, nq, P.V, P.vinv, Np, nv, dout, d_qoff, h_qoff, Bq, S, argmax, sc, s);
}

void match_backward(const float* q, const std::vector<int32_t>& h_qoff, int32_t Bq, const float* p, int32_t Np,
                    int32_t nv, const float* W, int32_t din, int32_t dout, const float* gS, const int16_t* argmax,
                    float* dW, float* dQ, float* dP, Scratch& sc, cudaStream_t s) {
  const int64_t nq = h_qoff[Bq];
  const int64_t nr = (int64_t)Np * nv;
  Proj P = project(q, nq, p, nr, W, din, dout, sc, s);
  int32_t* d_qoff = device_offsets(h_qoff, sc, s);
  int32_t* vquery = sc.get<int32_t>(nq);
  k_view_query<<<(unsigned)Bq, 128, 0, s>>>(d_qoff, Bq, vquery);
  GIFT_LAUNCHED("k_view_query");
  float* sv = sc.get<float>((size_t)nq * Np);
  k_pair_cos<<<(unsigned)cdiv(nq * Np * 32, 256), 256, 0, s>>>(P.U, P.uinv, P.V, P.vinv, argmax, nq, Np, nv,
                                                                dout, sv);
  GIFT_LAUNCHED("k_pair_cos");
  // gradients w.r.t. the projected views (W == NULL: these are dQ, dP)
  float* dU = (W || !dQ) ? sc.get<float>((size_t)nq * dout) : dQ;
  float* dV = (W || !dP) ? sc.get<float>((size_t)nr * dout) : dP;
  GIFT_CUDA(cudaFuncSetAttribute(k_grad_u, cudaFuncAttributeMaxDynamicSharedMemorySize, dout * 4));
  k_grad_u<<<(unsigned)nq, 256, (size_t)dout * 4, s>>>(P.U, P.uinv, P.V, P.vinv, argmax, sv, gS, vquery, d_qoff,
                                                       Np, nv, dout, dU);
  GIFT_LAUNCHED("k_grad_u");
  int dchunk = dout;
  while ((int64_t)nv * dchunk * 4 + nv * 4 > 200 * 1024 && dchunk > 32) dchunk = (dchunk + 1) / 2;
  GIFT_REQUIRE((int64_t)nv * dchunk * 4 + nv * 4 <= 200 * 1024, "views per shape too large for the backward");
  const size_t smem = (size_t)nv * dchunk * 4 + (size_t)nv * 4;
  GIFT_CUDA(cudaFuncSetAttribute(k_grad_v, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_grad_v<<<dim3((unsigned)Np, (unsigned)cdiv(dout, dchunk)), 256, smem, s>>>(
      P.U, P.uinv, P.V, P.vinv, argmax, sv, gS, vquery, d_qoff, nq, Np, nv, dout, dchunk, dV);
  GIFT_LAUNCHED("k_grad_v");
  if (W) {
    if (dW) {
      gemm_tn_via_transpose(dU, nq, dout, q, din, dW, 0, sc, s);
      gemm_tn_via_transpose(dV, nr, dout, p, din, dW, 1, sc, s);
    }
    // dQ = dU W: NT product with W^T [din, dout]
    float* Wt = sc.get<float>((size_t)din * dout);
    k_transpose<<<dim3((unsigned)cdiv(din, 32), (unsigned)cdiv(dout, 32)), dim3(32, 8), 0, s>>>(W, dout, din, Wt,
                                                                                            dout);
    GIFT_LAUNCHED("k_transpose");
    if (dQ) launch_sgemm_nt(dU, nq, Wt, din, dout, EpiStore{dQ, nq, din, din, 0}, 0, s);
    if (dP) launch_sgemm_nt(dV, nr, Wt, din, dout, EpiStore{dP, nr, din, din, 0}, 0, s);
  }
}

}  // namespace gift
