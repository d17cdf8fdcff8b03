// Quantiser c(x) = argmin_k ||x - b_k||^2 with multiple assignment (Sec. 2.3).
//
// Stage 1 (coarse): score_k = x.b_k - ||b_k||^2 / 2 for all codewords by a
// tile GEMM; argmax of the score is argmin of the distance.
// Stage 2 (refine, one warp per row): every codeword whose coarse score lies
// within twice the coarse error bound of the ma-th best coarse score is a
// candidate; candidates get their exact squared distance in two-float (~2^-44
// relative) arithmetic and the ma smallest by (distance, index) are kept. The
// bound makes the candidate set contain the true ma nearest codewords, so the
// result agrees with an exact evaluation except where distances tie to ~1e-13.
#include "gift_internal.cuh"
#include "sgemm_nt.cuh"

namespace gift {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxCand = 32;

struct EpiScores {
  float* C;  // [M, N]
  int64_t M, N;
  const float* half_sq;
  __device__ __forceinline__ void operator()(int64_t m0, int64_t n0, const SgemmFrag& f,
                                             float (&acc)[8][8]) const {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t m = m0 + f.row(i);
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t n = n0 + f.col(j);
        if (n < N) C[m * N + n] = acc[i][j] - half_sq[n];
      }
    }
  }
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// exact-ish ||x - b||^2 as a normalised two-float (hi, lo), warp cooperative
__device__ void dist_df(const float* __restrict__ x, const float* __restrict__ b, int D, int lane,
                        float& ohi, float& olo) {
  float hi = 0.f, lo = 0.f;
  for (int d = lane * 4; d < D; d += 128) {
    const float4 xv = *reinterpret_cast<const float4*>(x + d);
    const float4 bv = *reinterpret_cast<const float4*>(b + d);
    const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
    const float bs[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float s, e;
      two_sum(xs[c], -bs[c], s, e);         // x - b = s + e exactly
      const float p = s * s;
      float pe = fmaf(s, s, -p);            // s^2 = p + pe exactly
      pe = fmaf(2.f * s, e, pe);            // + 2 s e (e^2 is below 2^-48 s^2)
      float t, te;
      two_sum(hi, p, t, te);
      hi = t;
      lo += te + pe;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(kFull, hi, o);
    const float l2 = __shfl_xor_sync(kFull, lo, o);
    float t, te;
    two_sum(hi, h2, t, te);
    hi = t;
    lo = lo + l2 + te;
  }
  float t, te;
  two_sum(hi, lo, t, te);
  ohi = t;
  olo = te;
}

__device__ __forceinline__ bool df_less(float ah, float al, int ak, float bh, float bl, int bk) {
  if (ah != bh) return ah < bh;
  if (al != bl) return al < bl;
  return ak < bk;
}

// insert (h, l, k) into an ascending list of length ma (registers)
__device__ __forceinline__ void keep_best(float (&H)[GIFT_MAX_MA], float (&L)[GIFT_MAX_MA],
                                          int (&Kx)[GIFT_MAX_MA], int ma, float h, float l, int k) {
  if (!df_less(h, l, k, H[ma - 1], L[ma - 1], Kx[ma - 1])) return;
  int pos = ma - 1;
#pragma unroll
  for (int a = GIFT_MAX_MA - 1; a > 0; --a) {
    if (a <= pos && a - 1 < ma && df_less(h, l, k, H[a - 1], L[a - 1], Kx[a - 1])) {
      H[a] = H[a - 1];
      L[a] = L[a - 1];
      Kx[a] = Kx[a - 1];
      pos = a - 1;
    }
  }
  H[pos] = h;
  L[pos] = l;
  Kx[pos] = k;
}

__global__ __launch_bounds__(256) void k_assign_refine(const float* __restrict__ X, int64_t n, int D,
                                                       const float* __restrict__ scores, int K,
                                                       const float* __restrict__ cb, int ma,
                                                       float cb_max_norm, int32_t* __restrict__ codes,
                                                       int64_t row0) {
  __shared__ int cand_s[8][kMaxCand];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + w;
  if (r >= n) return;
  const float* sr = scores + r * (int64_t)K;
  const float* x = X + r * (int64_t)D;

  // ma-th best coarse score: per-lane top-ma, then ma rounds of warp max
  float top[GIFT_MAX_MA];
#pragma unroll
  for (int a = 0; a < GIFT_MAX_MA; ++a) top[a] = -INFINITY;
  for (int k = lane; k < K; k += 32) {
    float v = sr[k];
#pragma unroll
    for (int a = 0; a < GIFT_MAX_MA; ++a) {
      if (a < ma && v > top[a]) {
        const float t = top[a];
        top[a] = v;
        v = t;
      }
    }
  }
  float thr = -INFINITY;
  int head = 0;
  for (int a = 0; a < ma; ++a) {
    float mine = head < ma ? top[0] : -INFINITY;
    float m = mine;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    thr = m;
    const unsigned who = __ballot_sync(kFull, mine == m && head < ma);
    if (lane == __ffs(who) - 1) {
#pragma unroll
      for (int b = 0; b + 1 < GIFT_MAX_MA; ++b) top[b] = top[b + 1];
      top[GIFT_MAX_MA - 1] = -INFINITY;
      ++head;
    }
  }

  // coarse error bound E: recursive FMA summation of D products plus the
  // norm term; candidates lie within 2E of the ma-th best coarse score.
  float xx = 0.f;
  for (int d = lane; d < D; d += 32) xx = fmaf(x[d], x[d], xx);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) xx += __shfl_xor_sync(kFull, xx, o);
  const float xn = sqrtf(xx) * 1.0001f;
  const float u = 5.9604645e-08f;  // 2^-24
  const float gam = (float)(D + 2) * u * 1.01f;
  const float E = gam * (xn * cb_max_norm + 0.5f * cb_max_norm * cb_max_norm) + 1e-30f;
  const float lim = thr - 2.f * E;

  // collect candidates in index order
  int cnt = 0;
  bool overflow = false;
  for (int k0 = 0; k0 < K; k0 += 32) {
    const int k = k0 + lane;
    const bool c = k < K && sr[k] >= lim;
    const unsigned m = __ballot_sync(kFull, c);
    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
    if (c && pos < kMaxCand) cand_s[w][pos] = k;
    cnt += __popc(m);
  }
  __syncwarp();
  if (cnt > kMaxCand) overflow = true;

  float H[GIFT_MAX_MA], L[GIFT_MAX_MA];
  int Kx[GIFT_MAX_MA];
#pragma unroll
  for (int a = 0; a < GIFT_MAX_MA; ++a) {
    H[a] = INFINITY;
    L[a] = 0.f;
    Kx[a] = 0x7fffffff;
  }
  const int ncheck = overflow ? K : cnt;
  for (int c = 0; c < ncheck; ++c) {
    const int k = overflow ? c : cand_s[w][c];
    float h, l;
    dist_df(x, cb + (int64_t)k * D, D, lane, h, l);
    keep_best(H, L, Kx, ma, h, l, k);
  }
  if (lane < ma) {
    int out = Kx[0];
#pragma unroll
    for (int a = 1; a < GIFT_MAX_MA; ++a)
      if (a == lane) out = Kx[a];
    codes[(row0 + r) * ma + lane] = out;
  }
}

}  // namespace

void assign_codes(const Index& ix, const float* X, int64_t n, int ma, int32_t* codes, Scratch& sc,
                  cudaStream_t s) {
  if (n <= 0) return;
  const int K = ix.prm.n_codewords, D = ix.prm.dim;
  GIFT_REQUIRE(ma >= 1 && ma <= GIFT_MAX_MA && ma <= K, "multiple assignment must be in [1, min(8, K)]");
  // rows per chunk: the coarse score block stays under 1 GiB
  const int64_t chunk = std::max<int64_t>(128, std::min<int64_t>(n, ((int64_t)1 << 28) / K / 128 * 128));
  float* scores = sc.get<float>((size_t)std::min(chunk, n) * K);
  for (int64_t r0 = 0; r0 < n; r0 += chunk) {
    const int64_t m = std::min(chunk, n - r0);
    EpiScores epi{scores, m, K, ix.cb_half_sq};
    launch_sgemm_nt(X + r0 * D, m, ix.codebook, K, D, epi, 0, s);
    k_assign_refine<<<(unsigned)cdiv(m, 8), 256, 0, s>>>(X + r0 * D, m, D, scores, K, ix.codebook, ma,
                                                          ix.cb_max_norm, codes, r0);
    GIFT_LAUNCHED("k_assign_refine");
  }
}

}  // namespace gift
