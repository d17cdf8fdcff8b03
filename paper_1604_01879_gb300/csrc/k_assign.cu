// Quantiser c(x) = argmin_k ||x - b_k||^2 with multiple assignment (Sec. 2.3).
//
// Coarse stage (tensor cores): score_k = x.b_k - ||b_k||^2 / 2 (argmax of the
// score is argmin of the distance) from two-part BF16 operands (x = hi + lo,
// three products, FP32 accumulate). A work item is 128 rows x one chunk of 256
// codewords; the chunks of one row tile are consecutive items, so the CTAs
// that run them at the same time share the row tile through L2. The epilogue
// keeps each row's 16 best coarse scores of its chunk.
// Refine stage (CUDA cores, one warp per row): every codeword whose coarse
// score lies within 2E of the ma-th best over all chunks is a candidate, where
// E bounds the coarse error:
//   E = 2^-12 (||x|| max_k ||b_k|| + max_k ||b_k||^2 / 2),
// about five times the representation bound of the split (3 * 2^-16 relative
// per product) plus the measured accumulation error. When a chunk's 16th kept
// score is still a candidate, that chunk may hold more, and the row takes the
// exact pass over every codeword. A single candidate with ma = 1 is the code
// without further work; otherwise the candidates' squared distances are
// evaluated in two-float (~2^-44 relative) arithmetic; the ma smallest by
// (distance, index) are the codes. Results equal an exact evaluation except
// where distances tie to ~1e-13.
#include "gift_internal.cuh"
#include "tc_engine.cuh"

namespace gift {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kT = 16;    // coarse candidates kept per row and chunk
constexpr int TNA = 256;  // codewords per chunk (AssignPolicy::TN)

struct AssignPolicy {
  static constexpr int TN = TNA, NBUF = 2, STAGES = 2, SPLIT = 3, EB = 2;
  static constexpr int kWarpSmem = TN * 4;
  int64_t n;          // rows
  int K;
  int nch;            // codeword chunks of TN
  int nkb;
  const float* half_sq;
  float* cval;        // [n, nch, kT] best coarse scores of each chunk, descending
  int32_t* cidx;      // [n, nch, kT] their codewords (0x7fffffff: none)
  struct Item {
    int64_t r0;
    int nr;
    int c;
  };
  struct Ctx {
    float val[kT];
    int idx[kT];
  };
  __device__ __forceinline__ int64_t total() const { return cdiv(n, tc::kTM) * nch; }
  __device__ __forceinline__ Item decode(int64_t item) const {
    Item it;
    it.r0 = (item / nch) * tc::kTM;
    it.c = (int)(item % nch);
    it.nr = (int)min((int64_t)tc::kTM, n - it.r0);
    return it;
  }
  __device__ __forceinline__ int nchunks(const Item&) const { return 1; }
  __device__ __forceinline__ void chunk(const Item& it, int, int& br, int& kb0, int& kb1) const {
    br = it.c * TN;
    kb0 = 0;
    kb1 = nkb;
  }
  __device__ __forceinline__ int a_row(const Item& it) const { return (int)it.r0; }
  __device__ __forceinline__ void epi_begin(const Item&, Ctx& x, int, int, uint8_t*) const {
#pragma unroll
    for (int t = 0; t < kT; ++t) {
      x.val[t] = -INFINITY;
      x.idx[t] = 0x7fffffff;
    }
  }
  __device__ __forceinline__ void epi_chunk(const Item& it, int, uint32_t taddr, Ctx& x, int, uint8_t* ws) const {
    float* hs = reinterpret_cast<float*>(ws);
    const int lane = threadIdx.x & 31;
    const int c = it.c;
    for (int j = lane; j < TN; j += 32) {
      const int k = c * TN + j;
      hs[j] = k < K ? half_sq[k] : INFINITY;
    }
    __syncwarp();
    const int npieces = min(TN, K - c * TN + 31) >> 5;
    for (int pc = 0; pc < npieces; ++pc) {
      uint32_t r[32];
      tc::tmem_ld32(taddr + pc * 32, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float s = __uint_as_float(r[j]) - hs[pc * 32 + j];
        if (s > x.val[kT - 1]) {  // strict: an equal later index never displaces an earlier one
          x.val[kT - 1] = s;
          x.idx[kT - 1] = c * TN + pc * 32 + j;
#pragma unroll
          for (int t = kT - 1; t > 0; --t) {
            if (x.val[t] > x.val[t - 1]) {
              const float tv = x.val[t];
              x.val[t] = x.val[t - 1];
              x.val[t - 1] = tv;
              const int ti = x.idx[t];
              x.idx[t] = x.idx[t - 1];
              x.idx[t - 1] = ti;
            }
          }
        }
      }
    }
    __syncwarp();
  }
  __device__ __forceinline__ void epi_end(const Item& it, Ctx& x, int m, uint8_t*) const {
    if (m >= it.nr) return;
    const int64_t o = ((it.r0 + m) * nch + it.c) * kT;
#pragma unroll
    for (int t = 0; t < kT; ++t) {
      cval[o + t] = x.val[t];
      cidx[o + t] = x.idx[t];
    }
  }
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// exact-ish ||x - b||^2 as a normalised two-float (hi, lo), warp cooperative
__device__ void dist_df(const float* __restrict__ x, const float* __restrict__ b, int D, int lane, float& ohi,
                        float& olo) {
  float hi = 0.f, lo = 0.f;
  for (int d = lane * 4; d < D; d += 128) {
    const float4 xv = *reinterpret_cast<const float4*>(x + d);
    const float4 bv = *reinterpret_cast<const float4*>(b + d);
    const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
    const float bs[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float s, e;
      two_sum(xs[c], -bs[c], s, e);  // x - b = s + e exactly
      const float p = s * s;
      float pe = fmaf(s, s, -p);     // s^2 = p + pe exactly
      pe = fmaf(2.f * s, e, pe);     // + 2 s e (e^2 is below 2^-48 s^2)
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

// the same two-float distances for up to kBatch candidates at once: each chunk
// of the row is read once and compared with every candidate
constexpr int kBatch = 8;
__device__ void dist_df_batch(const float* __restrict__ x, const float* __restrict__ cb, const int (&kc)[kBatch],
                              int n, int D, int lane, float (&ohi)[kBatch], float (&olo)[kBatch]) {
  float hi[kBatch], lo[kBatch];
#pragma unroll
  for (int c = 0; c < kBatch; ++c) {
    hi[c] = 0.f;
    lo[c] = 0.f;
  }
  for (int d = lane * 4; d < D; d += 128) {
    const float4 xv = *reinterpret_cast<const float4*>(x + d);
    const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
    for (int c = 0; c < kBatch; ++c) {
      if (c >= n) break;
      const float4 bv = *reinterpret_cast<const float4*>(cb + (int64_t)kc[c] * D + d);
      const float bs[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float s2, e;
        two_sum(xs[q], -bs[q], s2, e);
        const float p = s2 * s2;
        float pe = fmaf(s2, s2, -p);
        pe = fmaf(2.f * s2, e, pe);
        float t, te;
        two_sum(hi[c], p, t, te);
        hi[c] = t;
        lo[c] += te + pe;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kBatch; ++c) {
    if (c >= n) break;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(kFull, hi[c], o);
      const float l2 = __shfl_xor_sync(kFull, lo[c], o);
      float t, te;
      two_sum(hi[c], h2, t, te);
      hi[c] = t;
      lo[c] = lo[c] + l2 + te;
    }
    float t, te;
    two_sum(hi[c], lo[c], t, te);
    ohi[c] = t;
    olo[c] = te;
  }
}

__device__ __forceinline__ bool df_less(float ah, float al, int ak, float bh, float bl, int bk) {
  if (ah != bh) return ah < bh;
  if (al != bl) return al < bl;
  return ak < bk;
}

// warp-wide best entry of (value desc, position asc) strictly after the key
// (pv, pp) in that order; positions index the row's nch * kT kept entries
__device__ __forceinline__ void next_best(const float* __restrict__ v, const int32_t* __restrict__ id, int tot,
                                          float pv, int pp, int lane, float& bv, int& bp) {
  bv = -INFINITY;
  bp = 0x7fffffff;
  for (int e = lane; e < tot; e += 32) {
    const float x = v[e];
    if (id[e] == 0x7fffffff) continue;
    const bool after = x < pv || (x == pv && e > pp);
    if (after && (x > bv || (x == bv && e < bp))) {
      bv = x;
      bp = e;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(kFull, bv, o);
    const int op = __shfl_xor_sync(kFull, bp, o);
    if (ov > bv || (ov == bv && op < bp)) {
      bv = ov;
      bp = op;
    }
  }
}

__global__ __launch_bounds__(256) void k_assign_refine(const float* __restrict__ X, int64_t n, int D,
                                                       const float* __restrict__ cb, int K, int ma,
                                                       const float* __restrict__ cval,
                                                       const int32_t* __restrict__ cidx, int nch,
                                                       const float* __restrict__ x_inv, float bmax,
                                                       int32_t* __restrict__ codes) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + w;
  if (r >= n) return;
  const float* x = X + r * (int64_t)D;
  const int tot = nch * kT;
  const float* v = cval + r * tot;
  const int32_t* id = cidx + r * tot;
  // the ma-th best coarse score over all chunks
  float thr = INFINITY;
  int tp = -1, found = 0;
  for (int a = 0; a < ma; ++a) {
    float bv;
    int bp;
    next_best(v, id, tot, thr, tp, lane, bv, bp);
    if (bp == 0x7fffffff) break;
    thr = bv;
    tp = bp;
    ++found;
  }
  const float xi = x_inv[r];
  const float xn = xi > 0.f ? 1.0001f / xi : 0.f;
  const float E = 2.44140625e-4f * (xn * bmax + 0.5f * bmax * bmax) + 1e-30f;
  const float lim = thr - 2.f * E;
  // a chunk whose last kept score is a candidate may hold more candidates
  bool full = xi == 0.f || found < ma;  // (fewer kept scores than ma only with non-finite inputs)
  for (int c = lane; c < nch; c += 32) {
    const int e = c * kT + kT - 1;
    if (id[e] != 0x7fffffff && v[e] >= lim && min(TNA, K - c * TNA) > kT) full = true;
  }
  full = __any_sync(kFull, full);
  if (!full && ma == 1) {
    // a single candidate is the nearest codeword: the true nearest always lies in
    // the window, and so would any codeword at an equal true distance
    int cnt = 0, only = 0x7fffffff;
    for (int base = 0; base < tot; base += 32) {
      const int e = base + lane;
      const int kk = e < tot ? id[e] : 0x7fffffff;
      const bool take = e < tot && kk != 0x7fffffff && v[e] >= lim;
      const unsigned m = __ballot_sync(kFull, take);
      if (m && cnt == 0) only = __shfl_sync(kFull, kk, __ffs(m) - 1);
      cnt += __popc(m);
    }
    if (cnt == 1) {
      if (lane == 0) codes[r] = only;
      return;
    }
  }
  float H[GIFT_MAX_MA], Lo[GIFT_MAX_MA];
  int Kx[GIFT_MAX_MA];
#pragma unroll
  for (int a = 0; a < GIFT_MAX_MA; ++a) {
    H[a] = INFINITY;
    Lo[a] = 0.f;
    Kx[a] = 0x7fffffff;
  }
  auto insert = [&](float h, float l, int k) {  // into the ascending list of the ma best (registers, unrolled)
    if (df_less(h, l, k, H[GIFT_MAX_MA - 1], Lo[GIFT_MAX_MA - 1], Kx[GIFT_MAX_MA - 1])) {
      H[GIFT_MAX_MA - 1] = h;
      Lo[GIFT_MAX_MA - 1] = l;
      Kx[GIFT_MAX_MA - 1] = k;
#pragma unroll
      for (int t = GIFT_MAX_MA - 1; t > 0; --t) {
        if (df_less(H[t], Lo[t], Kx[t], H[t - 1], Lo[t - 1], Kx[t - 1])) {
          const float th = H[t], tl = Lo[t];
          const int tk = Kx[t];
          H[t] = H[t - 1];
          Lo[t] = Lo[t - 1];
          Kx[t] = Kx[t - 1];
          H[t - 1] = th;
          Lo[t - 1] = tl;
          Kx[t - 1] = tk;
        }
      }
    }
  };
  bool batched = false;
  if (!full) {
    // up to kBatch candidates: one pass over the row for all of them
    int kc[kBatch];
    int n = 0;
#pragma unroll
    for (int c = 0; c < kBatch; ++c) kc[c] = 0;
    for (int base = 0; base < tot; base += 32) {
      const int e = base + lane;
      const int kk = e < tot ? id[e] : 0x7fffffff;
      unsigned m = __ballot_sync(kFull, e < tot && kk != 0x7fffffff && v[e] >= lim);
      while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        const int k = __shfl_sync(kFull, kk, j);
#pragma unroll
        for (int c = 0; c < kBatch; ++c)
          if (c == n) kc[c] = k;
        ++n;
      }
    }
    if (n <= kBatch) {
      float hh[kBatch], ll[kBatch];
      dist_df_batch(x, cb, kc, n, D, lane, hh, ll);
#pragma unroll
      for (int c = 0; c < kBatch; ++c)
        if (c < n) insert(hh[c], ll[c], kc[c]);
      batched = true;
    }
  }
  const int nscan = batched ? 0 : full ? K : tot;
  for (int base = 0; base < nscan; base += 32) {
    const int e = base + lane;
    bool take;
    int kk;
    if (full) {
      take = e < K;
      kk = e;
    } else {
      kk = e < tot ? id[e] : 0x7fffffff;
      take = e < tot && kk != 0x7fffffff && v[e] >= lim;
    }
    unsigned mask = __ballot_sync(kFull, take);
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      const int k = __shfl_sync(kFull, kk, j);
      float h, l;
      dist_df(x, cb + (int64_t)k * D, D, lane, h, l);
      insert(h, l, k);
    }
  }
  if (lane < ma) {
    int out = Kx[0];
#pragma unroll
    for (int a = 1; a < GIFT_MAX_MA; ++a)
      if (a == lane) out = Kx[a];
    codes[r * ma + lane] = out;
  }
}

// hi = bf16(x), lo = bf16(x - hi), row-major [n, D]
__global__ void k_split_rows(const float* __restrict__ X, int64_t n, int D, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // index of a float4
  if (i >= n * (D / 4)) return;
  const float4 v = reinterpret_cast<const float4*>(X)[i];
  const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
  const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
  reinterpret_cast<__nv_bfloat162*>(hi)[2 * i] = a;
  reinterpret_cast<__nv_bfloat162*>(hi)[2 * i + 1] = b;
  const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  reinterpret_cast<__nv_bfloat162*>(lo)[2 * i] = __floats2bfloat162_rn(v.x - fa.x, v.y - fa.y);
  reinterpret_cast<__nv_bfloat162*>(lo)[2 * i + 1] = __floats2bfloat162_rn(v.z - fb.x, v.w - fb.y);
}

}  // namespace

void split_rows_bf16(const float* X, int64_t n, int D, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t n4 = n * (D / 4);
  k_split_rows<<<(unsigned)cdiv(n4, 256), 256, 0, s>>>(X, n, D, hi, lo);
  GIFT_LAUNCHED("k_split_rows");
}

void assign_codes(const Index& ix, const float* X, int64_t n, int ma, int32_t* codes, Scratch& sc, cudaStream_t s,
                  const float* x_inv, KernelClock* kc) {
  if (n <= 0) return;
  const int K = ix.prm.n_codewords, D = ix.prm.dim;
  GIFT_REQUIRE(ma >= 1 && ma <= GIFT_MAX_MA && ma <= K, "multiple assignment must be in [1, min(8, K)]");
  const int64_t chunk = std::min<int64_t>(n, 131072);
  const int64_t rows_alloc = chunk + tc::kTM;  // one box of padding rows
  __nv_bfloat16* hi = sc.get<__nv_bfloat16>((size_t)rows_alloc * D);
  __nv_bfloat16* lo = sc.get<__nv_bfloat16>((size_t)rows_alloc * D);
  const int nch = (int)cdiv(K, TNA);
  float* cval = sc.get<float>((size_t)chunk * nch * kT);
  int32_t* cidx = sc.get<int32_t>((size_t)chunk * nch * kT);
  float* inv = nullptr;
  if (!x_inv) {
    inv = sc.get<float>(n);
    launch_row_invnorm(X, n, D, inv, s);
    x_inv = inv;
  }
  const CUtensorMap tB = make_tmap_bf16(ix.cb_hi, ix.cb_rows_alloc, D, AssignPolicy::TN);
  const CUtensorMap tB2 = make_tmap_bf16(ix.cb_lo, ix.cb_rows_alloc, D, AssignPolicy::TN);
  const int sms = device_sm_count();
  for (int64_t r0 = 0; r0 < n; r0 += chunk) {
    const int64_t m = std::min(chunk, n - r0);
    split_rows_bf16(X + r0 * D, m, D, hi, lo, s);
    AssignPolicy p;
    p.n = m;
    p.K = K;
    p.nch = nch;
    p.nkb = (int)cdiv(D, tc::kTK);
    p.half_sq = ix.cb_half_sq;
    p.cval = cval;
    p.cidx = cidx;
    const CUtensorMap tA = make_tmap_bf16(hi, rows_alloc, D, tc::kTM);
    const CUtensorMap tA2 = make_tmap_bf16(lo, rows_alloc, D, tc::kTM);
    const int grid = (int)std::min<int64_t>(sms, cdiv(m, tc::kTM) * nch);
    if (kc) kc->begin(0);
    tc::launch_engine(tA, tB, tA2, tB2, p, ix.d_err, grid, s);
    if (kc) {
      kc->end(0);
      kc->assign_rows += m;
    }
    k_assign_refine<<<(unsigned)cdiv(m, 8), 256, 0, s>>>(X + r0 * D, m, D, ix.codebook, K, ma, cval, cidx, nch,
                                                          x_inv + r0, ix.cb_max_norm, codes + r0 * ma);
    GIFT_LAUNCHED("k_assign_refine");
  }
}

}  // namespace gift
