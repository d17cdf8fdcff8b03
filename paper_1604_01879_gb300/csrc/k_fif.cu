// Approximate multi-view matching through the first inverted file (Eq. 4).
//
//  bucket  : query views (with their query_ma codewords) are grouped by
//            codeword with a stable counting sort: a "slot" is one
//            (query view, assigned codeword) pair, slots of codeword k are
//            contiguous (M_k of them).
//  scan    : for every list k touched by the batch, the L_k list entries are
//            multiplied with the M_k slots of bucket k (a grouped contraction);
//            cosines are reduced by max over each run of equal shape id inside
//            the list and folded into a per-(slot, run) table with atomicMax
//            on an order-preserving key of the float (f2key; 0 = no value).
//  combine : per query, per view, the max over its query_ma slots of each
//            shape's run value, summed over the views in signed 64-bit fixed
//            point (exact, order-free) and divided by |V(x_q)| -> S(x_q, .)
//            (Eq. 4, normaliser of Eq. 3). Eq. 4's max runs over every view
//            of the shape, so 0 joins it whenever some view of the shape
//            shares no codeword with the query view: a negative maximum
//            counts only when every view of the shape is matched (checked
//            from the database codes; never needed for non-negative features).
//  rescore : the same scan over the FP32 feature master for the top-R
//            candidate shapes only, combined into FP32 candidate scores.
#include <algorithm>

#include "gift_internal.cuh"
#include "fif_plan.cuh"

namespace gift {

namespace {

constexpr int kCombineT = 256;

__global__ void k_slot_setup(const int32_t* __restrict__ perm, int64_t nslots, int ma,
                             const int32_t* __restrict__ skeys, const int32_t* __restrict__ nruns,
                             int32_t* __restrict__ slot_view, int32_t* __restrict__ view_slot,
                             int64_t* __restrict__ run_cnt) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s == nslots) run_cnt[s] = 0;  // so that the scan's last element is the table size
  if (s >= nslots) return;
  const int32_t item = perm[s];
  slot_view[s] = item / ma;
  view_slot[item] = (int32_t)s;
  run_cnt[s] = nruns[skeys[s]];
}

// work items of list k: ceil(L_k / TE) entry tiles x ceil(M_k / TS) slot chunks
__global__ void k_work_count(const int64_t* __restrict__ boff, const int64_t* __restrict__ list_off,
                             int K, int64_t* __restrict__ wcnt, int64_t row_bytes,
                             int64_t rescore_row_bytes, unsigned long long* __restrict__ stats) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > K) return;
  if (k == K) {
    wcnt[K] = 0;
    return;
  }
  const int64_t M = boff[k + 1] - boff[k];
  const int64_t L = list_off[k + 1] - list_off[k];
  wcnt[k] = (M > 0 && L > 0) ? cdiv(L, kScanTE) * cdiv(M, kScanTS) : 0;
  if (stats && M > 0 && L > 0) {
    atomicAdd(&stats[0], (unsigned long long)(L * row_bytes));
    atomicAdd(&stats[1], (unsigned long long)(L * M));
    atomicAdd(&stats[2], (unsigned long long)(L * rescore_row_bytes));
  }
}

template <typename TF>
struct Load4;
template <>
struct Load4<float> {
  static __device__ __forceinline__ float4 get(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
  }
};
template <>
struct Load4<__nv_bfloat16> {
  static __device__ __forceinline__ float4 get(const __nv_bfloat16* p) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
};
template <>
struct Load4<__nv_fp8_e4m3> {
  static __device__ __forceinline__ float4 get(const __nv_fp8_e4m3* p) {
    const uint32_t u = __ldg(reinterpret_cast<const unsigned int*>(p));
    __nv_fp8x4_e4m3 v;
    v.__x = u;
    return static_cast<float4>(v);
  }
};

// binary search of `key` in sorted a[0..n); -1 if absent
__device__ __forceinline__ int find_sorted(const int32_t* a, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < n && a[lo] == key) ? lo : -1;
}
__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

struct ScanArgs {
  const int64_t* woff;     // [K+1] work-item offsets; woff[K] = total
  int K;
  const int64_t* boff;     // [K+1] slot offsets per codeword
  const int64_t* list_off; // [K+1]
  const int32_t* slot_view;
  const int64_t* runbase;
  const int32_t* vquery;
  const float* q;
  const float* q_inv;
  int D;
  const void* feat;        // list-ordered store (scan) or FP32 master (rescore)
  const float* scale;      // list_scale (scan) or row_inv (rescore)
  const int32_t* list_row;
  const int32_t* list_shape;
  const int32_t* entry_run;
  uint32_t* table;
  const int32_t* cand;     // [B, R] candidate ids sorted ascending (rescore)
  int R;
};

template <typename TF, bool RESCORE>
__global__ __launch_bounds__(256) void k_fif_scan(const ScanArgs a) {
  __shared__ __align__(16) float Qs[2][16][kScanTS];
  __shared__ __align__(16) float Fs[2][16][kScanTE];
  __shared__ float Ts[kScanTS][kScanTE + 1];
  __shared__ int32_t e_run[kScanTE], e_shape[kScanTE];
  __shared__ float e_scale[kScanTE];
  __shared__ const TF* e_ptr[kScanTE];
  __shared__ int32_t s_view[kScanTS], s_q[kScanTS];
  __shared__ float s_inv[kScanTS];
  __shared__ int64_t s_rb[kScanTS];
  __shared__ int64_t sh[4];

  const int tid = threadIdx.x;
  const int64_t item = blockIdx.x;
  if (item >= a.woff[a.K]) return;
  if (tid == 0) {
    int lo = 0, hi = a.K;  // largest k with woff[k] <= item
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.woff[mid] <= item) lo = mid; else hi = mid;
    }
    const int k = lo;
    const int64_t local = item - a.woff[k];
    const int64_t M = a.boff[k + 1] - a.boff[k];
    const int64_t chunks = cdiv(M, kScanTS);
    const int64_t tile = local / chunks, chunk = local % chunks;
    const int64_t e0 = a.list_off[k] + tile * kScanTE;
    const int64_t s0 = a.boff[k] + chunk * kScanTS;
    sh[0] = e0;
    sh[1] = std::min<int64_t>(kScanTE, a.list_off[k + 1] - e0);
    sh[2] = s0;
    sh[3] = std::min<int64_t>(kScanTS, a.boff[k + 1] - s0);
  }
  __syncthreads();
  const int64_t e0 = sh[0], s0 = sh[2];
  const int ne = (int)sh[1], ns = (int)sh[3];
  const int D = a.D;
  if (tid < kScanTE) {
    if (tid < ne) {
      const int64_t e = e0 + tid;
      e_run[tid] = a.entry_run[e];
      e_shape[tid] = a.list_shape[e];
      if (RESCORE) {
        const int32_t row = a.list_row[e];
        e_scale[tid] = a.scale[row];
        e_ptr[tid] = reinterpret_cast<const TF*>(a.feat) + (int64_t)row * D;
      } else {
        e_scale[tid] = a.scale[e];
        e_ptr[tid] = reinterpret_cast<const TF*>(a.feat) + e * D;
      }
    } else {
      e_run[tid] = -1;
      e_ptr[tid] = nullptr;
    }
  } else if (tid < kScanTE + kScanTS) {
    const int sl = tid - kScanTE;
    if (sl < ns) {
      const int32_t v = a.slot_view[s0 + sl];
      s_view[sl] = v;
      s_q[sl] = a.vquery[v];
      s_inv[sl] = a.q_inv[v];
      s_rb[sl] = a.runbase[s0 + sl];
    } else {
      s_view[sl] = -1;
    }
  }
  __syncthreads();

  const int lrow = tid >> 2, lk = (tid & 3) * 4;
  const float* qrow = (lrow < ns) ? a.q + (int64_t)s_view[lrow] * D : nullptr;
  const TF* frow = (lrow < ne) ? e_ptr[lrow] : nullptr;
  float4 rq = make_float4(0.f, 0.f, 0.f, 0.f), rf = rq;
  const float4 z4 = rq;
  auto gload = [&](int k0) {
    rq = qrow ? __ldg(reinterpret_cast<const float4*>(qrow + k0 + lk)) : z4;
    rf = frow ? Load4<TF>::get(frow + k0 + lk) : z4;
  };
  auto sstore = [&](int b) {
    Qs[b][lk + 0][lrow] = rq.x;
    Qs[b][lk + 1][lrow] = rq.y;
    Qs[b][lk + 2][lrow] = rq.z;
    Qs[b][lk + 3][lrow] = rq.w;
    Fs[b][lk + 0][lrow] = rf.x;
    Fs[b][lk + 1][lrow] = rf.y;
    Fs[b][lk + 2][lrow] = rf.z;
    Fs[b][lk + 3][lrow] = rf.w;
  };

  const int tx = tid & 15, ty = tid >> 4;  // entries tx*4.., slots ty*4..
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  gload(0);
  sstore(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < D; k0 += 16) {
    const bool more = k0 + 16 < D;
    if (more) gload(k0 + 16);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float4 qa = *reinterpret_cast<const float4*>(&Qs[buf][kk][ty * 4]);
      const float4 fb = *reinterpret_cast<const float4*>(&Fs[buf][kk][tx * 4]);
      const float qv[4] = {qa.x, qa.y, qa.z, qa.w};
      const float fv[4] = {fb.x, fb.y, fb.z, fb.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(qv[i], fv[j], acc[i][j]);
    }
    if (more) {
      sstore(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int sl = ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int el = tx * 4 + j;
      float v = 0.f;
      if (sl < ns && el < ne) v = acc[i][j] * s_inv[sl] * e_scale[el];
      Ts[sl][el] = v;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < kScanTS * kScanTE; idx += 256) {
    const int sl = idx / kScanTE, el = idx % kScanTE;
    if (sl >= ns || el >= ne) continue;
    const int run = e_run[el];
    if (el > 0 && e_run[el - 1] == run) continue;  // not the first entry of its run here
    float m = Ts[sl][el];
    for (int e2 = el + 1; e2 < ne && e_run[e2] == run; ++e2) m = fmaxf(m, Ts[sl][e2]);
    if (RESCORE) {
      if (find_sorted(a.cand + (int64_t)s_q[sl] * a.R, a.R, e_shape[el]) < 0) continue;
    }
    atomicMax(a.table + s_rb[sl] + run, f2key(m));
  }
}

struct CombineArgs {
  const int32_t* qoff;       // [B+1] device
  int ma;
  const int32_t* q_code;     // [nv*ma] codewords of each query view
  const int32_t* db_codes;   // [N*Nv*db_ma] codewords of each database view
  int db_ma, Nv;
  const int32_t* view_slot;  // [nv*ma]
  const int32_t* skeys;      // [nslots] codeword of each slot
  const int64_t* runbase;    // [nslots]
  const int32_t* nruns;      // [K]
  const int64_t* run_off;    // [K]
  const int32_t* run_shape;  // [n_runs]
  const uint32_t* table;
  int N;
  float* S;                  // [B, N] dense (not CAND)
  const int32_t* cand;       // [B, R] sorted ids (CAND)
  int R;
  float* cand_score;         // [B, R] (CAND)
  const int32_t* vquery;     // [nv] query of each view
  unsigned long long* acc;   // [B, N] (dense) or [B, R] (candidates, ma > 1) fixed-point sums, zeroed
  int64_t nv;
  int groups;                // blocks per query of k_fif_combine_ma_cand
};

// a shape's term in signed 2^-32 fixed point; two's complement sums in uint64
// are exact and order-free for |sum| < 2^31
__device__ __forceinline__ unsigned long long fix32(float f) {
  return (unsigned long long)__float2ll_rn(f * 4294967296.0f);
}
__device__ __forceinline__ float unfix32(unsigned long long acc, float Vq) {
  return __fdiv_rn(__ll2float_rn((long long)acc) * 2.3283064365386963e-10f, Vq);
}

// Eq. 4's delta is 1 for every view of shape p: each of p's views shares a
// codeword with query view v (the max then has no 0 candidate)
__device__ __noinline__ bool all_views_matched(const CombineArgs& a, int64_t v, int32_t p) {
  const int32_t* qc = a.q_code + v * a.ma;
  const int32_t* dc = a.db_codes + (int64_t)p * a.Nv * a.db_ma;
  for (int j = 0; j < a.Nv; ++j) {
    bool hit = false;
    for (int t = 0; t < a.db_ma; ++t)
      for (int u = 0; u < a.ma; ++u) hit |= dc[j * a.db_ma + t] == qc[u];
    if (!hit) return false;
  }
  return true;
}

// term of (view v, shape p) from its table key (0 = shape not reached): the
// run maximum, or nothing (Eq. 4's 0) when it is negative and a view of p is
// outside v's lists
__device__ __forceinline__ bool view_term(const CombineArgs& a, int64_t v, int32_t p, uint32_t key, float& t) {
  if (key == 0u) return false;
  t = key2f(key);
  return !(t < 0.f) || all_views_matched(a, v, p);
}

// Dense shape scores: one warp per (query view, assignment) walks the runs of
// that list and adds each shape's term into the query's row of fixed-point
// sums (global atomics; the runs of one list are distinct shapes). A shape
// reached through several of the view's lists counts once, with the largest
// maximum, added by the lowest assignment that reaches it.
__global__ __launch_bounds__(kCombineT) void k_fif_combine_views(const CombineArgs a) {
  const int64_t item = ((int64_t)blockIdx.x * kCombineT + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= a.nv * a.ma) return;
  const int64_t v = item / a.ma;
  const int s_a = (int)(item % a.ma);
  const int32_t s = a.view_slot[item];
  const int k = a.skeys[s];
  const int32_t* rs = a.run_shape + a.run_off[k];
  const int nr = a.nruns[k];
  const int64_t rb = a.runbase[s];
  unsigned long long* row = a.acc + (int64_t)a.vquery[v] * a.N;
  for (int r = lane; r < nr; r += 32) {
    const int32_t p = rs[r];
    uint32_t m = a.table[rb + r];
    bool skip = false;
    for (int s_b = 0; s_b < a.ma && !skip; ++s_b) {
      if (s_b == s_a) continue;
      const int32_t s2 = a.view_slot[v * a.ma + s_b];
      const int k2 = a.skeys[s2];
      const int r2 = find_sorted(a.run_shape + a.run_off[k2], a.nruns[k2], p);
      if (r2 < 0) continue;
      if (s_b < s_a) skip = true;  // the lower assignment owns this shape
      else m = max(m, a.table[a.runbase[s2] + r2]);
    }
    float t;
    if (skip || !view_term(a, v, p, m, t)) continue;
    atomicAdd(row + p, fix32(t));
  }
}

// fixed-point sums -> scores (1/|V(x_q)|) sum (Eq. 4), n = row width
__global__ void k_unfix_rows(const unsigned long long* __restrict__ acc, const int32_t* __restrict__ qoff, int B,
                             int64_t n, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * n) return;
  const int q = (int)(i / n);
  out[i] = unfix32(acc[i], (float)(qoff[q + 1] - qoff[q]));
}

// Candidate scores (ma = 1): one block per query, its warps over the query's
// views; a run's term is added at its shape's position among the query's
// sorted candidates (shared fixed-point sums).
__global__ __launch_bounds__(kCombineT) void k_fif_combine_cand(const CombineArgs a) {
  extern __shared__ unsigned long long acc[];
  const int q = blockIdx.x;
  for (int i = threadIdx.x; i < a.R; i += kCombineT) acc[i] = 0ull;
  __syncthreads();
  const int v0 = a.qoff[q], v1 = a.qoff[q + 1];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t* cand = a.cand + (int64_t)q * a.R;
  for (int v = v0 + w; v < v1; v += kCombineT / 32) {
    const int32_t s = a.view_slot[v];
    const int k = a.skeys[s];
    const int32_t* rs = a.run_shape + a.run_off[k];
    const int nr = a.nruns[k];
    const int64_t rb = a.runbase[s];
    for (int r = lane; r < nr; r += 32) {
      const int32_t p = rs[r];
      float t;
      if (!view_term(a, v, p, a.table[rb + r], t)) continue;
      const int idx = find_sorted(cand, a.R, p);
      if (idx >= 0) atomicAdd(&acc[idx], fix32(t));
    }
  }
  __syncthreads();
  const float Vq = (float)(v1 - v0);
  for (int i = threadIdx.x; i < a.R; i += kCombineT) a.cand_score[(int64_t)q * a.R + i] = unfix32(acc[i], Vq);
}

// Candidate scores with multiple assignment (ma > 1): each warp takes one view
// at a time; the runs of the view's ma lists fold their maxima into the warp's
// shared array over the query's candidates (atomicMax on the keys), so a
// shape reached through several lists counts once with the largest maximum;
// the array is then added into the block's fixed-point sums and cleared. Each
// list's runs are merged against a shared copy of the query's sorted candidates
// (the dense sums keep k_fif_combine, whose warps look the other lists up
// directly).
constexpr int kCombineWarps = kCombineT / 32;
__global__ __launch_bounds__(kCombineT) void k_fif_combine_ma_cand(const CombineArgs a) {
  extern __shared__ unsigned long long acc[];  // [R] sums, then int32 cand[R], then uint32 [warps][R] view maxima
  const int q = blockIdx.x / a.groups, g = blockIdx.x % a.groups, R = a.R;
  int32_t* cs = reinterpret_cast<int32_t*>(acc + R);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* vmax = reinterpret_cast<uint32_t*>(cs + R) + (size_t)w * R;
  for (int i = threadIdx.x; i < R; i += kCombineT) {
    acc[i] = 0ull;
    cs[i] = a.cand[(int64_t)q * R + i];
  }
  for (int i = lane; i < R; i += 32) vmax[i] = 0u;
  __syncthreads();
  const int v0 = a.qoff[q], v1 = a.qoff[q + 1];
  for (int v = v0 + g * kCombineWarps + w; v < v1; v += a.groups * kCombineWarps) {
    // lane t < ma: the list of assignment t
    int64_t off = 0, rb = 0;
    int n = 0;
    if (lane < a.ma) {
      const int32_t sl = a.view_slot[(int64_t)v * a.ma + lane];
      const int k = a.skeys[sl];
      off = a.run_off[k];
      rb = a.runbase[sl];
      n = a.nruns[k];
    }
    for (int t = 0; t < a.ma; ++t) {
      const int64_t o = __shfl_sync(0xffffffffu, off, t);
      const int64_t b = __shfl_sync(0xffffffffu, rb, t);
      const int nt = __shfl_sync(0xffffffffu, n, t);
      // runs (strictly ascending shape ids) and candidates (ascending) are merged:
      // each lane walks a contiguous segment of the runs with a cursor into the
      // candidates, and reads the table only for candidate shapes
      const int seg = (nt + 31) >> 5;
      const int r0 = min(nt, lane * seg), r1 = min(nt, r0 + seg);
      if (r0 < r1) {
        // run shapes are strictly ascending within a list (entries are in
        // (shape, view) order and a run is a maximal group of one shape)
        int c = lower_bound_i32(cs, R, a.run_shape[o + r0]);
        for (int r = r0; r < r1 && c < R; ++r) {
          const int32_t p = a.run_shape[o + r];
          while (c < R && cs[c] < p) ++c;
          if (c < R && cs[c] == p) {
            const uint32_t m = a.table[b + r];
            if (m != 0u) atomicMax(&vmax[c], m);  // key 0: run not written
          }
        }
      }
    }
    __syncwarp();
    for (int i = lane; i < R; i += 32) {
      const uint32_t m = vmax[i];
      if (m != 0u) {
        float t;
        if (view_term(a, v, cs[i], m, t)) atomicAdd(&acc[i], fix32(t));
        vmax[i] = 0u;
      }
    }
    __syncwarp();
  }
  __syncthreads();
  // this block's views' part of the sums (the query's groups add up in a.acc)
  for (int i = threadIdx.x; i < R; i += kCombineT)
    if (acc[i] != 0ull) atomicAdd(a.acc + (int64_t)q * R + i, acc[i]);
}

// zero the first *n cells (n read on the device)
__global__ void k_zero_cells(uint32_t* __restrict__ t, const int64_t* __restrict__ n_dev) {
  const int64_t n = *n_dev;
  const int64_t n4 = n >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint4* t4 = reinterpret_cast<uint4*>(t);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
    t4[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) t[i] = 0u;
}

}  // namespace

void fif_zero_table(const FifPlan& P, uint32_t* table, cudaStream_t s) {
  if (P.nslots <= 0) return;
  k_zero_cells<<<1216, 256, 0, s>>>(table, P.runbase + P.nslots);  // 8 blocks per SM of a GB300
  GIFT_LAUNCHED("k_zero_cells");
}

void fif_plan(const Index& ix, FifPlan& P, Scratch& sc, cudaStream_t s) {
  const int K = ix.prm.n_codewords;
  P.nslots = P.nv * P.ma;
  const int64_t n = P.nslots;
  P.skeys = sc.get<int32_t>(n);
  int32_t* perm = sc.get<int32_t>(n);
  stable_sort_by_key(P.q_code, n, K, perm, P.skeys, sc, s);
  P.boff = sc.get<int64_t>(K + 1);
  bin_offsets(P.skeys, n, K, P.boff, s);
  P.slot_view = sc.get<int32_t>(n);
  P.view_slot = sc.get<int32_t>(n);
  int64_t* run_cnt = sc.get<int64_t>(n + 1);
  k_slot_setup<<<(unsigned)cdiv(n + 1, 256), 256, 0, s>>>(perm, n, P.ma, P.skeys, ix.nruns, P.slot_view,
                                                            P.view_slot, run_cnt);
  GIFT_LAUNCHED("k_slot_setup");
  P.runbase = sc.get<int64_t>(n + 1);
  scan_exclusive_i64(run_cnt, P.runbase, n + 1, sc, s);  // runbase[n] = table cells in use
  P.table_upper = n * (int64_t)std::max(1, ix.max_runs);
  int64_t* wcnt = sc.get<int64_t>(K + 1);
  P.woff = sc.get<int64_t>(K + 1);
  const int64_t row_bytes = (int64_t)ix.prm.dim * (int64_t)dtype_bytes(ix.prm.storage) + 12;
  const int64_t rescore_row_bytes = (int64_t)ix.prm.dim * 4 + 12;
  k_work_count<<<(unsigned)cdiv(K + 1, 256), 256, 0, s>>>(P.boff, ix.list_off, K, wcnt, row_bytes,
                                                            rescore_row_bytes, P.stats);
  GIFT_LAUNCHED("k_work_count");
  scan_exclusive_i64(wcnt, P.woff, K + 1, sc, s);
  const int64_t max_tiles = cdiv(std::max(1, ix.max_list), kScanTE);
  P.upper_items = ix.scan_tiles_upper + max_tiles * (cdiv(n, kScanTS) + 1);
}

void fif_scan(const Index& ix, const FifPlan& P, uint32_t* table, bool rescore,
              const int32_t* cand_sorted, int R, cudaStream_t s) {
  if (P.upper_items <= 0) return;
  ScanArgs a;
  a.woff = P.woff;
  a.K = ix.prm.n_codewords;
  a.boff = P.boff;
  a.list_off = ix.list_off;
  a.slot_view = P.slot_view;
  a.runbase = P.runbase;
  a.vquery = P.vquery;
  a.q = P.q;
  a.q_inv = P.q_inv;
  a.D = ix.prm.dim;
  a.list_row = ix.list_row;
  a.list_shape = ix.list_shape;
  a.entry_run = ix.entry_run;
  a.table = table;
  a.cand = cand_sorted;
  a.R = R;
  const unsigned grid = (unsigned)P.upper_items;
  if (rescore) {
    a.feat = ix.master;
    a.scale = ix.row_inv;
    k_fif_scan<float, true><<<grid, 256, 0, s>>>(a);
  } else {
    a.feat = ix.list_feat;
    a.scale = ix.list_scale;
    switch (ix.prm.storage) {
      case GIFT_F32: k_fif_scan<float, false><<<grid, 256, 0, s>>>(a); break;
      case GIFT_BF16: k_fif_scan<__nv_bfloat16, false><<<grid, 256, 0, s>>>(a); break;
      default: k_fif_scan<__nv_fp8_e4m3, false><<<grid, 256, 0, s>>>(a); break;
    }
  }
  GIFT_LAUNCHED("k_fif_scan");
}

void fif_combine(const Index& ix, const FifPlan& P, const uint32_t* table, float* S_dense,
                 const int32_t* cand_sorted, int R, float* cand_score, Scratch& sc, cudaStream_t s) {
  CombineArgs a;
  a.qoff = P.qoff;
  a.ma = P.ma;
  a.q_code = P.q_code;
  a.db_codes = ix.db_codes;
  a.db_ma = ix.db_ma;
  a.Nv = ix.prm.views_per_shape;
  a.view_slot = P.view_slot;
  a.skeys = P.skeys;
  a.runbase = P.runbase;
  a.nruns = ix.nruns;
  a.run_off = ix.run_off;
  a.run_shape = ix.run_shape;
  a.table = table;
  a.N = ix.prm.n_shapes;
  a.S = S_dense;
  a.cand = cand_sorted;
  a.R = R;
  a.cand_score = cand_score;
  a.vquery = P.vquery;
  a.nv = P.nv;
  a.acc = nullptr;
  a.groups = 1;
  if (P.B <= 0) return;
  if (P.ma > 1 && cand_sorted) {
    GIFT_REQUIRE(R <= 1024, "rescore depth must be <= 1024");
    // a query's views spread over several blocks (about one view per warp), so
    // that a batch of a few hundred queries fills every SM
    const int64_t per_query = cdiv(P.nv, (int64_t)P.B);
    a.groups = (int)std::min<int64_t>(16, std::max<int64_t>(1, cdiv(per_query, (int64_t)kCombineWarps)));
    a.acc = sc.get<unsigned long long>((size_t)P.B * R);
    GIFT_CUDA(cudaMemsetAsync(a.acc, 0, (size_t)P.B * R * 8, s));
    const size_t smem = (size_t)R * (8 + 4 + 4 * kCombineWarps);
    GIFT_CUDA(cudaFuncSetAttribute(k_fif_combine_ma_cand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_fif_combine_ma_cand<<<(unsigned)(P.B * a.groups), kCombineT, smem, s>>>(a);
    GIFT_LAUNCHED("k_fif_combine_ma_cand");
    k_unfix_rows<<<(unsigned)cdiv((int64_t)P.B * R, 256), 256, 0, s>>>(a.acc, P.qoff, P.B, R, cand_score);
    GIFT_LAUNCHED("k_unfix_rows");
    return;
  }
  if (cand_sorted) {
    GIFT_REQUIRE(R <= 1024, "rescore depth must be <= 1024");
    k_fif_combine_cand<<<(unsigned)P.B, kCombineT, (size_t)R * 8, s>>>(a);
    GIFT_LAUNCHED("k_fif_combine_cand");
    return;
  }
  const int64_t n = (int64_t)P.B * a.N;
  a.acc = sc.get<unsigned long long>((size_t)n);
  GIFT_CUDA(cudaMemsetAsync(a.acc, 0, (size_t)n * 8, s));
  const int64_t warps = P.nv * P.ma;
  if (warps > 0) {
    k_fif_combine_views<<<(unsigned)cdiv(warps * 32, (int64_t)kCombineT), kCombineT, 0, s>>>(a);
    GIFT_LAUNCHED("k_fif_combine_views");
  }
  k_unfix_rows<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(a.acc, P.qoff, P.B, a.N, S_dense);
  GIFT_LAUNCHED("k_unfix_rows");
}

}  // namespace gift
