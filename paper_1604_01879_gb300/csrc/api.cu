// C ABI of the GIFT library: index build, queries, re-ranking, exports.
#include <cstdio>
#include <cstring>
#include <atomic>
#include <functional>
#include <memory>

#include "fif_plan.cuh"
#include "gift_internal.cuh"

namespace gift {

namespace {
thread_local std::string g_last_error;

enum Stage { ST_ASSIGN = 0, ST_BUCKET, ST_SCAN, ST_COMBINE, ST_TOPK, ST_RESCORE, ST_RERANK, ST_END };

// Records an event at the start of each stage when timing is on.
struct StageTimer {
  Index* ix;
  cudaStream_t s;
  bool on;
  std::vector<std::pair<int, cudaEvent_t>> marks;
  KernelClock kc;
  StageTimer(Index* i, cudaStream_t st) : ix(i), s(st), on(i && i->timing) {
    kc.on = on;
    kc.s = st;
  }
  void mark(int stage) {
    if (!on) return;
    cudaEvent_t e;
    GIFT_CUDA(cudaEventCreate(&e));
    GIFT_CUDA(cudaEventRecord(e, s));
    marks.emplace_back(stage, e);
  }
  // hand the events to the index (read back by gift_get_timing)
  void finish() {
    if (!on) return;
    mark(ST_END);
    for (cudaEvent_t e : ix->ev) cudaEventDestroy(e);
    ix->ev.clear();
    ix->ev_stage.clear();
    for (auto& m : marks) {
      ix->ev.push_back(m.second);
      ix->ev_stage.push_back(m.first);
    }
    marks.clear();
    for (auto& k : ix->kspans) {
      cudaEventDestroy(k.second.first);
      cudaEventDestroy(k.second.second);
    }
    ix->kspans = kc.spans;
    ix->k_assign_rows = kc.assign_rows;
    kc.spans.clear();
  }
  ~StageTimer() {
    for (auto& m : marks) cudaEventDestroy(m.second);
    for (auto& k : kc.spans) {
      cudaEventDestroy(k.second.first);
      cudaEventDestroy(k.second.second);
    }
  }
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A device view of a caller buffer: device pointers pass through, host
// pointers are staged into scratch (in) or copied back after the work (out).
template <class T>
const T* stage_in(const T* p, size_t n, Scratch& sc, cudaStream_t s) {
  if (!p || is_device_ptr(p)) return p;
  T* d = sc.get<T>(n);
  GIFT_CUDA(cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, s));
  return d;
}

struct OutBuf {
  void* user = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
};
template <class T>
T* stage_out(T* p, size_t n, Scratch& sc, std::vector<OutBuf>& outs) {
  if (!p || is_device_ptr(p)) return p;
  T* d = sc.get<T>(n);
  outs.push_back(OutBuf{p, d, n * sizeof(T)});
  return d;
}
void flush_out(std::vector<OutBuf>& outs, cudaStream_t s) {
  for (auto& o : outs) GIFT_CUDA(cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, s));
}

gift_status guard(const char* fn, const std::function<void()>& body);

__global__ void k_view_query_map(const int32_t* __restrict__ qoff, int32_t* __restrict__ vq) {
  const int b = blockIdx.x;
  for (int v = qoff[b] + threadIdx.x; v < qoff[b + 1]; v += blockDim.x) vq[v] = b;
}

template <typename TO>
__device__ __forceinline__ TO cvt_store(float x);
template <>
__device__ __forceinline__ float cvt_store<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_store<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __nv_fp8_e4m3 cvt_store<__nv_fp8_e4m3>(float x) { return __nv_fp8_e4m3(x); }

// list-ordered feature store: stored = x / scale (scale = max|x|/448 for FP8,
// 1 otherwise); list_scale = scale / ||x|| turns a stored dot into a cosine.
template <typename TO>
__global__ void k_pack_lists(const float* __restrict__ master, const int32_t* __restrict__ list_row,
                             const float* __restrict__ row_inv, int64_t n, int D, TO* __restrict__ out,
                             float* __restrict__ scale_out, int fp8) {
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= n) return;
  const int32_t row = list_row[e];
  const float* x = master + (int64_t)row * D;
  float sc = 1.f;
  if (fp8) {
    float m = 0.f;
    for (int d = lane; d < D; d += 32) m = fmaxf(m, fabsf(x[d]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    sc = m > 0.f ? m / 448.f : 1.f;
  }
  const float inv_sc = 1.f / sc;
  TO* o = out + e * D;
  for (int d = lane; d < D; d += 32) o[d] = cvt_store<TO>(fp8 ? x[d] * inv_sc : x[d]);
  if (lane == 0) scale_out[e] = sc * row_inv[row];
}

// residual of the BF16 store: lo = bf16(x - bf16(x)), list order
__global__ void k_pack_lo(const float* __restrict__ master, const int32_t* __restrict__ list_row, int64_t n, int D,
                          __nv_bfloat16* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= n) return;
  const float* x = master + (int64_t)list_row[e] * D;
  __nv_bfloat16* o = out + e * D;
  for (int d = lane; d < D; d += 32) {
    const float v = x[d];
    o[d] = __float2bfloat16_rn(v - __bfloat162float(__float2bfloat16_rn(v)));
  }
}

__global__ void k_list_meta(const int32_t* __restrict__ list_row, const int32_t* __restrict__ skeys, int64_t n,
                            int nv, int32_t* __restrict__ list_shape, int64_t* __restrict__ run_flag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int32_t shape = list_row[e] / nv;
  list_shape[e] = shape;
  const bool start = (e == 0) || skeys[e] != skeys[e - 1] || (list_row[e - 1] / nv) != shape;
  run_flag[e] = start ? 1 : 0;
}

// Runs of a list: maximal groups of consecutive entries with one shape id. The
// stable sort by codeword keeps the (row, assignment) item order inside a list,
// rows are shape * N_v + view and a view enters a list at most once, so list
// entries are in ascending (shape, view) order and the run shapes of a list
// are strictly ascending (the candidate merge of the combine relies on it).
__global__ void k_runs(const int64_t* __restrict__ run_id_excl, const int64_t* __restrict__ run_flag,
                       const int32_t* __restrict__ skeys, const int64_t* __restrict__ list_off,
                       const int32_t* __restrict__ list_shape, int64_t n, int32_t* __restrict__ entry_run,
                       int32_t* __restrict__ run_shape) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int64_t gid = run_id_excl[e] + run_flag[e] - 1;  // global run of entry e
  const int64_t first = list_off[skeys[e]];
  const int64_t base = run_id_excl[first] + run_flag[first] - 1;
  entry_run[e] = (int32_t)(gid - base);
  if (run_flag[e]) run_shape[gid] = list_shape[e];
}

__global__ void k_list_runs(const int64_t* __restrict__ list_off, const int64_t* __restrict__ run_id_excl,
                            const int64_t* __restrict__ run_flag, int K, int64_t n_runs_total,
                            int32_t* __restrict__ nruns, int64_t* __restrict__ run_off,
                            int* __restrict__ stats /* max_runs, max_list, nonempty */,
                            unsigned long long* __restrict__ tiles) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const int64_t a = list_off[k], b = list_off[k + 1];
  if (b > a) {
    const int64_t r0 = run_id_excl[a] + run_flag[a] - 1;
    const int64_t r1 = (b < list_off[K]) ? run_id_excl[b] + run_flag[b] - 1 : n_runs_total;
    nruns[k] = (int32_t)(r1 - r0);
    run_off[k] = r0;
    atomicMax(&stats[0], (int)(r1 - r0));
    atomicMax(&stats[1], (int)(b - a));
    atomicAdd(&stats[2], 1);
    atomicAdd(tiles, (unsigned long long)cdiv(b - a, kScanTE));
  } else {
    nruns[k] = 0;
    run_off[k] = 0;
  }
}

__global__ void k_cb_maxnorm(const float* __restrict__ half_sq, int K, float* __restrict__ out) {
  float m = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) m = fmaxf(m, half_sq[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float w[32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = fmaxf(r, w[i]);
    out[0] = sqrtf(2.f * r);
  }
}

}  // namespace

void prepare_codebook(Index& ix, cudaStream_t s) {
  const int K = ix.prm.n_codewords, D = ix.prm.dim;
  if (!ix.cb_half_sq) {
    ix.cb_half_sq = ix.alloc<float>(K);
    ix.cb_rows_alloc = (int64_t)K + 256;  // one TMA box of padding rows
    ix.cb_hi = ix.alloc<__nv_bfloat16>((size_t)ix.cb_rows_alloc * D);
    ix.cb_lo = ix.alloc<__nv_bfloat16>((size_t)ix.cb_rows_alloc * D);
    GIFT_CUDA(cudaMemsetAsync(ix.cb_hi, 0, (size_t)ix.cb_rows_alloc * D * 2, s));
    GIFT_CUDA(cudaMemsetAsync(ix.cb_lo, 0, (size_t)ix.cb_rows_alloc * D * 2, s));
  }
  launch_half_sq_norm(ix.codebook, K, D, ix.cb_half_sq, s);
  split_rows_bf16(ix.codebook, K, D, ix.cb_hi, ix.cb_lo, s);
  Scratch sc(s);
  float* d_cbmax = sc.get<float>(1);
  k_cb_maxnorm<<<1, 1024, 0, s>>>(ix.cb_half_sq, K, d_cbmax);
  GIFT_LAUNCHED("k_cb_maxnorm");
  GIFT_CUDA(cudaMemcpyAsync(&ix.cb_max_norm, d_cbmax, 4, cudaMemcpyDeviceToHost, s));
  GIFT_CUDA(cudaStreamSynchronize(s));
  ix.cb_max_norm *= 1.0001f;
}

namespace {

// pass 2 of a streamed build: pack the rows of one chunk into their list
// positions (store dtype + cosine factor; BF16 parts for the rescore)
template <typename TO>
__global__ void k_scatter_pack(const float* __restrict__ chunk, int64_t row0, int64_t n, int D, int ma,
                               const int32_t* __restrict__ pos, const float* __restrict__ row_inv,
                               TO* __restrict__ out, float* __restrict__ scale_out, int fp8,
                               __nv_bfloat16* __restrict__ hi, float* __restrict__ scale_hi,
                               __nv_bfloat16* __restrict__ lo) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const float* x = chunk + r * D;
  float sc = 1.f;
  if (fp8) {
    float m = 0.f;
    for (int d = lane; d < D; d += 32) m = fmaxf(m, fabsf(x[d]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    sc = m > 0.f ? m / 448.f : 1.f;
  }
  const float inv_sc = 1.f / sc;
  for (int a = 0; a < ma; ++a) {  // one copy per list the view entered
    const int64_t e = pos[(row0 + r) * ma + a];
    for (int d = lane; d < D; d += 32) {
      const float v = x[d];
      out[e * D + d] = cvt_store<TO>(fp8 ? v * inv_sc : v);
      if (lo) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        lo[e * D + d] = __float2bfloat16_rn(v - __bfloat162float(h));
        if (hi) hi[e * D + d] = h;
      }
    }
    if (lane == 0) {
      scale_out[e] = sc * row_inv[row0 + r];
      if (scale_hi) scale_hi[e] = row_inv[row0 + r];
    }
  }
}

// (row, assignment) item of each entry -> its row; pos[item] = entry (optional)
__global__ void k_items_to_rows(int32_t* __restrict__ list_row, int64_t n, int ma, int32_t* __restrict__ pos) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int32_t item = list_row[e];
  if (pos) pos[item] = (int32_t)e;
  list_row[e] = item / ma;
}

// F-IF from the database codes: stable sort of the (row, assignment) items by
// code (lists in (shape, view) order), shape ids, runs of equal shape per
// list, sizes. pos (optional, [n_entries]) receives the entry of each item.
void build_lists(Index& ix_, Scratch& sc, cudaStream_t s, int32_t* pos = nullptr) {
  Index* ix = &ix_;
  const int K = ix->prm.n_codewords, Nv = ix->prm.views_per_shape;
  const int64_t n_rows = ix->n_entries;  // list entries (views x database-side assignments)
  ix->list_row = ix->alloc<int32_t>(n_rows);
  int32_t* skeys = sc.get<int32_t>(n_rows);
  stable_sort_by_key(ix->db_codes, n_rows, K, ix->list_row, skeys, sc, s);
  k_items_to_rows<<<(unsigned)cdiv(n_rows, 256), 256, 0, s>>>(ix->list_row, n_rows, ix->db_ma, pos);
  GIFT_LAUNCHED("k_items_to_rows");
  ix->list_off = ix->alloc<int64_t>(K + 1);
  bin_offsets(skeys, n_rows, K, ix->list_off, s);
  ix->list_shape = ix->alloc<int32_t>(n_rows);
  int64_t* run_flag = sc.get<int64_t>(n_rows + 1);
  k_list_meta<<<(unsigned)cdiv(n_rows, 256), 256, 0, s>>>(ix->list_row, skeys, n_rows, Nv, ix->list_shape,
                                                            run_flag);
  GIFT_LAUNCHED("k_list_meta");
  int64_t* run_excl = sc.get<int64_t>(n_rows + 1);
  scan_exclusive_i64(run_flag, run_excl, n_rows, sc, s);
  int64_t h_last[2];
  GIFT_CUDA(cudaMemcpyAsync(&h_last[0], run_excl + n_rows - 1, 8, cudaMemcpyDeviceToHost, s));
  GIFT_CUDA(cudaMemcpyAsync(&h_last[1], run_flag + n_rows - 1, 8, cudaMemcpyDeviceToHost, s));
  GIFT_CUDA(cudaStreamSynchronize(s));
  ix->n_runs = h_last[0] + h_last[1];
  ix->entry_run = ix->alloc<int32_t>(n_rows);
  ix->run_shape = ix->alloc<int32_t>(ix->n_runs);
  k_runs<<<(unsigned)cdiv(n_rows, 256), 256, 0, s>>>(run_excl, run_flag, skeys, ix->list_off, ix->list_shape,
                                                       n_rows, ix->entry_run, ix->run_shape);
  GIFT_LAUNCHED("k_runs");
  ix->nruns = ix->alloc<int32_t>(K);
  ix->run_off = ix->alloc<int64_t>(K);
  int* d_stats = sc.get<int>(4);
  unsigned long long* d_tiles = sc.get<unsigned long long>(1);
  GIFT_CUDA(cudaMemsetAsync(d_stats, 0, 16, s));
  GIFT_CUDA(cudaMemsetAsync(d_tiles, 0, 8, s));
  k_list_runs<<<(unsigned)cdiv(K, 256), 256, 0, s>>>(ix->list_off, run_excl, run_flag, K, ix->n_runs, ix->nruns,
                                                       ix->run_off, d_stats, d_tiles);
  GIFT_LAUNCHED("k_list_runs");
  int h_stats[4];
  unsigned long long h_tiles = 0;
  ix->h_list_off.resize(K + 1);
  GIFT_CUDA(cudaMemcpyAsync(h_stats, d_stats, 16, cudaMemcpyDeviceToHost, s));
  GIFT_CUDA(cudaMemcpyAsync(&h_tiles, d_tiles, 8, cudaMemcpyDeviceToHost, s));
  GIFT_CUDA(cudaMemcpyAsync(ix->h_list_off.data(), ix->list_off, (K + 1) * 8, cudaMemcpyDeviceToHost, s));

  GIFT_CUDA(cudaStreamSynchronize(s));
  ix->max_runs = h_stats[0];
  ix->max_list = h_stats[1];
  ix->n_nonempty = h_stats[2];
  ix->scan_tiles_upper = (int64_t)h_tiles;
}

// ------------------------------------------------------------------ query core
// The BF16 store is the hi part of the two-part rescore rows: the scan runs at
// FP32 level over every touched pair (for D > 64; a single k-block keeps the
// BF16 scan and the separate rescore)
bool fused_scan_ok(const Index& ix) {
  return ix.prm.storage == GIFT_BF16 && ix.list_lo != nullptr && ix.list_hi == nullptr && ix.prm.dim > 64;
}

struct QueryOut {
  int32_t* ids;
  float* scores;
};

void run_fif(Index& ix, const float* q, int64_t nv, const std::vector<int32_t>& h_qoff, int32_t B,
             int32_t topk, int32_t* out_ids, float* out_scores, Scratch& sc, cudaStream_t s,
             StageTimer& tm, unsigned long long* stats, const int32_t* d_qoff_in = nullptr,
             const int32_t* vquery_in = nullptr) {
  const int K = ix.prm.n_codewords;
  const int N = ix.prm.n_shapes;
  const int ma = ix.prm.query_ma;
  const int R = ix.prm.rescore_r;
  (void)K;
  tm.mark(ST_ASSIGN);
  const int32_t* d_qoff = d_qoff_in;
  if (!d_qoff) {
    int32_t* t = sc.get<int32_t>(B + 1);
    GIFT_CUDA(cudaMemcpyAsync(t, h_qoff.data(), (B + 1) * 4, cudaMemcpyHostToDevice, s));
    d_qoff = t;
  }
  const int32_t* vquery = vquery_in;
  if (!vquery) {
    int32_t* t = sc.get<int32_t>(nv);
    k_view_query_map<<<(unsigned)B, 128, 0, s>>>(d_qoff, t);
    GIFT_LAUNCHED("k_view_query_map");
    vquery = t;
  }
  float* q_inv = sc.get<float>(nv);
  launch_row_invnorm(q, nv, ix.prm.dim, q_inv, s);
  int32_t* q_code = sc.get<int32_t>(nv * ma);
  assign_codes(ix, q, nv, ma, q_code, sc, s, q_inv, &tm.kc);

  tm.mark(ST_BUCKET);
  FifPlan P;
  P.nv = nv;
  P.ma = ma;
  P.B = B;
  P.q = q;
  P.q_inv = q_inv;
  P.q_code = q_code;
  P.qoff = d_qoff;
  P.vquery = vquery;
  P.stats = stats;
  P.kc = &tm.kc;
  fif_plan(ix, P, sc, s);
  uint32_t* table = sc.get<uint32_t>(P.table_upper);
  fif_zero_table(P, table, s);
  // a BF16 store that is the hi part of the rescore rows: one pass over every
  // touched pair at FP32 level gives the maxima both the candidate selection and
  // the candidates' scores read (no separate rescore)
  const bool fused = R > 0 && fused_scan_ok(ix);
  uint32_t* table32 = fused ? table : nullptr;

  tm.mark(ST_SCAN);
  if (fused)
    fif_scan_tc(ix, P, table, false, nullptr, 0, sc, s, table32);
  else if (ix.prm.storage != GIFT_F32)
    fif_scan_tc(ix, P, table, false, nullptr, 0, sc, s);
  else
    fif_scan(ix, P, table, false, nullptr, 0, s);

  tm.mark(ST_COMBINE);
  float* S = sc.get<float>((size_t)B * N);
  fif_combine(ix, P, table, S, nullptr, 0, nullptr, sc, s);

  tm.mark(ST_TOPK);
  if (R <= 0) {
    topk_rows_f32(S, B, N, topk, out_ids, out_scores, sc, s);
    return;
  }
  const int Rr = std::min(R, N);
  int32_t* cand = sc.get<int32_t>((size_t)B * Rr);
  topk_rows_f32(S, B, N, Rr, cand, nullptr, sc, s);
  int32_t* cand_sorted = sc.get<int32_t>((size_t)B * Rr);
  sort_ids_rows(cand, B, Rr, cand_sorted, s);

  tm.mark(ST_RESCORE);
  if (fused) fif_rescore_stats(ix, P, cand_sorted, Rr, sc, s);  // timed calls only
  if (!fused) {
    fif_zero_table(P, table, s);
    if (ix.list_lo)
      fif_scan_tc(ix, P, table, true, cand_sorted, Rr, sc, s);
    else
      fif_scan(ix, P, table, true, cand_sorted, Rr, s);
  }
  float* cand_score = sc.get<float>((size_t)B * Rr);
  fif_combine(ix, P, fused ? table32 : table, nullptr, cand_sorted, Rr, cand_score, sc, s);
  tm.mark(ST_TOPK);
  sort_candidates(cand_sorted, cand_score, B, Rr, topk, out_ids, out_scores, s);
}

}  // namespace

// ------------------------------------------------------------------ plumbing
void KernelClock::begin(int id) {
  if (!on) return;
  cudaEvent_t a, b;
  GIFT_CUDA(cudaEventCreate(&a));
  GIFT_CUDA(cudaEventCreate(&b));
  GIFT_CUDA(cudaEventRecord(a, s));
  spans.push_back({id, {a, b}});
}
void KernelClock::end(int id) {
  if (!on) return;
  for (auto it = spans.rbegin(); it != spans.rend(); ++it)
    if (it->first == id) {
      GIFT_CUDA(cudaEventRecord(it->second.second, s));
      return;
    }
}

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

[[noreturn]] void fail(gift_status s, const std::string& msg) { throw Error(s, msg); }

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  cudaGetLastError();
  throw Error(e == cudaErrorMemoryAllocation ? GIFT_ENOMEM : GIFT_ECUDA, buf);
}

Scratch::~Scratch() {
  for (void* p : blocks) cudaFreeAsync(p, stream);
}

void* Scratch::raw(size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, std::max<size_t>(bytes, 16), stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(GIFT_ENOMEM, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
  }
  blocks.push_back(p);
  return p;
}

template <class T>
T* Index::alloc(size_t n) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(n * sizeof(T), 16);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(GIFT_ENOMEM, "index allocation of " + std::to_string(bytes) + " bytes failed");
  }
  owned.push_back(p);
  device_bytes += bytes;
  return static_cast<T*>(p);
}

Index::~Index() {
  delete sb;
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  for (auto& k : kspans) {
    cudaEventDestroy(k.second.first);
    cudaEventDestroy(k.second.second);
  }
  if (stats_pinned) cudaFreeHost(stats_pinned);
  for (void* p : owned) cudaFree(p);
}

size_t dtype_bytes(int storage) { return storage == GIFT_F32 ? 4 : storage == GIFT_BF16 ? 2 : 1; }

namespace {

gift_status guard(const char* fn, const std::function<void()>& body) {
  try {
    body();
    g_last_error.clear();
    return GIFT_OK;
  } catch (const Error& e) {
    g_last_error = std::string(fn) + ": " + e.what();
    return e.status;
  } catch (const std::bad_alloc&) {
    g_last_error = std::string(fn) + ": host allocation failed";
    return GIFT_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = std::string(fn) + ": " + e.what();
    return GIFT_EINVAL;
  } catch (...) {
    g_last_error = std::string(fn) + ": unknown error";
    return GIFT_EINVAL;
  }
}

}  // namespace

gift_status guarded(const char* fn, const std::function<void()>& body) { return guard(fn, body); }

namespace {

std::vector<int32_t> host_offsets(const int32_t* q_view_offsets, int32_t B) {
  GIFT_REQUIRE(q_view_offsets != nullptr, "q_view_offsets is NULL");
  GIFT_REQUIRE(!is_device_ptr(q_view_offsets), "q_view_offsets must be a host pointer");
  std::vector<int32_t> h(q_view_offsets, q_view_offsets + B + 1);
  GIFT_REQUIRE(h[0] == 0, "q_view_offsets[0] must be 0");
  for (int b = 0; b < B; ++b) GIFT_REQUIRE(h[b + 1] > h[b], "every query needs at least one view");
  return h;
}

void build(const gift_index_params* prm, const float* db_feats, const float* codebook, cudaStream_t s,
           gift_index** out) {
  GIFT_REQUIRE(prm && db_feats && codebook && out, "NULL argument");
  const gift_index_params p = *prm;
  GIFT_REQUIRE(p.n_shapes > 0 && p.views_per_shape > 0 && p.n_codewords > 0, "sizes must be positive");
  GIFT_REQUIRE(p.dim > 0 && p.dim % 16 == 0, "dim must be a positive multiple of 16");
  GIFT_REQUIRE(p.storage >= GIFT_F32 && p.storage <= GIFT_FP8_E4M3, "unknown storage type");
  GIFT_REQUIRE(p.query_ma >= 1 && p.query_ma <= GIFT_MAX_MA && p.query_ma <= p.n_codewords,
               "query_ma must be in [1, min(8, K)]");
  GIFT_REQUIRE(p.sif_k1 >= 0 && p.sif_k1 <= std::min(1024, p.n_shapes), "sif_k1 must be in [0, min(1024, N)]");
  GIFT_REQUIRE(p.rescore_r >= 0 && p.rescore_r <= 1024, "rescore_r must be in [0, 1024]");
  GIFT_REQUIRE(p.views_per_shape <= 32767, "views_per_shape must be <= 32767");
  const int64_t n_rows = (int64_t)p.n_shapes * p.views_per_shape;
  GIFT_REQUIRE(p.db_ma >= 0 && p.db_ma <= GIFT_MAX_MA && p.db_ma <= p.n_codewords,
               "db_ma must be in [0, min(8, K)]");
  const int db_ma = std::max(1, p.db_ma);
  GIFT_REQUIRE(n_rows * db_ma < (int64_t)INT32_MAX, "too many database views");

  std::unique_ptr<Index> ix(new Index());
  ix->prm = p;
  ix->n_rows = n_rows;
  ix->db_ma = db_ma;
  ix->n_entries = n_rows * db_ma;
  GIFT_CUDA(cudaGetDevice(&ix->device));
  {
    // per-call scratch comes from the device's default stream-ordered pool;
    // keep freed blocks cached there so steady-state calls do not reallocate
    cudaMemPool_t pool;
    GIFT_CUDA(cudaDeviceGetDefaultMemPool(&pool, ix->device));
    uint64_t keep = UINT64_MAX;
    GIFT_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  }
  const int D = p.dim, K = p.n_codewords, N = p.n_shapes, Nv = p.views_per_shape;
  Scratch sc(s);

  // codebook
  ix->codebook = ix->alloc<float>((size_t)K * D);
  GIFT_CUDA(cudaMemcpyAsync(ix->codebook, codebook, (size_t)K * D * 4, cudaMemcpyDefault, s));
  ix->cb_half_sq = ix->alloc<float>(K);
  launch_half_sq_norm(ix->codebook, K, D, ix->cb_half_sq, s);
  ix->cb_rows_alloc = (int64_t)K + 256;  // one TMA box of padding rows
  ix->cb_hi = ix->alloc<__nv_bfloat16>((size_t)ix->cb_rows_alloc * D);
  ix->cb_lo = ix->alloc<__nv_bfloat16>((size_t)ix->cb_rows_alloc * D);
  GIFT_CUDA(cudaMemsetAsync(ix->cb_hi, 0, (size_t)ix->cb_rows_alloc * D * 2, s));
  GIFT_CUDA(cudaMemsetAsync(ix->cb_lo, 0, (size_t)ix->cb_rows_alloc * D * 2, s));
  split_rows_bf16(ix->codebook, K, D, ix->cb_hi, ix->cb_lo, s);
  float* d_cbmax = sc.get<float>(1);
  k_cb_maxnorm<<<1, 1024, 0, s>>>(ix->cb_half_sq, K, d_cbmax);
  GIFT_LAUNCHED("k_cb_maxnorm");

  // FP32 master (kept for the exact match and the rescore; otherwise scratch)
  const bool split_rescore = p.rescore_r > 0 && p.storage != GIFT_F32;
  const bool need_master = p.keep_exact || (p.rescore_r > 0 && !split_rescore);
  float* master = need_master ? ix->alloc<float>((size_t)n_rows * D) : sc.get<float>((size_t)n_rows * D);
  if (need_master) ix->master = master;
  ix->d_err = ix->alloc<int>(1);
  GIFT_CUDA(cudaMemsetAsync(ix->d_err, 0, sizeof(int), s));
  GIFT_CUDA(cudaMemcpyAsync(master, db_feats, (size_t)n_rows * D * 4, cudaMemcpyDefault, s));
  ix->row_inv = ix->alloc<float>(n_rows);
  launch_row_invnorm(master, n_rows, D, ix->row_inv, s);
  GIFT_CUDA(cudaMemcpyAsync(&ix->cb_max_norm, d_cbmax, 4, cudaMemcpyDeviceToHost, s));
  GIFT_CUDA(cudaStreamSynchronize(s));
  ix->cb_max_norm *= 1.0001f;

  // database codes (one assignment per view)
  ix->db_codes = ix->alloc<int32_t>(n_rows * db_ma);
  assign_codes(*ix, master, n_rows, db_ma, ix->db_codes, sc, s, ix->row_inv);

  build_lists(*ix, sc, s);

  // list-ordered feature store (a view appears once per list it enters)
  const int64_t n_ent = ix->n_entries;
  const size_t eb = dtype_bytes(p.storage);
  ix->list_rows_alloc = n_ent + 256;  // one TMA box of padding rows
  ix->list_feat = ix->alloc<uint8_t>((size_t)ix->list_rows_alloc * D * eb);
  GIFT_CUDA(cudaMemsetAsync((uint8_t*)ix->list_feat + (size_t)n_ent * D * eb, 0, (size_t)256 * D * eb, s));
  ix->list_scale = ix->alloc<float>(n_ent);
  const unsigned pg = (unsigned)cdiv(n_ent, 8);
  switch (p.storage) {
    case GIFT_F32:
      k_pack_lists<float><<<pg, 256, 0, s>>>(master, ix->list_row, ix->row_inv, n_ent, D,
                                             (float*)ix->list_feat, ix->list_scale, 0);
      break;
    case GIFT_BF16:
      k_pack_lists<__nv_bfloat16><<<pg, 256, 0, s>>>(master, ix->list_row, ix->row_inv, n_ent, D,
                                                     (__nv_bfloat16*)ix->list_feat, ix->list_scale, 0);
      break;
    default:
      k_pack_lists<__nv_fp8_e4m3><<<pg, 256, 0, s>>>(master, ix->list_row, ix->row_inv, n_ent, D,
                                                     (__nv_fp8_e4m3*)ix->list_feat, ix->list_scale, 1);
      break;
  }
  GIFT_LAUNCHED("k_pack_lists");
  if (split_rescore) {
    ix->list_lo = ix->alloc<__nv_bfloat16>((size_t)ix->list_rows_alloc * D);
    GIFT_CUDA(cudaMemsetAsync((__nv_bfloat16*)ix->list_lo + (size_t)n_ent * D, 0, (size_t)256 * D * 2, s));
    k_pack_lo<<<pg, 256, 0, s>>>(master, ix->list_row, n_ent, D, (__nv_bfloat16*)ix->list_lo);
    GIFT_LAUNCHED("k_pack_lo");
    if (p.storage == GIFT_FP8_E4M3) {
      // the FP8 store scans; the rescore reads a separate BF16 hi part
      ix->list_hi = ix->alloc<__nv_bfloat16>((size_t)ix->list_rows_alloc * D);
      GIFT_CUDA(cudaMemsetAsync((__nv_bfloat16*)ix->list_hi + (size_t)n_ent * D, 0, (size_t)256 * D * 2, s));
      ix->list_scale_hi = ix->alloc<float>(n_ent);
      k_pack_lists<__nv_bfloat16><<<pg, 256, 0, s>>>(master, ix->list_row, ix->row_inv, n_ent, D,
                                                     (__nv_bfloat16*)ix->list_hi, ix->list_scale_hi, 0);
      GIFT_LAUNCHED("k_pack_lists");
    }
  }
  if (p.keep_exact) {
    // shape-ordered two-part BF16 copy for the exact match on the tensor cores
    ix->ex_rows = n_rows + 128;
    ix->ex_hi = ix->alloc<__nv_bfloat16>((size_t)ix->ex_rows * D);
    ix->ex_lo = ix->alloc<__nv_bfloat16>((size_t)ix->ex_rows * D);
    GIFT_CUDA(cudaMemsetAsync(ix->ex_hi + (size_t)n_rows * D, 0, (size_t)128 * D * 2, s));
    GIFT_CUDA(cudaMemsetAsync(ix->ex_lo + (size_t)n_rows * D, 0, (size_t)128 * D * 2, s));
    split_rows_bf16(master, n_rows, D, ix->ex_hi, ix->ex_lo, s);
  }
  GIFT_CUDA(cudaStreamSynchronize(s));

  // S-IF: every database shape as a query, first k1 neighbours (self included)
  if (p.sif_k1 > 0) {
    ix->k1 = p.sif_k1;
    ix->sif_n = N;
    ix->sif_off = ix->alloc<int64_t>(N + 1);
    ix->sif_ids = ix->alloc<int32_t>((size_t)N * p.sif_k1);
    ix->sif_mem = ix->alloc<uint32_t>((size_t)N * p.sif_k1);
    ix->sif_card = ix->alloc<uint64_t>(N);
    int32_t* nbr_ids = ix->row_ids = ix->alloc<int32_t>((size_t)N * p.sif_k1);
    float* nbr_sc = ix->row_sc = ix->alloc<float>((size_t)N * p.sif_k1);
    // batches of database shapes, bounded by the dense score block
    const int64_t per = std::max<int64_t>(1, std::min<int64_t>(1024, ((int64_t)1 << 26) / std::max(1, N)));
    const int topk = p.rescore_r > 0 ? std::min(p.sif_k1, p.rescore_r) : p.sif_k1;
    GIFT_REQUIRE(p.rescore_r == 0 || p.sif_k1 <= p.rescore_r, "sif_k1 must be <= rescore_r when rescoring");
    for (int64_t b0 = 0; b0 < N; b0 += per) {
      const int32_t nb = (int32_t)std::min<int64_t>(per, N - b0);
      std::vector<int32_t> h(nb + 1);
      for (int32_t i = 0; i <= nb; ++i) h[i] = i * Nv;
      Scratch bsc(s);
      StageTimer none(nullptr, s);
      run_fif(*ix, master + b0 * Nv * (int64_t)D, (int64_t)nb * Nv, h, nb, topk, nbr_ids + b0 * p.sif_k1,
              nbr_sc + b0 * p.sif_k1, bsc, s, none, nullptr);
    }
    sif_build(*ix, nbr_ids, nbr_sc, sc, s);
  }
  GIFT_CUDA(cudaStreamSynchronize(s));
  *out = reinterpret_cast<gift_index*>(ix.release());
}

void stream_begin(const gift_index_params* prm, const float* codebook, cudaStream_t s, gift_index** out) {
  GIFT_REQUIRE(prm && codebook && out, "NULL argument");
  const gift_index_params p = *prm;
  GIFT_REQUIRE(p.n_shapes > 0 && p.views_per_shape > 0 && p.n_codewords > 0, "sizes must be positive");
  GIFT_REQUIRE(p.dim > 0 && p.dim % 16 == 0, "dim must be a positive multiple of 16");
  GIFT_REQUIRE(p.storage >= GIFT_F32 && p.storage <= GIFT_FP8_E4M3, "unknown storage type");
  GIFT_REQUIRE(p.storage != GIFT_F32 || p.rescore_r == 0, "a streamed FP32 store does not rescore");
  GIFT_REQUIRE(p.query_ma >= 1 && p.query_ma <= GIFT_MAX_MA && p.query_ma <= p.n_codewords,
               "query_ma must be in [1, min(8, K)]");
  GIFT_REQUIRE(p.sif_k1 >= 0 && p.sif_k1 <= std::min(1024, p.n_shapes), "sif_k1 must be in [0, min(1024, N)]");
  GIFT_REQUIRE(p.rescore_r >= 0 && p.rescore_r <= 1024, "rescore_r must be in [0, 1024]");
  GIFT_REQUIRE(p.rescore_r == 0 || p.sif_k1 <= p.rescore_r, "sif_k1 must be <= rescore_r when rescoring");
  GIFT_REQUIRE(!p.keep_exact, "a streamed build keeps no FP32 master (keep_exact must be 0)");
  GIFT_REQUIRE(p.views_per_shape <= 32767, "views_per_shape must be <= 32767");
  const int64_t n_rows = (int64_t)p.n_shapes * p.views_per_shape;
  GIFT_REQUIRE(p.db_ma >= 0 && p.db_ma <= GIFT_MAX_MA && p.db_ma <= p.n_codewords,
               "db_ma must be in [0, min(8, K)]");
  const int db_ma = std::max(1, p.db_ma);
  GIFT_REQUIRE(n_rows * db_ma < (int64_t)INT32_MAX, "too many database views");
  std::unique_ptr<Index> ix(new Index());
  ix->prm = p;
  ix->n_rows = n_rows;
  ix->db_ma = db_ma;
  ix->n_entries = n_rows * db_ma;
  GIFT_CUDA(cudaGetDevice(&ix->device));
  {
    cudaMemPool_t pool;
    GIFT_CUDA(cudaDeviceGetDefaultMemPool(&pool, ix->device));
    uint64_t keep = UINT64_MAX;
    GIFT_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  }
  const int D = p.dim, K = p.n_codewords;
  Scratch sc(s);
  ix->codebook = ix->alloc<float>((size_t)K * D);
  GIFT_CUDA(cudaMemcpyAsync(ix->codebook, codebook, (size_t)K * D * 4, cudaMemcpyDefault, s));
  ix->cb_half_sq = ix->alloc<float>(K);
  launch_half_sq_norm(ix->codebook, K, D, ix->cb_half_sq, s);
  ix->cb_rows_alloc = (int64_t)K + 256;
  ix->cb_hi = ix->alloc<__nv_bfloat16>((size_t)ix->cb_rows_alloc * D);
  ix->cb_lo = ix->alloc<__nv_bfloat16>((size_t)ix->cb_rows_alloc * D);
  GIFT_CUDA(cudaMemsetAsync(ix->cb_hi, 0, (size_t)ix->cb_rows_alloc * D * 2, s));
  GIFT_CUDA(cudaMemsetAsync(ix->cb_lo, 0, (size_t)ix->cb_rows_alloc * D * 2, s));
  split_rows_bf16(ix->codebook, K, D, ix->cb_hi, ix->cb_lo, s);
  float* d_cbmax = sc.get<float>(1);
  k_cb_maxnorm<<<1, 1024, 0, s>>>(ix->cb_half_sq, K, d_cbmax);
  GIFT_LAUNCHED("k_cb_maxnorm");
  GIFT_CUDA(cudaMemcpyAsync(&ix->cb_max_norm, d_cbmax, 4, cudaMemcpyDeviceToHost, s));
  ix->row_inv = ix->alloc<float>(n_rows);
  ix->db_codes = ix->alloc<int32_t>(n_rows * db_ma);
  ix->d_err = ix->alloc<int>(1);
  GIFT_CUDA(cudaMemsetAsync(ix->d_err, 0, sizeof(int), s));
  GIFT_CUDA(cudaStreamSynchronize(s));
  ix->cb_max_norm *= 1.0001f;
  ix->sb = new StreamBuild();
  *out = reinterpret_cast<gift_index*>(ix.release());
}

void stream_add(Index& ix, int pass, const float* feats, int32_t first, int32_t n, cudaStream_t s) {
  if (!ix.sb) fail(GIFT_ESTATE, "the index is not being built in a stream");
  GIFT_REQUIRE(pass == ix.sb->stage, "chunks of pass " + std::to_string(ix.sb->stage) + " are expected");
  GIFT_REQUIRE(feats && n > 0 && first >= 0 && (int64_t)first + n <= ix.prm.n_shapes, "chunk out of range");
  std::vector<uint8_t>& seen = ix.sb->seen;
  if (seen.empty()) seen.assign(ix.prm.n_shapes, 0);
  for (int32_t i = first; i < first + n; ++i)
    GIFT_REQUIRE(!seen[i], "shape " + std::to_string(i) + " was already added in this pass");
  const int D = ix.prm.dim, Nv = ix.prm.views_per_shape;
  const int64_t row0 = (int64_t)first * Nv, rows = (int64_t)n * Nv;
  Scratch sc(s);
  const float* x = feats;
  if (!is_device_ptr(feats)) {
    float* d = sc.get<float>((size_t)rows * D);
    GIFT_CUDA(cudaMemcpyAsync(d, feats, (size_t)rows * D * 4, cudaMemcpyHostToDevice, s));
    x = d;
  }
  if (pass == 1) {
    launch_row_invnorm(x, rows, D, ix.row_inv + row0, s);
    assign_codes(ix, x, rows, ix.db_ma, ix.db_codes + row0 * ix.db_ma, sc, s, ix.row_inv + row0);
  } else if (pass == 2) {
    const unsigned g = (unsigned)cdiv(rows, 8);
    __nv_bfloat16* hi = (__nv_bfloat16*)ix.list_hi;
    __nv_bfloat16* lo = (__nv_bfloat16*)ix.list_lo;
    switch (ix.prm.storage) {
      case GIFT_F32:
        k_scatter_pack<float><<<g, 256, 0, s>>>(x, row0, rows, D, ix.db_ma, ix.sb->pos, ix.row_inv, (float*)ix.list_feat,
                                                ix.list_scale, 0, nullptr, nullptr, nullptr);
        break;
      case GIFT_BF16:
        k_scatter_pack<__nv_bfloat16><<<g, 256, 0, s>>>(x, row0, rows, D, ix.db_ma, ix.sb->pos, ix.row_inv,
                                                        (__nv_bfloat16*)ix.list_feat, ix.list_scale, 0, nullptr,
                                                        nullptr, lo);
        break;
      default:
        k_scatter_pack<__nv_fp8_e4m3><<<g, 256, 0, s>>>(x, row0, rows, D, ix.db_ma, ix.sb->pos, ix.row_inv,
                                                        (__nv_fp8_e4m3*)ix.list_feat, ix.list_scale, 1, hi,
                                                        ix.list_scale_hi, lo);
        break;
    }
    GIFT_LAUNCHED("k_scatter_pack");
  } else {
    const int k1 = ix.prm.sif_k1;
    const int R = ix.prm.rescore_r;
    const int topk = R > 0 ? std::min(k1, R) : k1;
    const int64_t per = std::max<int64_t>(1, std::min<int64_t>(1024, ((int64_t)1 << 26) / ix.prm.n_shapes));
    for (int64_t b0 = 0; b0 < n; b0 += per) {
      const int32_t nb = (int32_t)std::min<int64_t>(per, n - b0);
      std::vector<int32_t> h(nb + 1);
      for (int32_t i = 0; i <= nb; ++i) h[i] = i * Nv;
      Scratch bsc(s);
      StageTimer none(nullptr, s);
      const int64_t shape0 = first + b0;
      run_fif(ix, x + b0 * Nv * (int64_t)D, (int64_t)nb * Nv, h, nb, topk, ix.row_ids + shape0 * k1,
              ix.row_sc + shape0 * k1, bsc, s, none, nullptr);
    }
  }
  GIFT_CUDA(cudaStreamSynchronize(s));  // the chunk buffer may be reused by the caller
  std::fill(seen.begin() + first, seen.begin() + first + n, (uint8_t)1);
  ix.sb->rows_added += rows;
}

void stream_end(Index& ix, int pass, cudaStream_t s) {
  if (!ix.sb) fail(GIFT_ESTATE, "the index is not being built in a stream");
  GIFT_REQUIRE(pass == ix.sb->stage, "pass " + std::to_string(ix.sb->stage) + " is the open pass");
  GIFT_REQUIRE(ix.sb->rows_added == ix.n_rows, "every database shape must be added once in each pass");
  const int D = ix.prm.dim;
  Scratch sc(s);
  if (pass == 1) {
    const int64_t n_ent = ix.n_entries;
    GIFT_CUDA(cudaMalloc(&ix.sb->pos, n_ent * sizeof(int32_t)));
    build_lists(ix, sc, s, ix.sb->pos);
    {  // the stores need most of the device: hand cached scratch back first
      cudaMemPool_t pool;
      GIFT_CUDA(cudaDeviceGetDefaultMemPool(&pool, ix.device));
      GIFT_CUDA(cudaStreamSynchronize(s));
      GIFT_CUDA(cudaMemPoolTrimTo(pool, 0));
    }
    const size_t eb = dtype_bytes(ix.prm.storage);
    ix.list_rows_alloc = n_ent + 256;
    ix.list_feat = ix.alloc<uint8_t>((size_t)ix.list_rows_alloc * D * eb);
    GIFT_CUDA(cudaMemsetAsync((uint8_t*)ix.list_feat + (size_t)n_ent * D * eb, 0, (size_t)256 * D * eb, s));
    ix.list_scale = ix.alloc<float>(n_ent);
    if (ix.prm.rescore_r > 0) {
      ix.list_lo = ix.alloc<__nv_bfloat16>((size_t)ix.list_rows_alloc * D);
      GIFT_CUDA(cudaMemsetAsync((__nv_bfloat16*)ix.list_lo + (size_t)n_ent * D, 0, (size_t)256 * D * 2, s));
      if (ix.prm.storage == GIFT_FP8_E4M3) {
        ix.list_hi = ix.alloc<__nv_bfloat16>((size_t)ix.list_rows_alloc * D);
        GIFT_CUDA(cudaMemsetAsync((__nv_bfloat16*)ix.list_hi + (size_t)n_ent * D, 0, (size_t)256 * D * 2, s));
        ix.list_scale_hi = ix.alloc<float>(n_ent);
      }
    }
    ix.sb->stage = 2;
  } else if (pass == 2) {
    if (ix.prm.sif_k1 > 0) {
      const int64_t n = (int64_t)ix.prm.n_shapes * ix.prm.sif_k1;
      GIFT_CUDA(cudaFree(ix.sb->pos));
      ix.sb->pos = nullptr;
      ix.row_ids = ix.alloc<int32_t>(n);
      ix.row_sc = ix.alloc<float>(n);
      ix.sb->stage = 3;
    } else {
      ix.sb->stage = 4;
    }
  } else {
    // the S-IF arrays appear only now, so no call sees a half-built S-IF
    const int64_t n = (int64_t)ix.prm.n_shapes * ix.prm.sif_k1;
    ix.k1 = ix.prm.sif_k1;
    ix.sif_n = ix.prm.n_shapes;
    ix.sif_off = ix.alloc<int64_t>(ix.prm.n_shapes + 1);
    ix.sif_ids = ix.alloc<int32_t>(n);
    ix.sif_mem = ix.alloc<uint32_t>(n);
    ix.sif_card = ix.alloc<uint64_t>(ix.prm.n_shapes);
    sif_build(ix, ix.row_ids, ix.row_sc, sc, s);
    ix.sb->stage = 4;
  }
  GIFT_CUDA(cudaStreamSynchronize(s));
  ix.sb->rows_added = 0;
  ix.sb->seen.clear();
  if (ix.sb->stage == 4) {
    delete ix.sb;
    ix.sb = nullptr;
  }
}

}  // namespace
}  // namespace gift

using gift::Index;

extern "C" {

gift_status gift_build_index(const gift_index_params* params, const float* db_feats, const float* codebook,
                             cudaStream_t stream, gift_index** out) {
  return gift::guard("gift_build_index", [&] { gift::build(params, db_feats, codebook, stream, out); });
}

gift_status gift_build_begin(const gift_index_params* params, const float* codebook, cudaStream_t stream,
                             gift_index** out) {
  return gift::guard("gift_build_begin", [&] { gift::stream_begin(params, codebook, stream, out); });
}

gift_status gift_build_add(gift_index* index, int32_t pass, const float* feats, int32_t first_shape,
                           int32_t n_shapes, cudaStream_t stream) {
  return gift::guard("gift_build_add", [&] {
    GIFT_REQUIRE(index, "NULL index");
    gift::stream_add(*reinterpret_cast<Index*>(index), pass, feats, first_shape, n_shapes, stream);
  });
}

gift_status gift_build_end_pass(gift_index* index, int32_t pass, cudaStream_t stream) {
  return gift::guard("gift_build_end_pass", [&] {
    GIFT_REQUIRE(index, "NULL index");
    gift::stream_end(*reinterpret_cast<Index*>(index), pass, stream);
  });
}

void gift_destroy_index(gift_index* index) {
  if (!index) return;
  cudaDeviceSynchronize();
  Index* ix = reinterpret_cast<Index*>(index);
  const int dev = ix->device;
  delete ix;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  cudaGetLastError();
}

gift_status gift_query(gift_index* index, const float* q_feats, const int32_t* q_view_offsets, int32_t B,
                       int32_t mode, int32_t topk, int32_t* out_ids, float* out_scores, cudaStream_t stream) {
  return gift::guard("gift_query", [&] {
    GIFT_REQUIRE(index && q_feats && out_ids && out_scores, "NULL argument");
    GIFT_REQUIRE(B > 0, "B must be positive");
    GIFT_REQUIRE(topk > 0 && topk <= 1024, "topk must be in [1, 1024]");
    Index& ix = *reinterpret_cast<Index*>(index);
    if (!ix.ready()) gift::fail(GIFT_ESTATE, "the streamed build of this index is not complete");
    std::vector<int32_t> h = gift::host_offsets(q_view_offsets, B);
    const int64_t nv = h[B];
    const int D = ix.prm.dim;
    gift::Scratch sc(stream);
    gift::StageTimer tm(&ix, stream);
    std::vector<gift::OutBuf> outs;
    unsigned long long* stats = nullptr;
    if (tm.on) {
      stats = sc.get<unsigned long long>(8);
      GIFT_CUDA(cudaMemsetAsync(stats, 0, 64, stream));
    }
    tm.mark(gift::ST_ASSIGN);
    const float* q = gift::stage_in(q_feats, (size_t)nv * D, sc, stream);
    int32_t* oid = gift::stage_out(out_ids, (size_t)B * topk, sc, outs);
    float* osc = gift::stage_out(out_scores, (size_t)B * topk, sc, outs);
    if (mode == GIFT_MATCH_EXACT) {
      if (!ix.ex_hi && !ix.list_lo)
        gift::fail(GIFT_EUNSUPPORTED, "exact match needs keep_exact or a two-part rescore store");
      int32_t* d_qoff = sc.get<int32_t>(B + 1);
      GIFT_CUDA(cudaMemcpyAsync(d_qoff, h.data(), (B + 1) * 4, cudaMemcpyHostToDevice, stream));
      float* q_inv = sc.get<float>(nv);
      gift::launch_row_invnorm(q, nv, D, q_inv, stream);
      tm.mark(gift::ST_SCAN);
      float* S = sc.get<float>((size_t)B * ix.prm.n_shapes);
      if (ix.ex_hi)
        gift::exact_scores_tc(ix, q, q_inv, nv, d_qoff, h, B, S, sc, stream);
      else
        gift::exact_scores_lists(ix, q, q_inv, nv, d_qoff, h, B, S, sc, stream);
      tm.mark(gift::ST_TOPK);
      gift::topk_rows_f32(S, B, ix.prm.n_shapes, topk, oid, osc, sc, stream);
    } else if (mode == GIFT_MATCH_FIF) {
      if (ix.prm.rescore_r > 0 && topk > std::min(ix.prm.rescore_r, ix.prm.n_shapes) && ix.prm.n_shapes >= topk)
        gift::fail(GIFT_EUNSUPPORTED, "topk exceeds the rescore depth");
      gift::run_fif(ix, q, nv, h, B, topk, oid, osc, sc, stream, tm, stats);
    } else {
      gift::fail(GIFT_EINVAL, "unknown matching mode");
    }
    gift::flush_out(outs, stream);
    if (tm.on) {
      if (!ix.stats_pinned) GIFT_CUDA(cudaMallocHost(&ix.stats_pinned, 8 * sizeof(unsigned long long)));
      GIFT_CUDA(cudaMemcpyAsync(ix.stats_pinned, stats, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                stream));
      ix.stats_valid = true;
      tm.finish();
    }
  });
}

gift_status gift_rerank(gift_index* index, const int32_t* cand_ids, const float* cand_scores, int32_t B,
                        int32_t n_cand, int32_t k1, int32_t topk, int32_t* out_ids, float* out_sprime,
                        cudaStream_t stream) {
  return gift::guard("gift_rerank", [&] {
    GIFT_REQUIRE(index && cand_ids && cand_scores && out_ids && out_sprime, "NULL argument");
    Index& ix = *reinterpret_cast<Index*>(index);
    if (!ix.ready()) gift::fail(GIFT_ESTATE, "the streamed build of this index is not complete");
    if (!ix.sif_off) gift::fail(GIFT_EUNSUPPORTED, "index built without an S-IF (sif_k1 == 0)");
    GIFT_REQUIRE(B > 0 && n_cand > 0 && k1 > 0 && k1 <= n_cand, "need 0 < k1 <= n_cand and B > 0");
    GIFT_REQUIRE(topk > 0 && topk <= 1024, "topk must be in [1, 1024]");
    gift::Scratch sc(stream);
    gift::StageTimer tm(&ix, stream);
    std::vector<gift::OutBuf> outs;
    tm.mark(gift::ST_RERANK);
    const int32_t* ci = gift::stage_in(cand_ids, (size_t)B * n_cand, sc, stream);
    const float* cs = gift::stage_in(cand_scores, (size_t)B * n_cand, sc, stream);
    int32_t* oid = gift::stage_out(out_ids, (size_t)B * topk, sc, outs);
    float* osp = gift::stage_out(out_sprime, (size_t)B * topk, sc, outs);
    gift::sif_rerank(ix, ci, cs, B, n_cand, k1, topk, oid, osp, sc, stream);
    gift::flush_out(outs, stream);
    ix.stats_valid = false;
    tm.finish();
  });
}

gift_status gift_render_views(const float* vertices, const int32_t* triangles, const int64_t* vert_off,
                             const int64_t* tri_off, int32_t M, int32_t n_az, int32_t n_el, int32_t H, int32_t W,
                             float* depth, cudaStream_t stream) {
  return gift::guard("gift_render_views", [&] {
    GIFT_REQUIRE(vertices && triangles && vert_off && tri_off && depth, "NULL argument");
    GIFT_REQUIRE(M >= 1 && n_az >= 1 && n_el >= 1 && n_az * n_el <= 4096, "need M >= 1 and 1 <= N_v <= 4096");
    GIFT_REQUIRE(H >= 1 && W >= 1 && H <= 4096 && W <= 4096, "image sides must be in [1, 4096]");
    std::vector<int64_t> vo(vert_off, vert_off + M + 1), to(tri_off, tri_off + M + 1);
    GIFT_REQUIRE(vo[0] == 0 && to[0] == 0, "offsets must start at 0");
    for (int m = 0; m < M; ++m)
      GIFT_REQUIRE(vo[m + 1] >= vo[m] && to[m + 1] >= to[m], "offsets must not decrease");
    GIFT_REQUIRE(vo[M] < (int64_t)INT32_MAX && to[M] * (int64_t)n_az * n_el < ((int64_t)1 << 40),
                 "too many vertices or triangle views");
    gift::Scratch sc(stream);
    std::vector<gift::OutBuf> outs;
    const float* V = gift::stage_in(vertices, (size_t)vo[M] * 3, sc, stream);
    const int32_t* T = gift::stage_in(triangles, (size_t)to[M] * 3, sc, stream);
    float* out = gift::stage_out(depth, (size_t)M * n_az * n_el * H * W, sc, outs);
    gift::render_views(V, T, vo, to, M, n_az, n_el, H, W, out, sc, stream);
    gift::flush_out(outs, stream);
  });
}

gift_status gift_kmeans(const float* X, int64_t n, int32_t D, int32_t K, const int32_t* init_rows, int32_t iters,
                        float* codebook, cudaStream_t stream) {
  return gift::guard("gift_kmeans", [&] {
    GIFT_REQUIRE(X && init_rows && codebook, "NULL argument");
    GIFT_REQUIRE(D > 0 && D % 16 == 0, "D must be a positive multiple of 16");
    GIFT_REQUIRE(K >= 1 && n >= K && n < (int64_t)INT32_MAX, "need 1 <= K <= n < 2^31");
    GIFT_REQUIRE(iters >= 0, "iters must be >= 0");
    std::vector<int32_t> init(init_rows, init_rows + K);
    for (int32_t r : init) GIFT_REQUIRE(r >= 0 && r < n, "an initial row is out of range");
    gift::Scratch sc(stream);
    const float* x = gift::stage_in(X, (size_t)n * D, sc, stream);
    gift::kmeans(x, n, D, K, init, iters, codebook, sc, stream);
  });
}

gift_status gift_aca_build(const gift_index* measure1, const gift_index* measure2, int32_t k2, float alpha,
                           int32_t mode, cudaStream_t stream, gift_aca** out) {
  return gift::guard("gift_aca_build", [&] {
    GIFT_REQUIRE(measure1 && measure2 && out, "NULL argument");
    const Index& a = *reinterpret_cast<const Index*>(measure1);
    const Index& b = *reinterpret_cast<const Index*>(measure2);
    if (!a.ready() || !b.ready()) gift::fail(GIFT_ESTATE, "the streamed build of an index is not complete");
    if (!a.sif_off || !b.sif_off || !a.row_ids || !b.row_ids)
      gift::fail(GIFT_EUNSUPPORTED, "both indices need an S-IF (sif_k1 > 0)");
    if (a.sif_n != a.prm.n_shapes || b.sif_n != b.prm.n_shapes)
      gift::fail(GIFT_EUNSUPPORTED, "two measures need indices whose S-IF covers their own shapes");
    GIFT_REQUIRE(a.prm.n_shapes == b.prm.n_shapes, "the two indices must hold the same number of shapes");
    GIFT_REQUIRE(a.k1 == b.k1, "the two indices must have the same k1");
    GIFT_REQUIRE(mode >= GIFT_ACA_NONE && mode <= GIFT_ACA_CO_AUGMENT, "unknown mode");
    GIFT_REQUIRE(alpha > 0.f && alpha <= 16.f, "alpha must be in (0, 16]");
    GIFT_REQUIRE(mode == GIFT_ACA_NONE || (k2 >= 1 && k2 <= a.k1 && k2 * a.k1 <= 2048),
                 "need 1 <= k2 <= k1 and k2 * k1 <= 2048");
    GIFT_REQUIRE(mode != GIFT_ACA_NONE || a.k1 <= 1024, "k1 must be <= 1024");
    int dev = 0;
    GIFT_CUDA(cudaGetDevice(&dev));
    std::unique_ptr<gift::Aca> x(new gift::Aca());
    x->m[0] = &a;
    x->m[1] = &b;
    x->N = a.prm.n_shapes;
    x->k1 = a.k1;
    x->k2 = mode == GIFT_ACA_NONE ? 1 : k2;
    x->mode = mode;
    x->alpha = alpha;
    x->device = dev;
    gift::Scratch sc(stream);
    gift::aca_build(*x, sc, stream);
    *out = reinterpret_cast<gift_aca*>(x.release());
  });
}

gift_status gift_aca_rerank(gift_aca* aca, const int32_t* cand_ids1, const float* cand_scores1,
                            const int32_t* cand_ids2, const float* cand_scores2, int32_t B, int32_t n_cand,
                            int32_t topk, int32_t* out_ids, float* out_sprime, cudaStream_t stream) {
  return gift::guard("gift_aca_rerank", [&] {
    GIFT_REQUIRE(aca && cand_ids1 && cand_scores1 && cand_ids2 && cand_scores2 && out_ids && out_sprime,
                 "NULL argument");
    const gift::Aca& x = *reinterpret_cast<const gift::Aca*>(aca);
    GIFT_REQUIRE(B > 0 && n_cand >= x.k1, "need B > 0 and n_cand >= k1");
    GIFT_REQUIRE(topk > 0 && topk <= 1024, "topk must be in [1, 1024]");
    gift::Scratch sc(stream);
    std::vector<gift::OutBuf> outs;
    const size_t nc = (size_t)B * n_cand;
    const int32_t* c1 = gift::stage_in(cand_ids1, nc, sc, stream);
    const float* s1 = gift::stage_in(cand_scores1, nc, sc, stream);
    const int32_t* c2 = gift::stage_in(cand_ids2, nc, sc, stream);
    const float* s2 = gift::stage_in(cand_scores2, nc, sc, stream);
    int32_t* oid = gift::stage_out(out_ids, (size_t)B * topk, sc, outs);
    float* osp = gift::stage_out(out_sprime, (size_t)B * topk, sc, outs);
    gift::aca_rerank(x, c1, s1, c2, s2, B, n_cand, topk, oid, osp, sc, stream);
    gift::flush_out(outs, stream);
  });
}

gift_status gift_aca_pairs(const gift_aca* aca, int64_t* pairs) {
  return gift::guard("gift_aca_pairs", [&] {
    GIFT_REQUIRE(aca && pairs, "NULL argument");
    *pairs = reinterpret_cast<const gift::Aca*>(aca)->pairs;
  });
}

gift_status gift_aca_export(const gift_aca* aca, int64_t* entry_offsets, int32_t* entry_ids,
                            uint32_t* entry_members, uint64_t* card, cudaStream_t stream) {
  return gift::guard("gift_aca_export", [&] {
    GIFT_REQUIRE(aca, "NULL argument");
    const gift::Aca& x = *reinterpret_cast<const gift::Aca*>(aca);
    if (entry_offsets)
      GIFT_CUDA(cudaMemcpyAsync(entry_offsets, x.off, ((size_t)x.N + 1) * 8, cudaMemcpyDefault, stream));
    if (entry_ids && x.pairs)
      GIFT_CUDA(cudaMemcpyAsync(entry_ids, x.ids, (size_t)x.pairs * 4, cudaMemcpyDefault, stream));
    if (entry_members && x.pairs)
      GIFT_CUDA(cudaMemcpyAsync(entry_members, x.mem, (size_t)x.pairs * 4, cudaMemcpyDefault, stream));
    if (card) GIFT_CUDA(cudaMemcpyAsync(card, x.card, (size_t)x.N * 8, cudaMemcpyDefault, stream));
    GIFT_CUDA(cudaStreamSynchronize(stream));
  });
}

void gift_aca_destroy(gift_aca* aca) {
  if (!aca) return;
  cudaDeviceSynchronize();
  delete reinterpret_cast<gift::Aca*>(aca);
}

gift_status gift_assign(gift_index* index, const float* feats, int64_t n, int32_t ma, int32_t* out_codes,
                        cudaStream_t stream) {
  return gift::guard("gift_assign", [&] {
    GIFT_REQUIRE(index && feats && out_codes, "NULL argument");
    GIFT_REQUIRE(n >= 0, "n must be >= 0");
    Index& ix = *reinterpret_cast<Index*>(index);
    gift::Scratch sc(stream);
    gift::assign_codes(ix, feats, n, ma, out_codes, sc, stream);
  });
}

gift_status gift_export_fif(const gift_index* index, int32_t* db_codes, int64_t* list_offsets, int32_t* list_rows,
                            cudaStream_t stream) {
  return gift::guard("gift_export_fif", [&] {
    GIFT_REQUIRE(index, "NULL index");
    const Index& ix = *reinterpret_cast<const Index*>(index);
    if (!ix.list_off) gift::fail(GIFT_ESTATE, "the F-IF lists of this index are not built yet");
    if (db_codes)
      GIFT_CUDA(cudaMemcpyAsync(db_codes, ix.db_codes, ix.n_entries * 4, cudaMemcpyDefault, stream));
    if (list_offsets)
      GIFT_CUDA(cudaMemcpyAsync(list_offsets, ix.list_off, (ix.prm.n_codewords + 1) * 8, cudaMemcpyDefault, stream));
    if (list_rows)
      GIFT_CUDA(cudaMemcpyAsync(list_rows, ix.list_row, ix.n_entries * 4, cudaMemcpyDefault, stream));
    GIFT_CUDA(cudaStreamSynchronize(stream));
  });
}

gift_status gift_sif_from_neighbours(gift_index* index, const int32_t* nbr_ids, const float* nbr_scores,
                                     int32_t n_shapes_total, int32_t k1, cudaStream_t stream) {
  return gift::guard("gift_sif_from_neighbours", [&] {
    GIFT_REQUIRE(index && nbr_ids && nbr_scores, "NULL argument");
    Index& ix = *reinterpret_cast<Index*>(index);
    if (!ix.ready()) gift::fail(GIFT_ESTATE, "the streamed build of this index is not complete");
    if (ix.sif_off) gift::fail(GIFT_ESTATE, "the index already has an S-IF");
    GIFT_REQUIRE(n_shapes_total >= 1, "n_shapes_total must be positive");
    GIFT_REQUIRE(k1 >= 1 && k1 <= std::min(1024, n_shapes_total), "k1 must be in [1, min(1024, n_shapes_total)]");
    int dev = 0;
    GIFT_CUDA(cudaGetDevice(&dev));
    GIFT_REQUIRE(dev == ix.device, "call with the index's device current");
    gift::Scratch sc(stream);
    const int64_t n = (int64_t)n_shapes_total * k1;
    const int32_t* ids = gift::stage_in(nbr_ids, (size_t)n, sc, stream);
    const float* scs = gift::stage_in(nbr_scores, (size_t)n, sc, stream);
    ix.row_ids = ix.alloc<int32_t>(n);
    ix.row_sc = ix.alloc<float>(n);
    GIFT_CUDA(cudaMemcpyAsync(ix.row_ids, ids, n * 4, cudaMemcpyDeviceToDevice, stream));
    GIFT_CUDA(cudaMemcpyAsync(ix.row_sc, scs, n * 4, cudaMemcpyDeviceToDevice, stream));
    int64_t* off = ix.alloc<int64_t>((size_t)n_shapes_total + 1);
    int32_t* sids = ix.alloc<int32_t>(n);
    uint32_t* mem = ix.alloc<uint32_t>(n);
    uint64_t* card = ix.alloc<uint64_t>(n_shapes_total);
    ix.k1 = k1;
    ix.sif_n = n_shapes_total;
    ix.sif_ids = sids;
    ix.sif_mem = mem;
    ix.sif_card = card;
    ix.sif_off = off;
    try {
      gift::sif_build(ix, ix.row_ids, ix.row_sc, sc, stream);
    } catch (...) {
      ix.sif_off = nullptr;  // no half-built S-IF is visible to later calls
      throw;
    }
  });
}

gift_status gift_merge_topk(const int32_t* ids, const float* scores, int32_t B, int64_t n, int32_t k,
                            int32_t* out_ids, float* out_scores, cudaStream_t stream) {
  return gift::guard("gift_merge_topk", [&] {
    GIFT_REQUIRE(ids && scores && out_ids && out_scores, "NULL argument");
    GIFT_REQUIRE(B > 0 && n > 0 && n < (int64_t)INT32_MAX, "need B > 0 and 0 < n < 2^31");
    GIFT_REQUIRE(k > 0 && k <= 1024, "k must be in [1, 1024]");
    gift::Scratch sc(stream);
    std::vector<gift::OutBuf> outs;
    const int32_t* ci = gift::stage_in(ids, (size_t)B * n, sc, stream);
    const float* cs = gift::stage_in(scores, (size_t)B * n, sc, stream);
    int32_t* oid = gift::stage_out(out_ids, (size_t)B * k, sc, outs);
    float* osc = gift::stage_out(out_scores, (size_t)B * k, sc, outs);
    gift::merge_topk_rows(ci, cs, B, n, k, oid, osc, sc, stream);
    gift::flush_out(outs, stream);
  });
}

gift_status gift_export_sif(const gift_index* index, int64_t* entry_offsets, int32_t* entry_ids,
                            uint32_t* entry_members, uint64_t* card, cudaStream_t stream) {
  return gift::guard("gift_export_sif", [&] {
    GIFT_REQUIRE(index, "NULL index");
    const Index& ix = *reinterpret_cast<const Index*>(index);
    if (!ix.sif_off) gift::fail(GIFT_EUNSUPPORTED, "index built without an S-IF");
    const int64_t N = ix.sif_n, n = N * ix.k1;
    if (entry_offsets)
      GIFT_CUDA(cudaMemcpyAsync(entry_offsets, ix.sif_off, (N + 1) * 8, cudaMemcpyDefault, stream));
    if (entry_ids) GIFT_CUDA(cudaMemcpyAsync(entry_ids, ix.sif_ids, n * 4, cudaMemcpyDefault, stream));
    if (entry_members) GIFT_CUDA(cudaMemcpyAsync(entry_members, ix.sif_mem, n * 4, cudaMemcpyDefault, stream));
    if (card) GIFT_CUDA(cudaMemcpyAsync(card, ix.sif_card, N * 8, cudaMemcpyDefault, stream));
    GIFT_CUDA(cudaStreamSynchronize(stream));
  });
}

gift_status gift_index_info(const gift_index* index, gift_index_info_t* out) {
  return gift::guard("gift_index_info", [&] {
    GIFT_REQUIRE(index && out, "NULL argument");
    const Index& ix = *reinterpret_cast<const Index*>(index);
    out->device_bytes = ix.device_bytes;
    out->n_rows = ix.n_rows;
    out->n_entries = ix.n_entries;
    out->n_lists_nonempty = ix.n_nonempty;
    out->max_list_len = ix.max_list;
    out->n_runs = ix.n_runs;
    out->max_runs = ix.max_runs;
    out->max_sif_entry = ix.max_sif_entry;
    out->sif_shapes = ix.sif_off ? ix.sif_n : 0;
    out->sif_k1 = ix.sif_off ? ix.k1 : 0;
  });
}

gift_status gift_set_rescore_depth(gift_index* index, int32_t rescore_r) {
  return gift::guard("gift_set_rescore_depth", [&] {
    GIFT_REQUIRE(index, "NULL index");
    Index& ix = *reinterpret_cast<Index*>(index);
    if (!ix.ready()) gift::fail(GIFT_ESTATE, "the streamed build of this index is not complete");
    GIFT_REQUIRE(rescore_r >= 0 && rescore_r <= 1024, "rescore_r must be in [0, 1024]");
    if (rescore_r > 0 && !ix.list_lo && !ix.master)
      gift::fail(GIFT_EUNSUPPORTED, "the index was built without a rescore store (rescore_r == 0)");
    ix.prm.rescore_r = rescore_r;
  });
}

gift_status gift_set_timing(gift_index* index, int32_t enable) {
  return gift::guard("gift_set_timing", [&] {
    GIFT_REQUIRE(index, "NULL index");
    reinterpret_cast<Index*>(index)->timing = enable != 0;
  });
}

gift_status gift_get_timing(gift_index* index, gift_timing_t* out) {
  return gift::guard("gift_get_timing", [&] {
    GIFT_REQUIRE(index && out, "NULL argument");
    Index& ix = *reinterpret_cast<Index*>(index);
    if (ix.ev.empty()) gift::fail(GIFT_ESTATE, "no timed call recorded");
    GIFT_CUDA(cudaEventSynchronize(ix.ev.back()));
    gift_timing_t t{};
    float* slot[gift::ST_END] = {&t.assign_ms, &t.bucket_ms, &t.scan_ms, &t.combine_ms,
                                 &t.topk_ms,   &t.rescore_ms, &t.rerank_ms};
    for (size_t i = 0; i + 1 < ix.ev.size(); ++i) {
      float ms = 0.f;
      GIFT_CUDA(cudaEventElapsedTime(&ms, ix.ev[i], ix.ev[i + 1]));
      const int st = ix.ev_stage[i];
      if (st >= 0 && st < gift::ST_END) *slot[st] += ms;
    }
    GIFT_CUDA(cudaEventElapsedTime(&t.total_ms, ix.ev.front(), ix.ev.back()));
    for (auto& k : ix.kspans) {
      float ms = 0.f;
      GIFT_CUDA(cudaEventElapsedTime(&ms, k.second.first, k.second.second));
      if (k.first == 0) t.assign_kernel_ms += ms;
      if (k.first == 1) t.scan_kernel_ms += ms;
      if (k.first == 2) t.rescore_kernel_ms += ms;
    }
    t.assign_rows = ix.k_assign_rows;
    if (ix.stats_pinned && ix.stats_valid) {
      t.scan_bytes = (int64_t)ix.stats_pinned[0];
      t.scan_pairs = (int64_t)ix.stats_pinned[1];
      t.rescore_bytes = ix.prm.rescore_r > 0 ? (int64_t)ix.stats_pinned[2] : 0;
      t.rescore_items = (int64_t)ix.stats_pinned[3];
      t.rescore_items_kept = (int64_t)ix.stats_pinned[4];
      t.cand_pairs = (int64_t)ix.stats_pinned[5];
      t.cand_rows = (int64_t)ix.stats_pinned[6];
      t.rescore_rows_read = (int64_t)ix.stats_pinned[7];
    }
    *out = t;
  });
}

gift_status gift_match_forward(const void* q, const int32_t* q_view_offsets, int32_t Bq, const void* p, int32_t Np,
                               int32_t nv_p, const void* W, int32_t d_in, int32_t d_out, int32_t dtype, float* S,
                               int16_t* argmax, cudaStream_t stream) {
  return gift::guard("gift_match_forward", [&] {
    GIFT_REQUIRE(q && p && S && argmax, "NULL argument");
    GIFT_REQUIRE(Bq > 0 && Np > 0 && nv_p > 0 && nv_p <= 32767, "bad sizes");
    GIFT_REQUIRE(d_in > 0 && d_in % 16 == 0 && d_out > 0 && d_out % 16 == 0, "dims must be multiples of 16");
    GIFT_REQUIRE(W || d_in == d_out, "d_out must equal d_in without a projection");
    GIFT_REQUIRE(dtype == GIFT_F32 || dtype == GIFT_BF16, "dtype must be GIFT_F32 or GIFT_BF16");
    std::vector<int32_t> h = gift::host_offsets(q_view_offsets, Bq);
    gift::Scratch sc(stream);
    gift::match_forward(q, h, Bq, p, Np, nv_p, W, d_in, d_out, dtype, S, argmax, sc, stream);
  });
}

gift_status gift_match_backward(const void* q, const int32_t* q_view_offsets, int32_t Bq, const void* p, int32_t Np,
                                int32_t nv_p, const void* W, int32_t d_in, int32_t d_out, int32_t dtype,
                                const float* grad_S, const int16_t* argmax, float* dW, float* dQ, float* dP,
                                cudaStream_t stream) {
  return gift::guard("gift_match_backward", [&] {
    GIFT_REQUIRE(q && p && grad_S && argmax, "NULL argument");
    GIFT_REQUIRE(Bq > 0 && Np > 0 && nv_p > 0 && nv_p <= 32767, "bad sizes");
    GIFT_REQUIRE(d_in > 0 && d_in % 16 == 0 && d_out > 0 && d_out % 16 == 0, "dims must be multiples of 16");
    GIFT_REQUIRE(W || d_in == d_out, "d_out must equal d_in without a projection");
    GIFT_REQUIRE(W || !dW, "dW needs a projection");
    GIFT_REQUIRE(d_out <= 1024, "d_out must be at most 1024 for the backward");
    GIFT_REQUIRE(dtype == GIFT_F32 || dtype == GIFT_BF16, "dtype must be GIFT_F32 or GIFT_BF16");
    std::vector<int32_t> h = gift::host_offsets(q_view_offsets, Bq);
    gift::Scratch sc(stream);
    gift::match_backward(q, h, Bq, p, Np, nv_p, W, d_in, d_out, dtype, grad_S, argmax, dW, dQ, dP, sc, stream);
  });
}

const char* gift_last_error(void) { return gift::g_last_error.c_str(); }

int32_t gift_version(void) { return 101; }

int64_t gift_launch_count(void) { return gift::g_launches.load(); }

}  // extern "C"
