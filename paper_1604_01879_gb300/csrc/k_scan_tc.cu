// Posting-list scan and candidate rescore on the 5th-generation tensor cores
// (Eq. 4, Fig. 2), as policies of the tcgen05 engine.
//
// Work item: (list k, a tile of consecutive entries of list k, 128
// consecutive query slots of bucket k). Rows of the MMA (TMEM lanes) are
// query slots, columns are list entries; list entries of one shape are
// consecutive, so each epilogue thread walks its row of columns in order,
// keeps the max cosine of the current shape run and folds every run maximum
// into the per-(slot, run) table with atomicMax on its order-preserving key
// (f2key, so negative cosines keep their order; 0 = not written).
//
// (Lists touched by at most 80 slots of a batch swap the roles: entries are the
// MMA rows and slots the columns, see the slot-column policies below.)
//
// Scan: BF16 or E4M3 store, one product per k-block, 256 entries per tile.
// Rescore: two-part BF16 operands (x = hi + lo) and three products, the
// reduction split in four chunks accumulated in separate TMEM buffers and
// summed in FP32 by the epilogue; only runs of the query's top-R candidate
// shapes are kept, and only work items that hold such a run are run (a
// pre-pass lists them): the FP32-level rescore needs the rows of its
// candidates' runs, not every row of a touched list. For a BF16 store whose
// rows are the hi parts of the two-part store, the same policy runs over every
// touched pair with every run written: the scan itself is FP32-level.
#include <type_traits>

#include "fif_plan.cuh"
#include "gift_internal.cuh"
#include "tc_engine.cuh"

namespace gift {

namespace {

constexpr int kScanTN = 256;
constexpr int kRescTN = 128;
constexpr int kRescChunks = 4;

struct ListItem {
  int64_t e0, s0;
  int ne, ns, k;
};

struct ListSched {
  const int64_t* woff;      // [K+1] work items per list (exclusive), woff[K] = total
  int K;
  const int64_t* boff;      // [K+1] slots per codeword
  const int64_t* list_off;  // [K+1]
  int nkb;
  __device__ __forceinline__ int64_t total_items() const { return woff[K]; }
  // TN entries x TS slots per item
  template <int TN, int TS = tc::kTM>
  __device__ __forceinline__ ListItem decode_list(int64_t item) const {
    int lo = 0, hi = K;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (woff[mid] <= item) lo = mid; else hi = mid;
    }
    const int k = lo;
    const int64_t L = list_off[k + 1] - list_off[k];
    const int64_t M = boff[k + 1] - boff[k];
    const int64_t nts = cdiv(M, (int64_t)TS);
    const int64_t local = item - woff[k];
    const int64_t te = local / nts, ts = local % nts;
    ListItem it;
    it.k = k;
    it.e0 = list_off[k] + te * TN;
    it.ne = (int)min((int64_t)TN, L - te * TN);
    it.s0 = boff[k] + ts * TS;
    it.ns = (int)min((int64_t)TS, M - ts * TS);
    return it;
  }
};

struct SlotInfo {
  const int64_t* runbase;    // [nslots]
  const int32_t* slot_view;  // [nslots]
  const int32_t* vquery;     // [nv]
  const float* q_inv;        // [nv]
  const float* scale;        // [n_rows] list-ordered cosine factor
  const int32_t* entry_run;  // [n_rows]
  const int32_t* list_shape; // [n_rows]
  const float* slot_scale;   // [nslots] E4M3 slot scale, or null (BF16 slots)
  uint32_t* table;
};

__device__ __forceinline__ bool is_candidate(const int32_t* c, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (c[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo < n && c[lo] == key;
}

struct RowCtx {
  int64_t rb;
  float qi;
  int32_t qq;
  bool valid;
};

// per-warp shared copy of the tile's entry metadata
template <int TN>
__device__ __forceinline__ void load_entry_meta(const SlotInfo& si, const ListItem& it, uint8_t* ws) {
  int* e_run = reinterpret_cast<int*>(ws);
  float* e_scale = reinterpret_cast<float*>(e_run + TN);
  int* e_shape = e_run + 2 * TN;
  const int lane = threadIdx.x & 31;
  for (int c = lane; c < TN; c += 32) {
    if (c < it.ne) {
      const int64_t e = it.e0 + c;
      e_run[c] = si.entry_run[e];
      e_scale[c] = si.scale[e];
      e_shape[c] = si.list_shape[e];
    } else {
      e_run[c] = -1;
      e_scale[c] = 0.f;
      e_shape[c] = 0;
    }
  }
}

__device__ __forceinline__ void load_row(const SlotInfo& si, const ListItem& it, int m, RowCtx& r) {
  r.valid = m < it.ns;
  r.rb = 0;
  r.qi = 0.f;
  r.qq = 0;
  if (r.valid) {
    const int64_t s = it.s0 + m;
    r.rb = si.runbase[s];
    const int32_t v = si.slot_view[s];
    r.qi = si.q_inv[v] * (si.slot_scale ? si.slot_scale[s] : 1.f);
    r.qq = si.vquery[v];
  }
}

// ---------------------------------------------------------------- scan policy
// EB_ = 2: BF16 store and slots; EB_ = 1: E4M3 store and slots (per-row scales)
template <int EB_>
struct ScanPolicy : ListSched {
  static constexpr int TN = kScanTN, NBUF = 2, STAGES = 4, SPLIT = 1, EB = EB_;
  static constexpr int kWarpSmem = TN * 12;
  SlotInfo si;
  using Item = ListItem;
  struct Ctx {
    RowCtx row;
    int cur_run;
    float cur_max;
  };
  __device__ __forceinline__ int64_t total() const { return total_items(); }
  __device__ __forceinline__ Item decode(int64_t item) const { return decode_list<TN>(item); }
  __device__ __forceinline__ int nchunks(const Item&) const { return 1; }
  __device__ __forceinline__ void chunk(const Item& it, int, int& br, int& kb0, int& kb1) const {
    br = (int)it.e0;
    kb0 = 0;
    kb1 = nkb;
  }
  __device__ __forceinline__ int a_row(const Item& it) const { return (int)it.s0; }
  __device__ __forceinline__ void epi_begin(const Item& it, Ctx& x, int m, int, uint8_t* ws) const {
    load_entry_meta<TN>(si, it, ws);
    load_row(si, it, m, x.row);
    x.cur_run = -1;
    x.cur_max = 0.f;
  }
  __device__ __forceinline__ void flush(const Ctx& x) const {
    if (x.row.valid && x.cur_run >= 0) atomicMax(si.table + x.row.rb + x.cur_run, f2key(x.cur_max));
  }
  __device__ __forceinline__ void epi_chunk(const Item& it, int, uint32_t taddr, Ctx& x, int, uint8_t* ws) const {
    const int* e_run = reinterpret_cast<const int*>(ws);
    const float* e_scale = reinterpret_cast<const float*>(e_run + TN);
    const int npieces = (it.ne + 31) >> 5;
    for (int pc = 0; pc < npieces; ++pc) {
      uint32_t r[32];
      tc::tmem_ld32(taddr + pc * 32, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = pc * 32 + j;
        const int run = e_run[c];
        const float v = __uint_as_float(r[j]) * x.row.qi * e_scale[c];
        if (run != x.cur_run) {
          flush(x);
          x.cur_run = run;
          x.cur_max = v;
        } else {
          x.cur_max = fmaxf(x.cur_max, v);
        }
      }
    }
  }
  __device__ __forceinline__ void epi_end(const Item&, Ctx& x, int, uint8_t*) const { flush(x); }
};

// ---------------------------------------------------------------- rescore policy
struct RescorePolicy : ListSched {
  static constexpr int TN = kRescTN, NBUF = 4, STAGES = 3, SPLIT = 3, EB = 2;
  static constexpr int kWarpSmem = TN * 12;
  SlotInfo si;
  const int32_t* cand;      // [B, R] candidate ids sorted ascending
  int R;
  const int64_t* item_map;  // [n_items] the work items holding a candidate run (ascending); null: every item,
  const int64_t* n_items;   // every run written (the FP32-level scan of a BF16 store with its two-part rows)
  using Item = ListItem;
  struct Ctx {
    RowCtx row;
    float sum[TN];
  };
  __device__ __forceinline__ int64_t total() const { return item_map ? *n_items : total_items(); }
  __device__ __forceinline__ Item decode(int64_t item) const {
    return decode_list<TN>(item_map ? item_map[item] : item);
  }
  // never an empty chunk: each chunk must write its own accumulator
  // chunks bound the MMA steps feeding one accumulator (about 192, 3 products
  // x 4 sub-steps per k-block); short reductions use one chunk
  __device__ __forceinline__ int nch() const {
    const int want = (nkb * 12 + 191) / 192;
    return want < 1 ? 1 : (want > kRescChunks ? kRescChunks : want);
  }
  __device__ __forceinline__ int nchunks(const Item&) const { return nch(); }
  __device__ __forceinline__ void chunk(const Item& it, int c, int& br, int& kb0, int& kb1) const {
    br = (int)it.e0;
    const int nch = this->nch();
    kb0 = (int)((int64_t)nkb * c / nch);
    kb1 = (int)((int64_t)nkb * (c + 1) / nch);
  }
  __device__ __forceinline__ int a_row(const Item& it) const { return (int)it.s0; }
  __device__ __forceinline__ void epi_begin(const Item& it, Ctx& x, int m, int, uint8_t* ws) const {
    load_entry_meta<TN>(si, it, ws);
    load_row(si, it, m, x.row);
#pragma unroll
    for (int j = 0; j < TN; ++j) x.sum[j] = 0.f;
  }
  __device__ __forceinline__ void epi_chunk(const Item&, int c, uint32_t taddr, Ctx& x, int, uint8_t*) const {
#pragma unroll
    for (int pc = 0; pc < TN / 32; ++pc) {
      uint32_t r[32];
      tc::tmem_ld32(taddr + pc * 32, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 32; ++j) x.sum[pc * 32 + j] += __uint_as_float(r[j]);
    }
    (void)c;
  }
  __device__ __forceinline__ void epi_end(const Item& it, Ctx& x, int, uint8_t* ws) const {
    const int* e_run = reinterpret_cast<const int*>(ws);
    const float* e_scale = reinterpret_cast<const float*>(e_run + TN);
    const int* e_shape = e_run + 2 * TN;
    if (!x.row.valid) return;
    const int32_t* cq = cand ? cand + (int64_t)x.row.qq * R : nullptr;
    int cur_run = -1, cur_shape = 0;
    float cur_max = 0.f;
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const int run = e_run[c];
      const float v = x.sum[c] * x.row.qi * e_scale[c];
      if (run != cur_run) {
        if (cur_run >= 0 && (!cand || is_candidate(cq, R, cur_shape)))
          atomicMax(si.table + x.row.rb + cur_run, f2key(cur_max));
        cur_run = run;
        cur_max = v;
        cur_shape = e_shape[c];
      } else {
        cur_max = fmaxf(cur_max, v);
      }
    }
    if (cur_run >= 0 && (!cand || is_candidate(cq, R, cur_shape)))
      atomicMax(si.table + x.row.rb + cur_run, f2key(cur_max));
    (void)it;
  }
};

// ---------------------------------------------------------------- slot-column policies
// Most lists are touched by few query slots of a batch (a few to a few dozen,
// from the queries whose views share its codeword). For lists of up to 80
// slots these policies make the list entries the 128 MMA rows (A, TMEM lanes)
// and the slots the N columns (B), N = TS in {16, 32, 64, 80}, the smallest
// that holds the list's slots. The small slot tile leaves most of shared memory
// to the entry tiles, so more of them are in flight from DRAM (4 to 11 stages
// instead of 3 or 4), and the MMAs shrink with N. Each launch runs the lists
// of one slot class; lists of more slots keep the slot-row policies above.
//
// Epilogue: thread = entry row; it accumulates its TS slot columns, then per
// slot the warp takes the segmented max over its lanes by run (entries of one
// shape are consecutive, so a run is a contiguous group of lanes) with five
// shuffles, and the first lane of each run folds it into the per-(slot, run)
// table with atomicMax on the order-preserving key. A run split between warps
// or tiles is merged by the atomics. The rescore writes every run of its
// items: the candidate sums read the table only at candidate shapes.
//
// EB = 1, SPLIT = 1: E4M3 scan (per-slot and per-entry scales, one chunk).
// EB = 2, SPLIT = 3: FP32-level rescore with two-part BF16 operands, the
// reduction in kRescChunks chunks summed in FP32 (as RescorePolicy).
__host__ __device__ constexpr int slot_class(int64_t M) {
  return M <= 16 ? 16 : M <= 32 ? 32 : M <= 64 ? 64 : M <= 80 ? 80 : 128;
}

template <int EB_, int SPLIT_, int TS_>
struct SlotsPolicy : ListSched {
  static constexpr int TN = TS_, EB = EB_, SPLIT = SPLIT_;
  static constexpr bool kResc = SPLIT_ == 3;
  // the slot-row policies' product order (slot hi x entry lo before slot lo x
  // entry hi), so a (slot, entry) value does not depend on the list's class
  static constexpr bool SWAP_CROSS = true;
  static constexpr int NBUF = kResc ? kRescChunks : (TS_ <= 64 ? 4 : 2);
  // stage bytes: entries (A) 16 KB per part, slots (B) TS x 128 bytes per part
  static constexpr int kStage = (kResc ? 2 : 1) * (16384 + TS_ * 128);
  static constexpr int kWarpSmem = TS_ * 12;
  // as many stages as fit beside the engine's alignment pad, barriers and warp
  // areas in 227 KB, at most 11 (the barrier area): rescore 6, 5, 4, 4; scan
  // 11, 11, 9, 8 (TS = 16, 32, 64, 80)
  static constexpr int kFit = (232448 - 1024 - 256 - 4 * kWarpSmem) / kStage;
  static constexpr int STAGES = kFit > 11 ? 11 : kFit;
  static_assert(TS_ == 16 || TS_ == 32 || TS_ == 64 || TS_ == 80, "slot tile of 16, 32, 64 or 80");
  static_assert(kResc ? EB_ == 2 : (EB_ == 1 && SPLIT_ == 1), "E4M3 scan or two-part BF16 rescore");
  SlotInfo si;
  const int64_t* item_map;  // rescore: [n_items] the kept work items (ascending); scan: null
  const int64_t* n_items;
  using Item = ListItem;
  struct Ctx {
    int run;
    float esc;
    bool valid;
    float sum[TS_];
  };
  __device__ __forceinline__ int64_t total() const { return kResc ? *n_items : total_items(); }
  __device__ __forceinline__ Item decode(int64_t item) const {
    return decode_list<tc::kTM, TS_>(kResc ? item_map[item] : item);
  }
  __device__ __forceinline__ int nch() const {
    if (!kResc) return 1;
    const int want = (nkb * 12 + 191) / 192;
    return want < 1 ? 1 : (want > kRescChunks ? kRescChunks : want);
  }
  __device__ __forceinline__ int nchunks(const Item&) const { return nch(); }
  __device__ __forceinline__ void chunk(const Item& it, int c, int& br, int& kb0, int& kb1) const {
    br = (int)it.s0;
    const int n = nch();
    kb0 = (int)((int64_t)nkb * c / n);
    kb1 = (int)((int64_t)nkb * (c + 1) / n);
  }
  __device__ __forceinline__ int a_row(const Item& it) const { return (int)it.e0; }
  __device__ __forceinline__ void epi_begin(const Item& it, Ctx& x, int m, int, uint8_t* ws) const {
    int64_t* s_rb = reinterpret_cast<int64_t*>(ws);
    float* s_qi = reinterpret_cast<float*>(s_rb + TS_);
    const int lane = threadIdx.x & 31;
    for (int j = lane; j < TS_; j += 32) {
      int64_t rb = 0;
      float qi = 0.f;
      if (j < it.ns) {
        const int64_t s = it.s0 + j;
        rb = si.runbase[s];
        qi = si.q_inv[si.slot_view[s]] * (si.slot_scale ? si.slot_scale[s] : 1.f);
      }
      s_rb[j] = rb;
      s_qi[j] = qi;
    }
    x.valid = m < it.ne;
    const int64_t e = it.e0 + m;
    x.run = x.valid ? si.entry_run[e] : -1 - m;  // rows past the list: a group of their own
    x.esc = x.valid ? si.scale[e] : 0.f;
#pragma unroll
    for (int j = 0; j < TS_; ++j) x.sum[j] = 0.f;
  }
  __device__ __forceinline__ void epi_chunk(const Item&, int, uint32_t taddr, Ctx& x, int, uint8_t*) const {
#pragma unroll
    for (int pc = 0; pc < TS_ / 32; ++pc) {
      uint32_t r[32];
      tc::tmem_ld32(taddr + pc * 32, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 32; ++j) x.sum[pc * 32 + j] += __uint_as_float(r[j]);
    }
    if constexpr (TS_ % 32 == 16) {  // the last 16 columns (TS = 16, 80)
      uint32_t r[16];
      tc::tmem_ld16(taddr + (TS_ / 32) * 32, r);
      tc::tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) x.sum[(TS_ / 32) * 32 + j] += __uint_as_float(r[j]);
    }
  }
  __device__ __forceinline__ void epi_end(const Item& it, Ctx& x, int, uint8_t* ws) const {
    const int64_t* s_rb = reinterpret_cast<const int64_t*>(ws);
    const float* s_qi = reinterpret_cast<const float*>(s_rb + TS_);
    const int lane = threadIdx.x & 31;
    // lane + o holds the same run (the lanes between do too): offsets 1, 2, 4, 8, 16
    unsigned same = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      const int o = 1 << b;
      const int r2 = __shfl_down_sync(0xffffffffu, x.run, o);
      if (lane + o < 32 && r2 == x.run) same |= 1u << b;
    }
    const int up = __shfl_up_sync(0xffffffffu, x.run, 1);
    const bool head = x.valid && (lane == 0 || up != x.run);
    const int64_t tb = head ? (int64_t)x.run : 0;
#pragma unroll
    for (int j = 0; j < TS_; ++j) {
      if (j < it.ns) {  // warp-uniform
        float v = x.sum[j] * s_qi[j] * x.esc;  // the slot-row policies' rounding order
#pragma unroll
        for (int b = 0; b < 5; ++b) {
          const float y = __shfl_down_sync(0xffffffffu, v, 1 << b);
          if (same & (1u << b)) v = fmaxf(v, y);
        }
        if (head) atomicMax(si.table + s_rb[j] + tb, f2key(v));
      }
    }
  }
};

// slot-ordered BF16 copies of the query views: hi = bf16(q), lo = bf16(q - hi)
__global__ void k_slot_split(const float* __restrict__ q, const int32_t* __restrict__ slot_view, int64_t nslots,
                             int D, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t s = blockIdx.x;
  if (s >= nslots) return;
  const float4* src = reinterpret_cast<const float4*>(q + (int64_t)slot_view[s] * D);
  __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(hi + s * D);
  __nv_bfloat162* l2 = lo ? reinterpret_cast<__nv_bfloat162*>(lo + s * D) : nullptr;
  for (int i = threadIdx.x; i < D / 4; i += blockDim.x) {
    const float4 v = src[i];
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
    h2[2 * i] = a;
    h2[2 * i + 1] = b;
    if (l2) {
      const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
      l2[2 * i] = __floats2bfloat162_rn(v.x - fa.x, v.y - fa.y);
      l2[2 * i + 1] = __floats2bfloat162_rn(v.z - fb.x, v.w - fb.y);
    }
  }
}

// slot-ordered E4M3 copies of the query views with one scale per slot:
// stored = q / scale, scale = max|q| / 448 (the largest finite E4M3 value)
__global__ __launch_bounds__(256) void k_slot_fp8(const float* __restrict__ q, const int32_t* __restrict__ slot_view,
                                                  int64_t nslots, int D, __nv_fp8_e4m3* __restrict__ out,
                                                  float* __restrict__ scale) {
  __shared__ float red[8];
  const int64_t s = blockIdx.x;
  if (s >= nslots) return;
  const float* src = q + (int64_t)slot_view[s] * D;
  float m = 0.f;
  for (int i = threadIdx.x; i < D; i += blockDim.x) m = fmaxf(m, fabsf(src[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  float mx = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) mx = fmaxf(mx, red[w]);
  const float sc = mx > 0.f ? mx / 448.f : 1.f;
  const float inv = 1.f / sc;
  for (int i = threadIdx.x; i < D; i += blockDim.x) out[s * D + i] = __nv_fp8_e4m3(src[i] * inv);
  if (threadIdx.x == 0) scale[s] = sc;
}

// Rescore work items that hold a candidate run: item (list k, entry tile,
// slot tile) is kept when some slot of the tile has, among the tile's
// entries, a run whose shape is one of its query's top-R candidates. One warp
// per item tests every (slot, run start) pair; items past the real total (the
// grid covers an upper bound) are not kept. With stats (timed calls only):
//   [3] items, [4] kept items, [5] candidate (slot, entry) pairs, [6] candidate
//   rows (entries whose shape is a candidate of some slot of their list, each
//   list's entries counted once, by its first slot tile), [7] rows of kept items.
template <int TS>
__global__ __launch_bounds__(256) void k_resc_flags(const ListSched ls, const int32_t* __restrict__ slot_view,
                                                    const int32_t* __restrict__ vquery,
                                                    const int32_t* __restrict__ entry_run,
                                                    const int32_t* __restrict__ list_shape,
                                                    const int32_t* __restrict__ cand, int R, int64_t upper,
                                                    int64_t* __restrict__ flags,
                                                    unsigned long long* __restrict__ stats) {
  const int64_t item = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (item >= upper) return;
  if (item >= ls.total_items()) {
    if (lane == 0) flags[item] = 0;
    return;
  }
  const ListItem it = ls.decode_list<kRescTN, TS>(item);
  bool hit = false;
  for (int m = 0; m < it.ns && !hit; ++m) {
    const int32_t* cq = cand + (int64_t)vquery[slot_view[it.s0 + m]] * R;
    for (int c = lane; c < it.ne && !hit; c += 32) {
      const int64_t e = it.e0 + c;
      if ((c == 0 || entry_run[e] != entry_run[e - 1]) && is_candidate(cq, R, list_shape[e])) hit = true;
    }
    hit = __any_sync(0xffffffffu, hit);
  }
  if (lane == 0) flags[item] = hit ? 1 : 0;
  if (!stats) return;
  unsigned long long pairs = 0, rows = 0;
  for (int m = 0; m < it.ns; ++m) {
    const int32_t* cq = cand + (int64_t)vquery[slot_view[it.s0 + m]] * R;
    for (int c = lane; c < it.ne; c += 32) pairs += is_candidate(cq, R, list_shape[it.e0 + c]) ? 1 : 0;
  }
  if (it.s0 == ls.boff[it.k]) {  // the list's first slot tile counts its candidate rows
    const int64_t b0 = ls.boff[it.k], b1 = ls.boff[it.k + 1];
    for (int c = lane; c < it.ne; c += 32) {
      const int32_t shape = list_shape[it.e0 + c];
      bool any = false;
      for (int64_t s = b0; s < b1 && !any; ++s) any = is_candidate(cand + (int64_t)vquery[slot_view[s]] * R, R, shape);
      rows += any ? 1 : 0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    rows += __shfl_xor_sync(0xffffffffu, rows, o);
  }
  if (lane == 0) {
    atomicAdd(&stats[3], 1ull);
    atomicAdd(&stats[4], hit ? 1ull : 0ull);
    atomicAdd(&stats[5], pairs);
    atomicAdd(&stats[6], rows);
    atomicAdd(&stats[7], hit ? (unsigned long long)it.ne : 0ull);
  }
}

// item_map[pos[i]] = i for every kept item i < upper; *n_items = the count
__global__ void k_compact_items(const int64_t* __restrict__ flags, const int64_t* __restrict__ pos, int64_t upper,
                                int64_t* __restrict__ item_map, int64_t* __restrict__ n_items) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= upper) return;
  if (flags[i]) item_map[pos[i]] = i;
  if (i == upper - 1) *n_items = pos[i] + flags[i];
}

// ts_class > 0: only the lists of that slot class (slot tiles of ts_class slots);
// otherwise every touched list, slot tiles of 128
__global__ void k_work_count_tc(const int64_t* __restrict__ boff, const int64_t* __restrict__ list_off, int K,
                                int tn, int ts_class, int64_t* __restrict__ wcnt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > K) return;
  if (k == K) {
    wcnt[K] = 0;
    return;
  }
  const int64_t M = boff[k + 1] - boff[k];
  const int64_t L = list_off[k + 1] - list_off[k];
  const int ts = ts_class > 0 ? ts_class : tc::kTM;
  const bool mine = ts_class <= 0 || slot_class(M) == ts_class;
  wcnt[k] = (M > 0 && L > 0 && mine) ? cdiv(L, (int64_t)tn) * cdiv(M, (int64_t)ts) : 0;
}

// work items (list, entry tile of tn entries, slot tile) of the batch's touched lists
ListSched list_sched(const Index& ix, const FifPlan& P, int tn, Scratch& sc, cudaStream_t s, int ts_class = 0) {
  const int K = ix.prm.n_codewords;
  int64_t* wcnt = sc.get<int64_t>(K + 1);
  int64_t* woff = sc.get<int64_t>(K + 1);
  k_work_count_tc<<<(unsigned)cdiv(K + 1, 256), 256, 0, s>>>(P.boff, ix.list_off, K, tn, ts_class, wcnt);
  GIFT_LAUNCHED("k_work_count_tc");
  scan_exclusive_i64(wcnt, woff, K + 1, sc, s);
  ListSched ls;
  ls.woff = woff;
  ls.K = K;
  ls.boff = P.boff;
  ls.list_off = ix.list_off;
  ls.nkb = 0;
  return ls;
}

// E4M3 scan of the lists of one slot class
template <int TS>
void scan_fp8_class(const Index& ix, const FifPlan& P, const SlotInfo& si, const CUtensorMap& tA, const void* q8,
                    int64_t qrows, Scratch& sc, cudaStream_t s, int grid) {
  SlotsPolicy<1, 1, TS> pol;
  static_cast<ListSched&>(pol) = list_sched(ix, P, tc::kTM, sc, s, TS);
  pol.nkb = (int)cdiv((int64_t)ix.prm.dim, (int64_t)128);
  pol.si = si;
  pol.item_map = nullptr;
  pol.n_items = nullptr;
  const CUtensorMap tB = make_tmap_u8(q8, qrows, ix.prm.dim, TS);
  tc::launch_engine(tA, tB, tA, tB, pol, ix.d_err, grid, s);
}

// the rescore work of one slot class: its items that hold a candidate run
// (slot classes of up to 80 slots: slot columns; 128: slot rows, RescorePolicy)
template <int TS>
struct RescoreClass {
  using Pol = std::conditional_t<TS == 128, RescorePolicy, SlotsPolicy<2, 3, (TS < 128 ? TS : 64)>>;
  Pol pol;
  void plan(const Index& ix, const FifPlan& P, const SlotInfo& si, const int32_t* cand_sorted, int R,
            int64_t upper, int64_t* flags, int64_t* pos, Scratch& sc, cudaStream_t s) {
    ListSched ls = list_sched(ix, P, kRescTN, sc, s, TS);
    ls.nkb = (int)cdiv((int64_t)ix.prm.dim, (int64_t)64);
    static_cast<ListSched&>(pol) = ls;
    pol.si = si;
    if constexpr (TS == 128) {
      pol.cand = cand_sorted;
      pol.R = R;
    }
    int64_t* item_map = sc.get<int64_t>(upper);
    int64_t* n_items = sc.get<int64_t>(1);
    k_resc_flags<TS><<<(unsigned)cdiv(upper, 8), 256, 0, s>>>(ls, P.slot_view, P.vquery, ix.entry_run,
                                                             ix.list_shape, cand_sorted, R, upper, flags, P.stats);
    GIFT_LAUNCHED("k_resc_flags");
    scan_exclusive_i64(flags, pos, upper, sc, s);
    k_compact_items<<<(unsigned)cdiv(upper, 256), 256, 0, s>>>(flags, pos, upper, item_map, n_items);
    GIFT_LAUNCHED("k_compact_items");
    pol.item_map = item_map;
    pol.n_items = n_items;
  }
  // tE, tE2: the entry rows (hi, lo), 128-row boxes
  void run(const Index& ix, const CUtensorMap& tE, const CUtensorMap& tE2, const void* qhi, const void* qlo,
           int64_t qrows, int grid, cudaStream_t s) {
    const CUtensorMap tS = make_tmap_bf16(qhi, qrows, ix.prm.dim, TS);
    const CUtensorMap tS2 = make_tmap_bf16(qlo, qrows, ix.prm.dim, TS);
    if constexpr (TS == 128)
      tc::launch_engine(tS, tE, tS2, tE2, pol, ix.d_err, grid, s);  // slots are the MMA rows
    else
      tc::launch_engine(tE, tS, tE2, tS2, pol, ix.d_err, grid, s);
  }
};

}  // namespace

void fif_rescore_stats(const Index& ix, const FifPlan& P, const int32_t* cand_sorted, int R, Scratch& sc,
                       cudaStream_t s) {
  if (!P.stats || P.nslots <= 0) return;
  const ListSched ls = list_sched(ix, P, kRescTN, sc, s);
  const int64_t upper = std::max<int64_t>(P.upper_items, 1);
  int64_t* flags = sc.get<int64_t>(upper);
  k_resc_flags<tc::kTM><<<(unsigned)cdiv(upper, 8), 256, 0, s>>>(ls, P.slot_view, P.vquery, ix.entry_run, ix.list_shape,
                                                        cand_sorted, R, upper, flags, P.stats);
  GIFT_LAUNCHED("k_resc_flags");
}

void fif_scan_tc(const Index& ix, const FifPlan& P, uint32_t* table, bool rescore, const int32_t* cand_sorted,
                 int R, Scratch& sc, cudaStream_t s, uint32_t* table32) {
  const int D = ix.prm.dim;
  const int64_t ns = P.nslots;
  if (ns <= 0) return;
  const bool fused = table32 != nullptr;
  GIFT_REQUIRE(!fused || (!rescore && ix.prm.storage == GIFT_BF16 && ix.list_lo && !ix.list_hi && D > 64),
               "the FP32-level scan needs a BF16 store with its two-part rescore rows");
  if (fused) rescore = true;  // slot low parts, rescore tile width
  const bool fp8 = !rescore && ix.prm.storage == GIFT_FP8_E4M3;
  const int64_t qrows = ns + tc::kTM;  // one box of padding rows
  __nv_bfloat16* qhi = nullptr;
  __nv_bfloat16* qlo = nullptr;
  __nv_fp8_e4m3* q8 = nullptr;
  float* q8s = nullptr;
  if (fp8) {
    q8 = sc.get<__nv_fp8_e4m3>((size_t)qrows * D);
    q8s = sc.get<float>(ns);
    k_slot_fp8<<<(unsigned)ns, 256, 0, s>>>(P.q, P.slot_view, ns, D, q8, q8s);
    GIFT_LAUNCHED("k_slot_fp8");
  } else if (P.slot_hi && (P.slot_lo || !rescore)) {
    qhi = P.slot_hi;  // made by the scan of this batch
    qlo = P.slot_lo;
  } else {
    // the low parts too when this index rescores next, so the rescore reuses both
    const bool want_lo = rescore || (ix.prm.rescore_r > 0 && ix.list_lo != nullptr);
    qhi = sc.get<__nv_bfloat16>((size_t)qrows * D);
    qlo = want_lo ? sc.get<__nv_bfloat16>((size_t)qrows * D) : nullptr;
    k_slot_split<<<(unsigned)ns, 256, 0, s>>>(P.q, P.slot_view, ns, D, qhi, qlo);
    GIFT_LAUNCHED("k_slot_split");
    P.slot_hi = qhi;
    P.slot_lo = qlo;
  }
  // the BF16 scan and the FP32-level pass schedule 128 slots x tn entries per item
  auto sched = [&](int tn) {
    ListSched ls = list_sched(ix, P, tn, sc, s);
    ls.nkb = (int)cdiv(D, 64);
    return ls;
  };
  SlotInfo si;
  si.runbase = P.runbase;
  si.slot_view = P.slot_view;
  si.vquery = P.vquery;
  si.q_inv = P.q_inv;
  si.scale = ix.list_scale;
  si.entry_run = ix.entry_run;
  si.list_shape = ix.list_shape;
  si.slot_scale = q8s;
  si.table = table;
  const int grid = device_sm_count();
  if (fp8) {
    // lists of up to 80 slots: list entries are the MMA rows, query slots the columns,
    // one launch per slot class
    const CUtensorMap tA = make_tmap_u8(ix.list_feat, ix.list_rows_alloc, D, tc::kTM);
    if (P.kc) P.kc->begin(1);
    scan_fp8_class<16>(ix, P, si, tA, q8, qrows, sc, s, grid);
    scan_fp8_class<32>(ix, P, si, tA, q8, qrows, sc, s, grid);
    scan_fp8_class<64>(ix, P, si, tA, q8, qrows, sc, s, grid);
    scan_fp8_class<80>(ix, P, si, tA, q8, qrows, sc, s, grid);
    {  // lists of more than 80 slots: slots are the MMA rows, 256 entries per item
      ScanPolicy<1> pol;
      static_cast<ListSched&>(pol) = list_sched(ix, P, kScanTN, sc, s, 128);
      pol.nkb = (int)cdiv(D, 128);
      pol.si = si;
      const CUtensorMap tS = make_tmap_u8(q8, qrows, D, tc::kTM);
      const CUtensorMap tE = make_tmap_u8(ix.list_feat, ix.list_rows_alloc, D, ScanPolicy<1>::TN);
      tc::launch_engine(tS, tE, tS, tE, pol, ix.d_err, grid, s);
    }
    if (P.kc) P.kc->end(1);
  } else if (!rescore) {
    ScanPolicy<2> pol;
    static_cast<ListSched&>(pol) = sched(kScanTN);
    pol.si = si;
    const CUtensorMap tA = make_tmap_bf16(qhi, qrows, D, tc::kTM);
    const CUtensorMap tB = make_tmap_bf16(ix.list_feat, ix.list_rows_alloc, D, ScanPolicy<2>::TN);
    if (P.kc) P.kc->begin(1);
    tc::launch_engine(tA, tB, tA, tB, pol, ix.d_err, grid, s);
    if (P.kc) P.kc->end(1);
  } else if (fused) {
    // every touched pair at FP32 level (three products, reduction in chunks), every
    // run written: the top-R then comes from FP32-level scores and needs no rescore
    RescorePolicy pol;
    static_cast<ListSched&>(pol) = sched(kRescTN);
    pol.si = si;
    pol.si.table = table32;
    pol.cand = nullptr;
    pol.R = 0;
    pol.item_map = nullptr;
    pol.n_items = nullptr;
    const CUtensorMap tA = make_tmap_bf16(qhi, qrows, D, tc::kTM);
    const CUtensorMap tB = make_tmap_bf16(ix.list_feat, ix.list_rows_alloc, D, RescorePolicy::TN);
    const CUtensorMap tA2 = make_tmap_bf16(qlo, qrows, D, tc::kTM);
    const CUtensorMap tB2 = make_tmap_bf16(ix.list_lo, ix.list_rows_alloc, D, RescorePolicy::TN);
    if (P.kc) P.kc->begin(2);
    tc::launch_engine(tA, tB, tA2, tB2, pol, ix.d_err, grid, s);
    if (P.kc) P.kc->end(2);
  } else {
    GIFT_REQUIRE(ix.list_lo != nullptr, "rescore needs the two-part BF16 list store");
    // BF16 index: the store itself is the hi part; FP8 index: a separate BF16 hi store
    const void* bhi = ix.list_hi ? ix.list_hi : ix.list_feat;
    SlotInfo sr = si;
    sr.scale = ix.list_hi ? ix.list_scale_hi : ix.list_scale;
    // the work items that hold a candidate run, per slot class, in their original order
    const int64_t upper = std::max<int64_t>(P.upper_items, 1);
    int64_t* flags = sc.get<int64_t>(upper);
    int64_t* pos = sc.get<int64_t>(upper);
    RescoreClass<16> c16;
    RescoreClass<32> c32;
    RescoreClass<64> c64;
    RescoreClass<80> c80;
    RescoreClass<128> c128;
    c16.plan(ix, P, sr, cand_sorted, R, upper, flags, pos, sc, s);
    c32.plan(ix, P, sr, cand_sorted, R, upper, flags, pos, sc, s);
    c64.plan(ix, P, sr, cand_sorted, R, upper, flags, pos, sc, s);
    c80.plan(ix, P, sr, cand_sorted, R, upper, flags, pos, sc, s);
    c128.plan(ix, P, sr, cand_sorted, R, upper, flags, pos, sc, s);
    const CUtensorMap tA = make_tmap_bf16(bhi, ix.list_rows_alloc, D, tc::kTM);
    const CUtensorMap tA2 = make_tmap_bf16(ix.list_lo, ix.list_rows_alloc, D, tc::kTM);
    if (P.kc) P.kc->begin(2);
    c16.run(ix, tA, tA2, qhi, qlo, qrows, grid, s);
    c32.run(ix, tA, tA2, qhi, qlo, qrows, grid, s);
    c64.run(ix, tA, tA2, qhi, qlo, qrows, grid, s);
    c80.run(ix, tA, tA2, qhi, qlo, qrows, grid, s);
    c128.run(ix, tA, tA2, qhi, qlo, qrows, grid, s);
    if (P.kc) P.kc->end(2);
  }
}

}  // namespace gift
