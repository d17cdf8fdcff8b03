// Exact set-to-set match (Eq. 3) on the tensor cores:
// S(x_q, x_p) = (1/|V(x_q)|) sum_i max_j s(q_i, p_j), s the cosine.
//
// Work item: (128 database views = columns, 128 query views = rows); items run
// column-tile-major so CTAs working at the same time share the database tile.
// Operands are two-part BF16 (x = hi + lo, three products) with the reduction
// in four chunks summed in FP32 by the epilogue, which scales by the inverse
// norms and reduces each row over every run of N_v columns of one shape,
// folding (max, first argmax) into a per-(query view, shape) cell with a
// 64-bit atomicMax; a second kernel sums the cells of each query's views.
// An index without the shape-ordered copy (a streamed or FP8 index with a
// rescore store) runs the same contraction over its list-ordered two-part
// rows, folding runs of equal shape instead of N_v-column groups.
#include "gift_internal.cuh"
#include "segmax.cuh"
#include "tc_engine.cuh"

namespace gift {

namespace {

constexpr int kChunks = 4;

struct ExactPolicy {
  static constexpr int TN = 128, NBUF = 4, STAGES = 3, SPLIT = 3, EB = 2;
  static constexpr int kWarpSmem = TN * 4;
  int64_t rows;        // query views in this pass
  int64_t ncols;       // database views N * N_v
  int64_t n_rt;        // row tiles
  int nv;              // views per shape
  int64_t n_shapes;
  int nkb;
  const float* q_inv;  // [rows]
  const float* r_inv;  // [ncols]
  unsigned long long* cell;  // [rows, n_shapes]
  struct Item {
    int64_t r0, c0;
    int nr, nc;
  };
  struct Ctx {
    float sum[TN];
  };
  __device__ __forceinline__ int64_t total() const { return n_rt * cdiv(ncols, TN); }
  __device__ __forceinline__ Item decode(int64_t item) const {
    Item it;
    const int64_t ct = item / n_rt, rt = item % n_rt;
    it.r0 = rt * tc::kTM;
    it.c0 = ct * TN;
    it.nr = (int)min((int64_t)tc::kTM, rows - it.r0);
    it.nc = (int)min((int64_t)TN, ncols - it.c0);
    return it;
  }
  // never an empty chunk: each chunk must write its own accumulator
  // chunks bound the MMA steps feeding one accumulator (about 192, 3 products
  // x 4 sub-steps per k-block); short reductions use one chunk
  __device__ __forceinline__ int nch() const {
    const int want = (nkb * 12 + 191) / 192;
    return want < 1 ? 1 : (want > kChunks ? kChunks : want);
  }
  __device__ __forceinline__ int nchunks(const Item&) const { return nch(); }
  __device__ __forceinline__ void chunk(const Item& it, int c, int& br, int& kb0, int& kb1) const {
    br = (int)it.c0;
    const int nch = this->nch();
    kb0 = (int)((int64_t)nkb * c / nch);
    kb1 = (int)((int64_t)nkb * (c + 1) / nch);
  }
  __device__ __forceinline__ int a_row(const Item& it) const { return (int)it.r0; }
  __device__ __forceinline__ void epi_begin(const Item& it, Ctx& x, int, int, uint8_t* ws) const {
    float* ri = reinterpret_cast<float*>(ws);
    const int lane = threadIdx.x & 31;
    for (int c = lane; c < TN; c += 32) ri[c] = c < it.nc ? r_inv[it.c0 + c] : 0.f;
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
  __device__ __forceinline__ void epi_end(const Item& it, Ctx& x, int m, uint8_t* ws) const {
    if (m >= it.nr) return;
    const float* ri = reinterpret_cast<const float*>(ws);
    const int64_t row = it.r0 + m;
    const float qi = q_inv[row];
    unsigned long long* crow = cell + row * n_shapes;
    // walk the columns keeping (shape, j) incrementally: no division per column
    int64_t shape = it.c0 / nv;
    int j = (int)(it.c0 - shape * nv);
    float best = 0.f;
    int bj = 0;
    bool open = false;
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      if (c < it.nc) {
        const float v = x.sum[c] * qi * ri[c];
        if (!open || v > best) {
          best = v;
          bj = j;
          open = true;
        }
        if (++j == nv) {
          atomicMax(crow + shape, ((unsigned long long)f2key(best) << 32) | (0xFFFFull - (unsigned)bj));
          ++shape;
          j = 0;
          open = false;
        }
      }
    }
    if (open) atomicMax(crow + shape, ((unsigned long long)f2key(best) << 32) | (0xFFFFull - (unsigned)bj));
  }
};

// The same contraction for short reductions (one accumulator chunk, at most 16
// k-blocks: the projected match, D = d_out) with 64 views per shape, so a
// 128-column tile holds exactly two whole shapes. Each shape's (max, first
// argmax) is taken straight from the accumulator: the epilogue keeps no
// per-column sums, which would otherwise bound a kernel with this little MMA
// work per tile.
struct ShortSegPolicy {
  static constexpr int TN = 128, NBUF = 4, STAGES = 3, SPLIT = 3, EB = 2;
  static constexpr int kNv = 64;
  static constexpr int kWarpSmem = TN * 4;
  int64_t rows, ncols, n_rt, n_shapes;
  int nkb;
  const float* q_inv;
  const float* r_inv;
  unsigned long long* cell;
  struct Item {
    int64_t r0, c0;
    int nr, nc;
  };
  struct Ctx {
    float qi;
  };
  __device__ __forceinline__ int64_t total() const { return n_rt * cdiv(ncols, TN); }
  __device__ __forceinline__ Item decode(int64_t item) const {
    Item it;
    const int64_t ct = item / n_rt, rt = item % n_rt;
    it.r0 = rt * tc::kTM;
    it.c0 = ct * TN;
    it.nr = (int)min((int64_t)tc::kTM, rows - it.r0);
    it.nc = (int)min((int64_t)TN, ncols - it.c0);
    return it;
  }
  __device__ __forceinline__ int nchunks(const Item&) const { return 1; }
  __device__ __forceinline__ void chunk(const Item& it, int, int& br, int& kb0, int& kb1) const {
    br = (int)it.c0;
    kb0 = 0;
    kb1 = nkb;
  }
  __device__ __forceinline__ int a_row(const Item& it) const { return (int)it.r0; }
  __device__ __forceinline__ void epi_begin(const Item& it, Ctx& x, int m, int, uint8_t* ws) const {
    float* ri = reinterpret_cast<float*>(ws);
    const int lane = threadIdx.x & 31;
    for (int c = lane; c < TN; c += 32) ri[c] = c < it.nc ? r_inv[it.c0 + c] : 0.f;
    x.qi = m < it.nr ? q_inv[it.r0 + m] : 0.f;
  }
  __device__ __forceinline__ void epi_chunk(const Item& it, int, uint32_t taddr, Ctx& x, int m, uint8_t* ws) const {
    const float* ri = reinterpret_cast<const float*>(ws);
    unsigned long long* crow = cell + (it.r0 + m) * n_shapes + it.c0 / kNv;
#pragma unroll
    for (int g = 0; g < TN / kNv; ++g) {
      float best = 0.f;
      int bj = 0;
#pragma unroll
      for (int pc = 0; pc < kNv / 32; ++pc) {
        uint32_t r[32];
        tc::tmem_ld32(taddr + g * kNv + pc * 32, r);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = g * kNv + pc * 32 + j;
          const float v = __uint_as_float(r[j]) * x.qi * ri[c];
          if ((pc == 0 && j == 0) || v > best) {  // ties keep the first view
            best = v;
            bj = pc * 32 + j;
          }
        }
      }
      if (m < it.nr && g * kNv < it.nc)
        atomicMax(crow + g, ((unsigned long long)f2key(best) << 32) | (0xFFFFull - (unsigned)bj));
    }
  }
  __device__ __forceinline__ void epi_end(const Item&, Ctx&, int, uint8_t*) const {}
};

// The same match over the list-ordered two-part store of an index that keeps
// no shape-ordered copy: columns are list entries, the shape of each comes from
// the list structure, and each row folds the maximum of every run of equal
// shape (runs may continue into the next tile: the atomicMax merges them).
struct ExactListPolicy {
  static constexpr int TN = 128, NBUF = 4, STAGES = 3, SPLIT = 3, EB = 2;
  static constexpr int kWarpSmem = TN * 8;
  int64_t rows;               // query views in this pass
  int64_t ncols;              // list entries
  int64_t n_rt;               // row tiles
  int64_t n_shapes;
  int nkb;
  const float* q_inv;         // [rows]
  const float* c_scale;       // [ncols] 1/|x| of each entry's two-part row
  const int32_t* c_shape;     // [ncols] shape of each entry
  unsigned long long* cell;   // [rows, n_shapes]
  struct Item {
    int64_t r0, c0;
    int nr, nc;
  };
  struct Ctx {
    float sum[TN];
  };
  __device__ __forceinline__ int64_t total() const { return n_rt * cdiv(ncols, TN); }
  __device__ __forceinline__ Item decode(int64_t item) const {
    Item it;
    const int64_t ct = item / n_rt, rt = item % n_rt;
    it.r0 = rt * tc::kTM;
    it.c0 = ct * TN;
    it.nr = (int)min((int64_t)tc::kTM, rows - it.r0);
    it.nc = (int)min((int64_t)TN, ncols - it.c0);
    return it;
  }
  __device__ __forceinline__ int nch() const {
    const int want = (nkb * 12 + 191) / 192;
    return want < 1 ? 1 : (want > kChunks ? kChunks : want);
  }
  __device__ __forceinline__ int nchunks(const Item&) const { return nch(); }
  __device__ __forceinline__ void chunk(const Item& it, int c, int& br, int& kb0, int& kb1) const {
    br = (int)it.c0;
    const int nch = this->nch();
    kb0 = (int)((int64_t)nkb * c / nch);
    kb1 = (int)((int64_t)nkb * (c + 1) / nch);
  }
  __device__ __forceinline__ int a_row(const Item& it) const { return (int)it.r0; }
  __device__ __forceinline__ void epi_begin(const Item& it, Ctx& x, int, int, uint8_t* ws) const {
    float* sc = reinterpret_cast<float*>(ws);
    int32_t* sh = reinterpret_cast<int32_t*>(ws + TN * 4);
    const int lane = threadIdx.x & 31;
    for (int c = lane; c < TN; c += 32) {
      sc[c] = c < it.nc ? c_scale[it.c0 + c] : 0.f;
      sh[c] = c < it.nc ? c_shape[it.c0 + c] : -1;
    }
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
  __device__ __forceinline__ void epi_end(const Item& it, Ctx& x, int m, uint8_t* ws) const {
    if (m >= it.nr) return;
    const float* sc = reinterpret_cast<const float*>(ws);
    const int32_t* sh = reinterpret_cast<const int32_t*>(ws + TN * 4);
    const int64_t row = it.r0 + m;
    const float qi = q_inv[row];
    unsigned long long* crow = cell + row * n_shapes;
    int shape = -1;
    float best = 0.f;
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      if (c < it.nc) {
        const float v = x.sum[c] * qi * sc[c];
        if (sh[c] != shape) {
          if (shape >= 0) atomicMax(crow + shape, ((unsigned long long)f2key(best) << 32) | 0xFFFFull);
          shape = sh[c];
          best = v;
        } else {
          best = fmaxf(best, v);
        }
      }
    }
    if (shape >= 0) atomicMax(crow + shape, ((unsigned long long)f2key(best) << 32) | 0xFFFFull);
  }
};

}  // namespace

void segmax_tc(const __nv_bfloat16* a_hi, const __nv_bfloat16* a_lo, int64_t a_rows_alloc, const float* a_inv,
               const __nv_bfloat16* b_hi, const __nv_bfloat16* b_lo, int64_t b_rows_alloc, const float* b_inv,
               int64_t ncols, int nv, int D, const int32_t* d_qoff, const std::vector<int32_t>& h_qoff, int32_t B,
               float* S, int16_t* argmax, int* err, Scratch& sc, cudaStream_t s) {
  const int64_t N = ncols / nv;
  const int64_t cap = std::max<int64_t>(1, ((int64_t)1 << 27) / N);  // cell block <= 1 GiB
  unsigned long long* cell = nullptr;
  int64_t cell_rows = 0;
  const CUtensorMap tB = make_tmap_bf16(b_hi, b_rows_alloc, D, ExactPolicy::TN);
  const CUtensorMap tB2 = make_tmap_bf16(b_lo, b_rows_alloc, D, ExactPolicy::TN);
  const int sms = device_sm_count();
  int32_t b0 = 0;
  while (b0 < B) {
    int32_t b1 = b0 + 1;
    while (b1 < B && (int64_t)(h_qoff[b1 + 1] - h_qoff[b0]) <= cap) ++b1;
    const int64_t v0 = h_qoff[b0], rows = h_qoff[b1] - v0;
    if (rows > cell_rows) {
      cell = sc.get<unsigned long long>((size_t)rows * N);
      cell_rows = rows;
    }
    GIFT_CUDA(cudaMemsetAsync(cell, 0, (size_t)rows * N * 8, s));
    const CUtensorMap tA = make_tmap_bf16(a_hi + v0 * D, a_rows_alloc - v0, D, tc::kTM);
    const CUtensorMap tA2 = make_tmap_bf16(a_lo + v0 * D, a_rows_alloc - v0, D, tc::kTM);
    const int nkb = (int)cdiv(D, tc::kTK);
    if (nv == ShortSegPolicy::kNv && nkb <= 16) {
      ShortSegPolicy p;
      p.rows = rows;
      p.ncols = ncols;
      p.n_rt = cdiv(rows, tc::kTM);
      p.n_shapes = N;
      p.nkb = nkb;
      p.q_inv = a_inv + v0;
      p.r_inv = b_inv;
      p.cell = cell;
      const int grid = (int)std::min<int64_t>(sms, p.n_rt * cdiv(ncols, ShortSegPolicy::TN));
      tc::launch_engine(tA, tB, tA2, tB2, p, err, grid, s);
      segmax_reduce(cell, N, d_qoff, b0, b1 - b0, (int32_t)v0, S, argmax, s);
      b0 = b1;
      continue;
    }
    ExactPolicy p;
    p.rows = rows;
    p.ncols = ncols;
    p.n_rt = cdiv(rows, tc::kTM);
    p.nv = nv;
    p.n_shapes = N;
    p.nkb = (int)cdiv(D, tc::kTK);
    p.q_inv = a_inv + v0;
    p.r_inv = b_inv;
    p.cell = cell;
    const int grid = (int)std::min<int64_t>(sms, p.n_rt * cdiv(ncols, ExactPolicy::TN));
    tc::launch_engine(tA, tB, tA2, tB2, p, err, grid, s);
    segmax_reduce(cell, N, d_qoff, b0, b1 - b0, (int32_t)v0, S, argmax, s);
    b0 = b1;
  }
}

void exact_scores_tc(const Index& ix, const float* q, const float* q_inv, int64_t nv, const int32_t* d_qoff,
                     const std::vector<int32_t>& h_qoff, int32_t B, float* S, Scratch& sc, cudaStream_t s) {
  const int D = ix.prm.dim;
  const int64_t qrows = nv + tc::kTM;  // one box of padding rows
  __nv_bfloat16* hi = sc.get<__nv_bfloat16>((size_t)qrows * D);
  __nv_bfloat16* lo = sc.get<__nv_bfloat16>((size_t)qrows * D);
  split_rows_bf16(q, nv, D, hi, lo, s);
  segmax_tc(hi, lo, qrows, q_inv, ix.ex_hi, ix.ex_lo, ix.ex_rows, ix.row_inv, ix.n_rows, ix.prm.views_per_shape, D,
            d_qoff, h_qoff, B, S, nullptr, ix.d_err, sc, s);
}

}  // namespace gift

namespace gift {

// Eq. 3 for every query against all shapes from the list-ordered two-part store
void exact_scores_lists(const Index& ix, const float* q, const float* q_inv, int64_t nv, const int32_t* d_qoff,
                        const std::vector<int32_t>& h_qoff, int32_t B, float* S, Scratch& sc, cudaStream_t s) {
  const int D = ix.prm.dim;
  const int64_t N = ix.prm.n_shapes;
  const int64_t ncols = ix.n_entries;
  const int64_t qrows = nv + tc::kTM;  // one box of padding rows
  __nv_bfloat16* hi = sc.get<__nv_bfloat16>((size_t)qrows * D);
  __nv_bfloat16* lo = sc.get<__nv_bfloat16>((size_t)qrows * D);
  split_rows_bf16(q, nv, D, hi, lo, s);
  const void* bhi = ix.list_hi ? ix.list_hi : ix.list_feat;  // FP8 index: the separate BF16 part
  const float* bscale = ix.list_hi ? ix.list_scale_hi : ix.list_scale;
  const CUtensorMap tB = make_tmap_bf16(bhi, ix.list_rows_alloc, D, ExactListPolicy::TN);
  const CUtensorMap tB2 = make_tmap_bf16(ix.list_lo, ix.list_rows_alloc, D, ExactListPolicy::TN);
  const int64_t cap = std::max<int64_t>(1, ((int64_t)1 << 28) / N);  // cell block <= 2 GiB
  unsigned long long* cell = nullptr;
  int64_t cell_rows = 0;
  const int sms = device_sm_count();
  int32_t b0 = 0;
  while (b0 < B) {
    int32_t b1 = b0 + 1;
    while (b1 < B && (int64_t)(h_qoff[b1 + 1] - h_qoff[b0]) <= cap) ++b1;
    const int64_t v0 = h_qoff[b0], rows = h_qoff[b1] - v0;
    if (rows > cell_rows) {
      cell = sc.get<unsigned long long>((size_t)rows * N);
      cell_rows = rows;
    }
    GIFT_CUDA(cudaMemsetAsync(cell, 0, (size_t)rows * N * 8, s));
    ExactListPolicy p;
    p.rows = rows;
    p.ncols = ncols;
    p.n_rt = cdiv(rows, tc::kTM);
    p.n_shapes = N;
    p.nkb = (int)cdiv(D, tc::kTK);
    p.q_inv = q_inv + v0;
    p.c_scale = bscale;
    p.c_shape = ix.list_shape;
    p.cell = cell;
    const CUtensorMap tA = make_tmap_bf16(hi + v0 * D, qrows - v0, D, tc::kTM);
    const CUtensorMap tA2 = make_tmap_bf16(lo + v0 * D, qrows - v0, D, tc::kTM);
    const int grid = (int)std::min<int64_t>(sms, p.n_rt * cdiv(ncols, ExactListPolicy::TN));
    tc::launch_engine(tA, tB, tA2, tB2, p, ix.d_err, grid, s);
    segmax_reduce(cell, N, d_qoff, b0, b1 - b0, (int32_t)v0, S, nullptr, s);
    b0 = b1;
  }
}

}  // namespace gift
