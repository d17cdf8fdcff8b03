// Internal declarations of the GIFT CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <algorithm>
#include <functional>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/gift.h"

namespace gift {

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
  gift_status status;
  Error(gift_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

[[noreturn]] void fail(gift_status s, const std::string& msg);
// runs body, turning errors into a status and the thread's last-error message
gift_status guarded(const char* fn, const std::function<void()>& body);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
#define GIFT_CUDA(x) ::gift::check_cuda((x), #x, __FILE__, __LINE__)
void count_launch();
#define GIFT_LAUNCHED(name) \
  do { ::gift::count_launch(); ::gift::check_cuda(cudaGetLastError(), name, __FILE__, __LINE__); } while (0)
#define GIFT_REQUIRE(cond, msg) \
  do { if (!(cond)) ::gift::fail(GIFT_EINVAL, msg); } while (0)

// ---------------------------------------------------------------- scratch
// Stream-ordered scratch: every allocation is released (stream-ordered) when
// the Scratch object goes out of scope, so concurrent calls never share it.
struct Scratch {
  cudaStream_t stream;
  std::vector<void*> blocks;
  explicit Scratch(cudaStream_t s) : stream(s) {}
  ~Scratch();
  void* raw(size_t bytes);
  template <class T> T* get(size_t n) { return static_cast<T*>(raw(n * sizeof(T) + 16)); }
};

// ---------------------------------------------------------------- kernel timing
// CUDA events around single kernel launches (on the launching stream) when a
// call is timed; ids: 0 quantiser, 1 scan, 2 rescore.
struct KernelClock {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> spans;
  int64_t assign_rows = 0;
  void begin(int id);
  void end(int id);
};

// ---------------------------------------------------------------- fixed point
// Shape scores are sums of per-view maxima in [0, 1]; they are accumulated in
// uint64 fixed point so that the sum is exact and independent of the order.
constexpr double kScoreFix = 4294967296.0;  // 2^32
// S-IF memberships: uint32 round(S * 2^31), S in [0, 1].
constexpr double kMemberFix = 2147483648.0;  // 2^31

// ---------------------------------------------------------------- index
// State of a streamed build (gift_build_begin / add / end_pass).
struct StreamBuild {
  int stage = 1;               // pass accepting chunks: 1 codes, 2 stores, 3 S-IF; 4 = complete
  int64_t rows_added = 0;      // rows added in the current pass
  std::vector<uint8_t> seen;   // [N] shapes added in the current pass
  int32_t* pos = nullptr;      // [n_entries] list position of each (row, assignment) (pass 2)
  ~StreamBuild() { cudaFree(pos); }  // freed once the build completes
};

struct Index {
  gift_index_params prm{};
  int64_t n_rows = 0;     // N * Nv
  int db_ma = 1;          // codewords per database view
  int64_t n_entries = 0;  // F-IF entries: n_rows * db_ma
  int device = 0;

  // codebook
  float* codebook = nullptr;   // [K, D]
  float* cb_half_sq = nullptr; // [K]  0.5 * ||b_k||^2
  float cb_max_norm = 0.f;
  __nv_bfloat16* cb_hi = nullptr;  // [cb_rows_alloc, D] two-part BF16 codebook (+ padding rows)
  __nv_bfloat16* cb_lo = nullptr;
  int64_t cb_rows_alloc = 0;

  // database
  float* master = nullptr;     // [n_rows, D] FP32 views (keep_exact)
  float* row_inv = nullptr;    // [n_rows] 1/||x|| (0 for a zero row)
  int32_t* db_codes = nullptr; // [n_rows * db_ma]

  // F-IF
  int64_t* list_off = nullptr;   // [K+1]
  std::vector<int64_t> h_list_off;
  int32_t* list_row = nullptr;   // [n_entries] row of each entry (list order)
  int32_t* list_shape = nullptr; // [n_entries]
  void* list_feat = nullptr;     // [n_entries, D] in storage dtype
  void* list_lo = nullptr;       // [n_entries, D] BF16 residual x - bf16(x) (rescore)
  void* list_hi = nullptr;       // [n_entries, D] BF16 bf16(x) when the store is FP8 (rescore)
  float* list_scale_hi = nullptr;// [n_entries] 1/||x|| for the BF16 parts when the store is FP8
  int64_t list_rows_alloc = 0;   // rows of list_feat / list_lo including padding

  // exact match: shape-ordered two-part BF16 copy of the views (+ padding rows)
  __nv_bfloat16* ex_hi = nullptr;
  __nv_bfloat16* ex_lo = nullptr;
  int64_t ex_rows = 0;
  float* list_scale = nullptr;   // [n_entries] factor turning a stored dot into a cosine
  int32_t* entry_run = nullptr;  // [n_entries] run index within its list
  int32_t* nruns = nullptr;      // [K]
  int64_t* run_off = nullptr;    // [K] first global run of each list
  int32_t* run_shape = nullptr;  // [n_runs]
  int64_t n_runs = 0;
  int32_t max_runs = 0;
  int32_t max_list = 0;
  int32_t n_nonempty = 0;
  int64_t scan_tiles_upper = 0;  // sum_k ceil(L_k / kScanTE)

  // S-IF
  int32_t k1 = 0;
  int32_t sif_n = 0;             // shapes the S-IF covers: n_shapes, or the whole database of which
                                 // this index holds a shard (gift_sif_from_neighbours)
  int64_t* sif_off = nullptr;    // [N+1]
  int32_t* sif_ids = nullptr;    // [N*k1]
  uint32_t* sif_mem = nullptr;   // [N*k1]
  uint64_t* sif_card = nullptr;  // [N]
  int32_t max_sif_entry = 0;
  int32_t* row_ids = nullptr;    // [N*k1] N_k1(p) of every database shape, ranked (score desc, id asc)
  float* row_sc = nullptr;       // [N*k1] their scores S(x_p, x_i): the rows of F_p (Eq. 7)

  int* d_err = nullptr;          // device error flag set by bounded waits (0 = none)
  StreamBuild* sb = nullptr;     // non-null while a streamed build is in progress

  size_t device_bytes = 0;
  std::vector<void*> owned;

  // timing
  bool timing = false;
  gift_timing_t last_timing{};
  std::vector<cudaEvent_t> ev;  // stage events of the last timed call
  std::vector<int> ev_stage;    // stage id of each event interval
  unsigned long long* stats_pinned = nullptr;  // scan bytes, pairs, rescore bytes
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> kspans;  // of the last timed call
  int64_t k_assign_rows = 0;
  bool stats_valid = false;

  template <class T> T* alloc(size_t n);
  bool ready() const { return sb == nullptr; }
  ~Index();
};

size_t dtype_bytes(int storage);

// ---------------------------------------------------------------- kernels
// scan constants: entries and query slots per work item of the scan kernel
constexpr int kScanTE = 64;
constexpr int kScanTS = 64;

// k_util.cu
void launch_row_invnorm(const float* X, int64_t n, int D, float* inv, cudaStream_t s);
void launch_half_sq_norm(const float* X, int64_t n, int D, float* out, cudaStream_t s);
void scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, Scratch& sc, cudaStream_t s);
// Stable sort of items 0..n-1 by key (0 <= key < nbins): perm_out lists item
// indices grouped by key, ascending index within a key; keys_out the keys.
void stable_sort_by_key(const int32_t* keys, int64_t n, int32_t nbins, int32_t* perm_out,
                        int32_t* keys_out, Scratch& sc, cudaStream_t s);
// off[k] = first position of key k in sorted keys, off[nbins] = n.
void bin_offsets(const int32_t* sorted_keys, int64_t n, int32_t nbins, int64_t* off, cudaStream_t s);
void launch_fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s);

// k_assign.cu
// codes[v*ma + a] = a-th nearest codeword by (squared distance, index);
// x_inv (optional) holds 1/||x|| of the rows.
void assign_codes(const Index& ix, const float* X, int64_t n, int ma, int32_t* codes,
                  Scratch& sc, cudaStream_t s, const float* x_inv = nullptr, KernelClock* kc = nullptr);
// hi = bf16(x), lo = bf16(x - hi) of a row-major [n, D] FP32 matrix
void split_rows_bf16(const float* X, int64_t n, int D, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s);

// api.cu: the quantiser's derived codebook arrays (||b||^2 / 2, two-part BF16
// rows padded by one TMA box, max ||b||) from ix.codebook; allocates them on first use
void prepare_codebook(Index& ix, cudaStream_t s);

// k_kmeans.cu: Lloyd's k-means from the rows init_rows; C_out [K, D] (device or host)
void kmeans(const float* X, int64_t n, int D, int K, const std::vector<int32_t>& init_rows, int iters, float* C_out,
            Scratch& sc, cudaStream_t s);

// k_render.cu: the N_v = n_az * n_el depth views of every mesh (Sec. 2.1); depth [M, N_v, H, W] on the device
void render_views(const float* V, const int32_t* T, const std::vector<int64_t>& h_voff,
                  const std::vector<int64_t>& h_toff, int M, int n_az, int n_el, int H, int W, float* depth,
                  Scratch& sc, cudaStream_t s);

// k_exact_tc.cu: Eq. 3 over all N shapes on the tensor cores
void exact_scores_tc(const Index& ix, const float* q, const float* q_inv, int64_t nv, const int32_t* d_qoff,
                     const std::vector<int32_t>& h_qoff, int32_t B, float* S, Scratch& sc, cudaStream_t s);
// the same from the list-ordered two-part store (indices built without keep_exact)
void exact_scores_lists(const Index& ix, const float* q, const float* q_inv, int64_t nv, const int32_t* d_qoff,
                        const std::vector<int32_t>& h_qoff, int32_t B, float* S, Scratch& sc, cudaStream_t s);


// k_topk.cu
// Per row b of `scores` [B, n] (or of keys64 when scores == nullptr): the k
// largest by (value desc, index asc). ids_out/val_out [B, k] (val_out may be
// null). When n < k the tail gets id -1 and -INF.
void topk_rows_f32(const float* scores, int32_t B, int64_t n, int32_t k, int32_t* ids_out,
                   float* val_out, Scratch& sc, cudaStream_t s);
void topk_rows_u64(const uint64_t* keys, int32_t B, int64_t n, int32_t k, int32_t* ids_out,
                   uint64_t* key_out, Scratch& sc, cudaStream_t s);
// Rows of (id, score) pairs of length r: sort by (score desc, id asc) and keep k.
void sort_candidates(const int32_t* ids, const float* scores, int32_t B, int32_t r, int32_t k,
                     int32_t* ids_out, float* scores_out, cudaStream_t s);
// Rows of ids of length r: ascending copy.
void sort_ids_rows(const int32_t* ids, int32_t B, int32_t r, int32_t* out, cudaStream_t s);
// Rows of (id, score) pairs of any length n (ids distinct per row, id < 0 =
// none): the k best by (score desc, id asc); missing entries id -1, -INF.
void merge_topk_rows(const int32_t* ids, const float* scores, int32_t B, int64_t n, int32_t k, int32_t* ids_out,
                     float* scores_out, Scratch& sc, cudaStream_t s);

// k_sif.cu
void sif_build(Index& ix, const int32_t* nbr_ids, const float* nbr_scores, Scratch& sc,
               cudaStream_t s);
void sif_rerank(const Index& ix, const int32_t* cand_ids, const float* cand_scores, int32_t B,
                int32_t n_cand, int32_t k1, int32_t topk, int32_t* out_ids, float* out_sprime,
                Scratch& sc, cudaStream_t s);
// bytes of caller-provided scratch sif_rerank_into needs
size_t sif_rerank_scratch_bytes(int32_t B, int32_t N, int32_t topk);
void sif_rerank_into(const Index& ix, const int32_t* cand_ids, const float* cand_scores, int32_t B, int32_t n_cand,
                     int32_t k1, int32_t topk, int32_t* out_ids, float* out_sprime, void* scratch,
                     size_t scratch_bytes, cudaStream_t s);

// Two-measure contextual re-ranking (Sec. 2.4: Eqs. 9-11) over two indices of
// the same database shapes: the aggregated contextual activation of every
// database shape, transposed into its own second inverted file.
struct Aca {
  const Index* m[2] = {nullptr, nullptr};
  int32_t N = 0;
  int k1 = 0, k2 = 0, mode = 0, cap = 0;
  float alpha = 0.5f;
  int device = 0;
  int64_t* off = nullptr;              // [N+1]
  int32_t* ids = nullptr;              // [pairs] shapes p of entry i, ascending
  uint32_t* mem = nullptr;             // [pairs] round(F_p[i] * 2^31)
  unsigned long long* card = nullptr;  // [N] ||F_p||_1 in the same fixed point
  int64_t pairs = 0;
  int32_t max_entry = 0;
  std::vector<void*> owned;
  size_t device_bytes = 0;
  template <class T> T* alloc(size_t n);
  ~Aca();
};
void aca_build(Aca& a, Scratch& sc, cudaStream_t s);
void aca_rerank(const Aca& a, const int32_t* cand1, const float* sc1, const int32_t* cand2, const float* sc2,
                int32_t B, int32_t n_cand, int32_t topk, int32_t* out_ids, float* out_sprime, Scratch& sc,
                cudaStream_t s);

// k_match.cu (dtype: GIFT_F32 or GIFT_BF16 for q, p and W)
void match_forward(const void* q, const std::vector<int32_t>& h_qoff, int32_t Bq, const void* p, int32_t Np,
                   int32_t nv, const void* W, int32_t din, int32_t dout, int32_t dtype, float* S, int16_t* argmax,
                   Scratch& sc, cudaStream_t s);
void match_backward(const void* q, const std::vector<int32_t>& h_qoff, int32_t Bq, const void* p, int32_t Np,
                    int32_t nv, const void* W, int32_t din, int32_t dout, int32_t dtype, const float* gS,
                    const int16_t* argmax, float* dW, float* dQ, float* dP, Scratch& sc, cudaStream_t s);

// ---------------------------------------------------------------- device helpers
__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Order-preserving map of a float to uint32 (larger float -> larger key).
__device__ __forceinline__ uint32_t f2key(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

// Two-float (compensated) FP32 accumulation, in place of FP64 on the GPU:
// value = hi + lo. two_sum gives s + e == a + b exactly (Knuth's TwoSum, six
// FP32 additions, no products, so no contraction into FMA can change it);
// the rounding errors of the running sum collect in lo, whose own rounding
// is ~2^-24 |lo|, so n terms sum with ~n 2^-48 relative error before the
// final rounding of hi + lo.
struct F2 {
  float hi = 0.f, lo = 0.f;
};
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}
__device__ __forceinline__ void f2_add(F2& x, float v) {
  float s, e;
  two_sum(x.hi, v, s, e);
  x.hi = s;
  x.lo += e;
}
__device__ __forceinline__ F2 f2_merge(F2 a, const F2& b) {
  f2_add(a, b.hi);
  a.lo += b.lo;
  return a;
}
__device__ __forceinline__ F2 f2_shfl_xor(const F2& x, int o) {
  F2 y;
  y.hi = __shfl_xor_sync(0xffffffffu, x.hi, o);
  y.lo = __shfl_xor_sync(0xffffffffu, x.lo, o);
  return y;
}
__device__ __forceinline__ float f2_value(const F2& x) { return x.hi + x.lo; }

}  // namespace gift
