// Per-call plan of an F-IF batch (device buffers in the call's scratch).
#pragma once
#include "gift_internal.cuh"

namespace gift {

struct FifPlan {
  // inputs
  int64_t nv = 0;                 // query views in the batch
  int ma = 1;                     // assignments per view
  int32_t B = 0;                  // queries
  const float* q = nullptr;       // [nv, D] FP32 query views
  const float* q_inv = nullptr;   // [nv]
  const int32_t* q_code = nullptr;// [nv * ma]
  const int32_t* qoff = nullptr;  // [B+1] device
  const int32_t* vquery = nullptr;// [nv] query of each view
  unsigned long long* stats = nullptr;  // optional [8]: scanned bytes, pairs, rescore bytes, then the
                                        // rescore's items, kept items, candidate pairs, candidate rows,
                                        // rows of kept items
  KernelClock* kc = nullptr;            // optional kernel timing
  // derived
  int64_t nslots = 0;
  int32_t* skeys = nullptr;       // [nslots] codeword of each slot (ascending)
  int64_t* boff = nullptr;        // [K+1] slots of codeword k
  int32_t* slot_view = nullptr;   // [nslots]
  int32_t* view_slot = nullptr;   // [nv * ma]
  int64_t* runbase = nullptr;     // [nslots + 1] first table cell of each slot; [nslots] = cells in use
  int64_t* woff = nullptr;        // [K+1] scan work items per codeword (exclusive)
  int64_t upper_items = 0;        // bound on the number of scan work items
  int64_t table_upper = 0;        // bound on the table cells
  // slot-ordered two-part BF16 query rows, made by the first tensor-core pass
  // that needs them and reused by the next (scan, then rescore)
  mutable __nv_bfloat16* slot_hi = nullptr;
  mutable __nv_bfloat16* slot_lo = nullptr;
};

void fif_plan(const Index& ix, FifPlan& P, Scratch& sc, cudaStream_t s);
// clear the table cells the batch uses (runbase[nslots] of them; the table is
// allocated for table_upper)
void fif_zero_table(const FifPlan& P, uint32_t* table, cudaStream_t s);
void fif_scan(const Index& ix, const FifPlan& P, uint32_t* table, bool rescore,
              const int32_t* cand_sorted, int R, cudaStream_t s);
// tcgen05 scan of a BF16 or E4M3 store (rescore: two-part BF16, candidates only;
// table32 non-null: a BF16 store with its two-part rows scanned at FP32 level over
// every touched pair, which fills `table32` with the maxima of every run: the
// candidates and their scores both come from it, with no separate rescore)
void fif_scan_tc(const Index& ix, const FifPlan& P, uint32_t* table, bool rescore, const int32_t* cand_sorted,
                 int R, Scratch& sc, cudaStream_t s, uint32_t* table32 = nullptr);
// counts of the candidate work of a batch (stats [3..7]) without running the
// rescore: for the FP32-level pass over every touched pair of a BF16 store
void fif_rescore_stats(const Index& ix, const FifPlan& P, const int32_t* cand_sorted, int R, Scratch& sc,
                       cudaStream_t s);
void fif_combine(const Index& ix, const FifPlan& P, const uint32_t* table, float* S_dense,
                 const int32_t* cand_sorted, int R, float* cand_score, Scratch& sc, cudaStream_t s);

}  // namespace gift
