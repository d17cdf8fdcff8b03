// Host side of the engine GEMM (instantiations of GemmPolicy).
#include "tc_gemm.cuh"

namespace gift {

namespace {

template <int SPLIT>
void run_gemm(const CUtensorMap& tA, const CUtensorMap& tB, const CUtensorMap& tA2, const CUtensorMap& tB2, int64_t M,
              int64_t N, int K, float* C, int64_t ldc, int accumulate, int* err, cudaStream_t s) {
  GemmPolicy<SPLIT> p;
  p.M = M;
  p.N = N;
  p.nkb = (int)cdiv(K, tc::kTK);
  p.C = C;
  p.ldc = ldc;
  p.accumulate = accumulate;
  p.row_major = cdiv(M, tc::kTM) >= cdiv(N, 128);
  const int grid = (int)std::min<int64_t>(device_sm_count(), cdiv(M, tc::kTM) * cdiv(N, 128));
  tc::launch_engine(tA, tB, tA2, tB2, p, err, grid, s);
}

}  // namespace

void gemm_tc(const __nv_bfloat16* a_hi, const __nv_bfloat16* a_lo, int64_t M, int64_t a_rows_alloc, int64_t lda,
             const __nv_bfloat16* b_hi, const __nv_bfloat16* b_lo, int64_t N, int64_t b_rows_alloc, int64_t ldb, int K,
             float* C, int64_t ldc, int accumulate, int* err, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  GIFT_REQUIRE(a_lo != nullptr || b_lo == nullptr, "gemm_tc: a two-part B needs a two-part A");
  const CUtensorMap tA = make_tmap_bf16(a_hi, a_rows_alloc, K, tc::kTM, lda);
  const CUtensorMap tB = make_tmap_bf16(b_hi, b_rows_alloc, K, 128, ldb);
  if (a_lo && b_lo) {
    const CUtensorMap tA2 = make_tmap_bf16(a_lo, a_rows_alloc, K, tc::kTM, lda);
    const CUtensorMap tB2 = make_tmap_bf16(b_lo, b_rows_alloc, K, 128, ldb);
    run_gemm<3>(tA, tB, tA2, tB2, M, N, K, C, ldc, accumulate, err, s);
  } else if (a_lo) {
    const CUtensorMap tA2 = make_tmap_bf16(a_lo, a_rows_alloc, K, tc::kTM, lda);
    run_gemm<2>(tA, tB, tA2, tB, M, N, K, C, ldc, accumulate, err, s);
  } else {
    run_gemm<1>(tA, tB, tA, tB, M, N, K, C, ldc, accumulate, err, s);
  }
}

}  // namespace gift
